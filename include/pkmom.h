/*
 * pkmom - GPU estimator of the power spectra of the discrete cosmic momentum
 * field with the FFT (Pan, arXiv:2005.06170), for NVIDIA GB300 (sm_103a).
 *
 * The estimator (paper Secs. 2 and 3):
 *   1. moments of the catalogue: total mass, bulk flow v_b, the velocity tensors
 *      behind the shot noise (Eqs. rawppnoise, rawPtheta, thetanoise);
 *   2. assignment of the mass density and the three mass-weighted momentum
 *      components to four periodic grids with the third-order Battle-Lemarie
 *      (BL) scaling function (Sec. 2.4.1, Eq. rawFFTed);
 *   3. a 3D real-to-complex FFT of each grid (Sec. 2.4.1);
 *   4. per Fourier mode, removal of the shot noise times sum_J W^2(k + 2 k_N J)
 *      and division by the window W^2(k) (Eqs. psn, rawPp, rawPtheta, rawPx),
 *      then averages in |k| shells of P_deltadelta, P_pp = <|p|^2>,
 *      P_thetatheta = theta_scale^2 <|k.p|^2> and Re P_deltatheta, with and
 *      without the bulk flow (Sec. 3: p' = p - (1 + delta) v_b).
 *
 * Conventions
 *   - Positions are in [0, L) or anywhere (wrapped periodically); the grid
 *     coordinate is u = x * (ng / L), formed in the catalogue's precision.
 *   - Grid layout: four real grids back to back, each ng x ng x (ng + 2) in C
 *     order (x slowest, z fastest; the z rows padded by two elements for the
 *     in-place R2C transform). After pkmom_fft each grid holds its half spectrum,
 *     ng x ng x (ng/2 + 1) complex values, in place. Grid 0 is the mass density,
 *     grids 1..3 the momentum components m v_x, m v_y, m v_z.
 *   - The BL kernel phi (B-spline order m) is realised exactly as the order-m
 *     B-spline assignment followed, in Fourier space, by the periodic factor
 *     prod_a Sigma_m(k_a dx)^{-1/2}; Sigma_m is the B-spline alias sum.
 *   - Spectra are in units of volume ((Mpc/h)^3 for L in Mpc/h) times the squared
 *     unit of the velocities for the momentum spectra; k in 1/(unit of L).
 *   - theta = i k.p * theta_scale (theta_scale = 1/(H a f) in the paper; 1 gives
 *     theta = -div p).
 *
 * Ownership: every buffer passed in is owned by the caller. A context owns its
 * cuFFT plans, its cached per-grid tables and, for pkmom_estimate and
 * pkmom_estimate_host(_async) only, the grids, scratch and staging it allocates on
 * first use.
 * All calls are asynchronous on the given CUDA stream (a cudaStream_t passed as
 * void*; NULL = legacy default stream) unless stated. Argument errors are
 * returned synchronously; a device-side error (a non-finite position) is latched
 * in the context and returned by pkmom_sync or by the next synchronising call.
 * A context is used from one host thread at a time, and the work it queues must not
 * overlap on the GPU across streams: its cached per-grid tables hold the binning's
 * work counters and per-item partial sums (order such calls on one stream, or use
 * one context per stream; pkmom_estimate_host_async overlaps only its own copies).
 */
#ifndef PKMOM_H
#define PKMOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pkmom_ctx pkmom_ctx;

typedef enum {
    PKMOM_OK = 0,
    PKMOM_EINVAL = -1,      /* bad argument (shape, null pointer, range) */
    PKMOM_ENOMEM = -2,      /* device allocation failed */
    PKMOM_ECUDA = -3,       /* CUDA runtime error */
    PKMOM_ECUFFT = -4,      /* cuFFT error */
    PKMOM_ETIMEOUT = -5,    /* reserved: a bounded device wait gave up */
    PKMOM_EUNSUPPORTED = -6,/* valid request this build does not support */
    PKMOM_ESCRATCH = -7,    /* scratch buffer smaller than pkmom_assign_scratch_bytes */
    PKMOM_EDATA = -8        /* the catalogue held non-finite or out-of-range positions */
} pkmom_status;

enum { PKMOM_F32 = 0, PKMOM_F64 = 1 };

/* Rows of the output array: out[row * nbins + bin]. */
enum {
    PKMOM_ROW_K = 0,        /* mode-weighted mean |k| of the shell */
    PKMOM_ROW_NMODES = 1,   /* number of Fourier modes (full sphere count) */
    PKMOM_ROW_PDD = 2,      /* density auto spectrum, shot noise V/N removed */
    PKMOM_ROW_PPP = 3,      /* momentum P_p (Eq. rawPp), shot noise V sigma_v^2/N removed */
    PKMOM_ROW_PTT = 4,      /* momentum divergence P_theta (Eq. rawPtheta) */
    PKMOM_ROW_PDT = 5,      /* Re P_delta-theta (Eq. rawPx), no shot noise in the real part */
    PKMOM_ROW_PPP_B = 6,    /* P_p' with the bulk flow removed (Sec. 3.1) */
    PKMOM_ROW_PTT_B = 7,    /* P_theta' (Sec. 3.2) */
    PKMOM_ROW_PDT_B = 8,    /* Re P_delta-theta' */
    PKMOM_ROW_SNDD = 9,     /* the subtracted shot noise, shell mean of SN/W^2 */
    PKMOM_ROW_SNPP = 10,
    PKMOM_ROW_SNTT = 11,
    PKMOM_ROW_SNPP_B = 12,
    PKMOM_ROW_SNTT_B = 13,
    PKMOM_NROWS = 14
};

/* Rows of the (|k|, mu)-binned output of pkmom_spectra_mu: out[row * ncells + cell],
 * cell = bin * nmu + mu_bin. Spectra with their shot noise removed; Re/Im of the complex
 * density x momentum-divergence cross spectrum in the paper's convention. */
enum {
    PKMOM_MU_ROW_K = 0,       /* mode-weighted mean |k| */
    PKMOM_MU_ROW_MU = 1,      /* mode-weighted mean mu */
    PKMOM_MU_ROW_NMODES = 2,  /* number of modes (full sphere, Nyquist modes left out) */
    PKMOM_MU_ROW_PDD = 3,
    PKMOM_MU_ROW_PPP = 4,
    PKMOM_MU_ROW_PTT = 5,     /* the theta shot noise k.Q.k depends on mu_b (Eq. thetanoise) */
    PKMOM_MU_ROW_RE_DT = 6,
    PKMOM_MU_ROW_IM_DT = 7,   /* -k mu_b (v_b/Haf) P with a bulk flow (Eq. bfpdpx) */
    PKMOM_MU_ROW_PPP_B = 8,   /* bulk flow removed (Sec. 3.1) */
    PKMOM_MU_ROW_PTT_B = 9,
    PKMOM_MU_ROW_RE_DT_B = 10,
    PKMOM_MU_ROW_IM_DT_B = 11,
    PKMOM_MU_ROW_RE_DPB_B = 12, /* Re P_delta p'_b, p'_b = p'.v_b/|v_b| (Eq. bfpp) */
    PKMOM_MU_ROW_SNDD = 13,   /* subtracted shot noise of P_dd */
    PKMOM_MU_ROW_SNTT = 14,   /* subtracted shot noise of P_theta */
    PKMOM_MU_ROW_IM_SNDT = 15,/* subtracted (imaginary) shot noise of P_delta-theta (Eq. rawPx) */
    PKMOM_MU_NROWS = 16
};

/* A particle catalogue. x,y,z,vx,vy,vz are element pointers with a common stride
 * in elements (1 for separate arrays, 3 for interleaved (n,3) position and
 * velocity arrays). mass may be NULL (unit masses). dtype is PKMOM_F32 or
 * PKMOM_F64 and must equal the precision in pkmom_params. Device pointers for
 * every call except pkmom_estimate_host(_async) (host pointers there). */
typedef struct {
    int64_t n;
    const void *x, *y, *z, *vx, *vy, *vz;
    const void *mass;
    int64_t stride;
    int dtype;
} pkmom_catalog;

/* What to estimate. Zero-initialise and fill; pkmom_params_default sets the
 * paper's choices. */
typedef struct {
    double box_L;            /* side of the periodic box (> 0) */
    int ng;                  /* grid points per side: a multiple of 8 in 16..1024 */
    int order;               /* B-spline order m of the BL kernel: 1..5 (4 = BL3, default). With
                                the exact deconvolution the order-m estimate equals that of the
                                plain order-m B-spline with its exact alias-sum shot noise (5: the
                                fifth-order B-spline the paper compares BL3 with, Sec. 2.4.1) */
    int precision;           /* PKMOM_F32 (FP32 grids and FFT) or PKMOM_F64 */
    int nbins;               /* number of linear |k| shells, 1..1024 */
    double kmin_kf;          /* shell range in units of k_f = 2 pi / L; kmin_kf <= 0 means 1 */
    double kmax_kf;          /* kmax_kf <= 0 means ng/2 (Nyquist); must be <= ng/2 */
    double theta_scale;      /* theta = i k.p * theta_scale; 1/(H a f) in the paper */
    int subtract_shot_noise; /* 1: remove the shot noise (default), 0: raw / W^2 */
    int bulk;                /* 1: also the bulk-flow-subtracted spectra (rows 6-8, 12-13) */
    int theta_sn_mode;       /* 0: exact per-mode k.Q.k noise (default), 1: isotropic sigma^2/3 */
    int bl_radius;           /* 0: the exact BL kernel (B-spline deposit, Fourier-space factor;
                                default). R in 2..4: the BL function truncated to |x| < R cells,
                                deposited directly in real space (the literal stencil of
                                Sec. 2.4.1; (2R)^3 nodes per particle), then divided by the
                                same window W^2; order must be 4 */
} pkmom_params;

/* Catalogue moments written by pkmom_assign (device memory, 16 doubles):
 * M = sum m, S2 = sum m^2, sum m v (3), R = sum m^2 v (3),
 * Q = sum m^2 v v^T (xx, yy, zz, xy, xz, yz), n, and one spare. FP64. */
typedef struct {
    double M, S2, mv[3], R[3], Q[6], n, spare;
} pkmom_moments;

void pkmom_params_default(pkmom_params *p, double box_L, int ng, int nbins);

/* Create a context on CUDA device `device` (made current for the calling thread). */
pkmom_status pkmom_create(pkmom_ctx **ctx, int device);
pkmom_status pkmom_destroy(pkmom_ctx *ctx);
const char *pkmom_strerror(pkmom_status s);
/* Text of the last error seen by this context (never NULL). */
const char *pkmom_last_error(const pkmom_ctx *ctx);

/* Bytes of the four padded grids for (ng, precision). */
size_t pkmom_grid_bytes(int ng, int precision);
/* Bytes of scratch pkmom_assign needs for n particles with these params. */
size_t pkmom_assign_scratch_bytes(const pkmom_params *p, int64_t n);
/* Device bytes pkmom_estimate holds for a request (grids + scratch + plan
 * workspace estimate + staging of the catalogue for pkmom_estimate_host). */
size_t pkmom_footprint_bytes(const pkmom_params *p, int64_t n);

/* Steps 1-2 (Secs. 2.1-2.2, 2.4.1): moments of the catalogue into *moments_dev
 * (a device pkmom_moments) and the B-spline assignment of (m, m v) onto the four
 * grids at `grids` (pkmom_grid_bytes bytes, device, 16-byte aligned; every real
 * element is written, the two padding elements of each row are not). `scratch` is
 * 16-byte aligned device memory of at least pkmom_assign_scratch_bytes bytes (else
 * PKMOM_ESCRATCH). Misaligned grids or scratch give PKMOM_EINVAL. */
pkmom_status pkmom_assign(pkmom_ctx *ctx, const pkmom_catalog *cat, const pkmom_params *p,
                          void *grids, void *moments_dev, void *scratch, size_t scratch_bytes,
                          void *stream);

/* Step 3 (Sec. 2.4.1): in-place 3D R2C FFT (e^{-ikx}, unnormalised) of the four
 * grids. The first call for a given (ng, precision) creates and caches a cuFFT
 * plan (this allocates; call once before any stream capture). */
pkmom_status pkmom_fft(pkmom_ctx *ctx, const pkmom_params *p, void *grids, void *stream);

/* Step 4 (Eqs. psn, rawPp, rawPtheta, rawPx, bfpp, bfpdpx): shell-averaged
 * spectra from the transformed grids and the moments, into out_dev (device,
 * PKMOM_NROWS * nbins doubles, layout out[row * nbins + bin]). Empty shells give
 * NaN. The first call for a given (ng, order, nbins, range) builds and caches
 * the per-shell mode tables (allocates; call once before any stream capture). */
pkmom_status pkmom_spectra(pkmom_ctx *ctx, const pkmom_params *p, const void *grids,
                           const void *moments_dev, double *out_dev, void *stream);

/* Step 4 in bins of |k| (the shells of p) and of mu = k.e/(|k| |e|), nmu linear bins on
 * [-1, 1]: the direction-dependent parts that shell averages cancel, the imaginary
 * cross spectrum -i k mu_b (v_b/Haf) P of a bulk flow and the mu_b-dependent shot noise
 * of theta (Sec. 2.2 Eq. thetanoise, Sec. 3.2 Eq. bfpdpx, Fig. bfPpdiff). direction: 3
 * host doubles (any length > 0), or NULL for the catalogue's bulk flow. Each mode is
 * counted once over the full sphere; modes with a Nyquist component (no direction
 * sign) are left out. The mu bin is decided in FP32: m = floor((mu + 1) nmu/2) with
 * mu = ((n0 e0 + n1 e1) + n2 e2) / sqrt(|n|^2), e normalised in FP64 and rounded to
 * FP32. out_dev: device, PKMOM_MU_NROWS * nbins * nmu doubles; empty cells give NaN.
 * nmu in 1..64 (PKMOM_EINVAL otherwise). Allocates context-owned work arrays on first
 * use (and when larger ones are needed). */
pkmom_status pkmom_spectra_mu(pkmom_ctx *ctx, const pkmom_params *p, const void *grids, const void *moments_dev,
                              const double *direction, int nmu, double *out_dev, void *stream);

/* Steps 1-4 on a device catalogue, with grids and scratch owned by the context
 * (allocated on first use and grown when needed). out_dev as for pkmom_spectra. */
pkmom_status pkmom_estimate(pkmom_ctx *ctx, const pkmom_catalog *cat, const pkmom_params *p,
                            double *out_dev, void *stream);

/* Steps 1-4 on a HOST catalogue: copies the arrays to context-owned device
 * memory (cudaMemcpyAsync; pinned host memory makes the copies asynchronous and
 * fast), runs pkmom_estimate and copies the PKMOM_NROWS * nbins result to the
 * host array out_host. Synchronises the stream before returning. */
pkmom_status pkmom_estimate_host(pkmom_ctx *ctx, const pkmom_catalog *cat_host, const pkmom_params *p,
                                 double *out_host, void *stream);

/* Steps 1-4 on a HOST catalogue without waiting for them: the pipelined form of
 * pkmom_estimate_host for a stream of catalogues. The catalogue is copied (one
 * cudaMemcpyAsync per array) on a copy stream the context owns, into the one of two
 * context-owned device staging slots that the estimate before the previous one has
 * finished reading; the estimate runs on `stream` once its copy has landed, and its
 * PKMOM_NROWS * nbins result is copied to out_host on `stream`. So the copy of catalogue
 * i+1 overlaps the estimate of catalogue i. Returns at once with *ticket, the call's
 * sequence number on this context; pkmom_wait(ctx, ticket) waits for the result.
 * Until then the caller keeps cat_host's arrays unchanged and out_host alive. Host
 * arrays must be pinned (page-locked) for the copies to overlap the compute; pageable
 * memory gives correct results with the copies serialised. A context has one staging
 * pair and one set of grids: use one `stream` per context for these calls. */
pkmom_status pkmom_estimate_host_async(pkmom_ctx *ctx, const pkmom_catalog *cat_host, const pkmom_params *p,
                                       double *out_host, void *stream, int64_t *ticket);

/* Waits until the result of the pkmom_estimate_host_async call numbered `ticket` is in
 * its out_host array (and every earlier call's result is in its own), then returns any
 * device-side data error latched by the estimates finished so far (PKMOM_EDATA).
 * PKMOM_EINVAL for a ticket this context has not issued. */
pkmom_status pkmom_wait(pkmom_ctx *ctx, int64_t ticket);

/* Step 4 like pkmom_spectra, for callers that cannot allocate device memory: a host
 * application that owns a fixed device pool and forbids allocator calls, or a plug-in
 * that runs inside another program and must not grow its footprint or call into its
 * allocator. This one entry point has no counterpart
 * in the paper: it exists only so that such callers can run the binning step.
 * It allocates nothing: its scratch (shell table, window tables, partial and shell
 * sums) is one file-scope device array of 4 MiB, held by every GPU that loads the
 * library until the process exits. grids, moments_dev and out_dev are as for
 * pkmom_spectra (caller-owned device memory). Limits: nbins <= 256 and the tables for
 * ng <= 1024 must fit in 4 MiB (PKMOM_EUNSUPPORTED otherwise); other argument errors
 * give PKMOM_EINVAL, CUDA errors PKMOM_ECUDA. The first call on a device looks up the
 * array's device address for that device (the device must be current; make that
 * first call before any stream capture). Every call rebuilds what it reads in the
 * shared array, but calls whose work overlaps on the GPU race on it: order them on
 * one stream. No context is used. */
pkmom_status pkmom_spectra_static(const pkmom_params *p, const void *grids, const void *moments_dev,
                                  double *out_dev, void *stream);

/* One catalogue of a batched estimate (pkmom_estimate_batch): the device catalogue, its
 * parameters, the caller-owned device buffers its steps write (as for pkmom_assign and
 * pkmom_spectra) and its deposit tuning (pkmom_set_tuning's values; -1: automatic). */
typedef struct {
    pkmom_catalog cat;
    pkmom_params p;
    void *grids;          /* pkmom_grid_bytes(p.ng, p.precision) bytes, 16-byte aligned */
    void *moments_dev;    /* 16 doubles */
    void *scratch;        /* pkmom_assign_scratch_bytes_tuned for this tuning, 16-byte aligned */
    size_t scratch_bytes;
    double *out_dev;      /* PKMOM_NROWS * p.nbins doubles */
    int deposit_tile, list_cap;
} pkmom_batch_item;

enum { PKMOM_BATCH_MAX = 128 };

/* Device bytes of the work buffer pkmom_estimate_batch needs for these items (0 for bad
 * arguments): per FP32 catalogue its binning partials (ng * nbins * 7 doubles) and shell
 * sums, and a work counter. */
size_t pkmom_batch_work_bytes(int n, const pkmom_batch_item *items);

/* Steps 1-4 of n <= PKMOM_BATCH_MAX catalogues of any sizes in one launch sequence on one
 * stream (the batched workload of many catalogues): the moments and sort of each
 * catalogue; ONE persistent deposit kernel over the tiles of every catalogue that takes
 * the 16^3 gather deposit (cubic order, FP32, exact BL kernel; each CTA takes (catalogue,
 * tile) items from a work counter until none is left, with no waits between items), the
 * others deposited one by one; the FFTs; ONE persistent binning kernel over the (slab,
 * shell) items of every FP32 catalogue, the FP64 ones binned one by one. Each result
 * equals pkmom_estimate's on that catalogue with the same tuning. work: device memory of
 * at least pkmom_batch_work_bytes (else PKMOM_ESCRATCH). The first call for a grid size
 * builds its cuFFT plan and tables (this allocates; call once before any stream
 * capture); later calls allocate nothing and can be captured. */
pkmom_status pkmom_estimate_batch(pkmom_ctx *ctx, int n, const pkmom_batch_item *items, void *work,
                                  size_t work_bytes, void *stream);

/* Wait for the stream and return any latched device-side error (PKMOM_EDATA). */
pkmom_status pkmom_sync(pkmom_ctx *ctx, void *stream);

/* Per-stage timing with CUDA events recorded on the launching stream. When on,
 * every pkmom_assign/fft/spectra call records start/stop events around each
 * stage; pkmom_timing_read synchronises on the last events and returns the
 * accumulated milliseconds and call counts per stage, then resets them.
 * Stages: 0 histogram, 1 scan, 2 scatter (sort) and moments, 3 deposit, 4 FFT,
 * 5 deconvolution+binning, 6 finalize. */
enum { PKMOM_STAGE_HIST = 0, PKMOM_STAGE_SCAN, PKMOM_STAGE_SCATTER, PKMOM_STAGE_DEPOSIT,
       PKMOM_STAGE_FFT, PKMOM_STAGE_BIN, PKMOM_STAGE_FINAL, PKMOM_NSTAGES };
pkmom_status pkmom_timing_enable(pkmom_ctx *ctx, int on);
pkmom_status pkmom_timing_read(pkmom_ctx *ctx, double ms[PKMOM_NSTAGES], int64_t calls[PKMOM_NSTAGES]);

/* Number of kernels this context has launched (its own kernels; cuFFT's not counted). */
int64_t pkmom_kernel_launches(const pkmom_ctx *ctx);

/* 1 for the checked build (libpkmom_checked.so), 0 otherwise. The checked build tests
 * every grid, halo, shared-buffer, sort-key, record and bin index before its access,
 * skips the access when the test fails and reports it as PKMOM_EDATA from pkmom_sync
 * (or the next synchronising call); the same results otherwise, more slowly. */
int pkmom_checked(void);

/* Checked build only (PKMOM_EUNSUPPORTED otherwise): launches one kernel whose single
 * index test fails on purpose (no access follows it), so that the next pkmom_sync
 * returns PKMOM_EDATA: a test of the reporting path. */
pkmom_status pkmom_checked_selftest(pkmom_ctx *ctx, void *stream);

/* Device bytes this context holds now: the workspaces of its cached cuFFT plans, its
 * cached per-grid tables and the buffers that pkmom_estimate, pkmom_estimate_host(_async)
 * and pkmom_spectra_mu own. A caller that budgets device memory (the serving loop)
 * charges these beside the buffers it passes in. */
size_t pkmom_context_bytes(const pkmom_ctx *ctx);

/* Tuning knobs of the assignment (used by the autotuner): deposit tile shape id
 * (0: 16x16x16, 1: 16x16x32, 2: 8x8x32, 3: 8x8x8 for FP32 grids; 4: 8x8x16, 5: 16^3,
 * 6: 8^3 for FP64; a shape that does not divide ng is ignored) and the capacity of the
 * per-tile shared-memory particle list of FP32 deposits (0 = none, at most 8192).
 * -1 restores the automatic choice. The results do not depend on these. */
pkmom_status pkmom_set_tuning(pkmom_ctx *ctx, int deposit_tile, int list_cap);
/* pkmom_assign_scratch_bytes under this context's tuning. */
size_t pkmom_assign_scratch_bytes_tuned(const pkmom_ctx *ctx, const pkmom_params *p, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* PKMOM_H */
