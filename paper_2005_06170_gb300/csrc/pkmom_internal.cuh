// Internal declarations shared by the CUDA translation units of libpkmom.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pkmom.h"
#include "shells.h"

// Checked builds (compiled with -DPKMOM_CHECKED=1 into libpkmom_checked.so): every
// grid, halo, shared-buffer, sort-key, record and bin index is tested before its access;
// a failed test sets its code in the translation unit's device error word (check_index,
// defined in each .cu) and the access is skipped, so nothing is read or written out of
// range. pkmom_sync reports a set word as PKMOM_EDATA. In unchecked builds PK_IN is true.
#ifndef PKMOM_CHECKED
#define PKMOM_CHECKED 0
#endif
#if PKMOM_CHECKED
#define PK_IN(i, n, code) check_index(static_cast<long long>(i), static_cast<long long>(n), (code))
#else
#define PK_IN(i, n, code) true
#endif

namespace pkmom {

// Codes of the checked build's index tests (bits of the device error word).
enum : unsigned {
    kChkKey = 1u,        // sort key beyond the key table
    kChkRecord = 2u,     // record slot beyond the catalogue
    kChkGrid = 4u,       // grid element beyond a grid
    kChkShared = 8u,     // node beyond a shared accumulator
    kChkHalo = 16u,      // halo scratch element beyond the scratch
    kChkMode = 32u,      // Fourier mode beyond a half spectrum
    kChkBin = 64u,       // shell or item beyond the partial sums
    kChkSelf = 1u << 31  // the self-test's deliberate failed test (no access follows it)
};
// Host: reads and clears the error word of assign.cu / spectra.cu (0 in unchecked builds).
unsigned take_check_word_assign();
unsigned take_check_word_spectra();
// Host: launches a kernel whose one index test fails on purpose (checked builds).
cudaError_t launch_check_selftest(cudaStream_t s);

// Number of doubles in a device pkmom_moments.
constexpr int kMomentWords = 16;
// Per-block moment partials: M, S2, mv[3], R[3], Q[6] = 14 values (padded to 16).
constexpr int kMomentVals = 14;
// Values accumulated per shell by the binning kernel:
// 0 |F_d|^2, 1 |F_p|^2, 2 |n.F_p|^2, 3 Im(conj F_d  n.F_p), 4-6 the same three
// for F_p' = F_p - v_b F_d. Each weighted by mode weight * g(n) = w / prod Bhat^2.
constexpr int kBinVals = 7;
// Data-independent per-shell sums: 0 sum w, 1 sum w |n|, 2 sum w h, 3-8 sum w h n_a n_b
// (xx, yy, zz, xy, xz, yz), h = prod Sigma / prod Bhat^2 = 1 / W^2.
constexpr int kModeVals = 9;

// One sorted particle: grid coordinates u (3) and the four deposited values
// (m, m vx, m vy, m vz). 32 bytes in FP32, 64 in FP64.
template <typename T> struct alignas(4 * sizeof(T)) Vec4 { T x, y, z, w; };
template <typename T> struct Record { Vec4<T> u; Vec4<T> q; };

// Host-side decisions for one assignment (see plan_assign in capi.cu).
struct AssignPlan {
    int ng = 0, order = 4, prec = PKMOM_F32;
    int bl_radius = 0;       // > 0: direct truncated BL deposit of this radius (cells)
    int sshift = 0;          // z-segment length S = 1 << sshift cells per sort key
    int64_t nkeys = 0;       // ng * ng * (ng >> sshift)
    int tile = 0;            // deposit tile id (see deposit launcher)
    int list_cap = 0;        // shared-memory particle list of an FP32 deposit tile (0 = none)
    int hist_blocks = 0;     // blocks of the moments+histogram kernel
    int64_t scan_blocks = 0; // blocks of the key scan
    size_t off_counts = 0, off_records = 0, off_partials = 0, off_blocksums = 0, off_qmax = 0;
    size_t off_halo = 0;     // home-tile deposit: per-tile halo nodes (0 = not used)
    size_t total = 0;
};

struct LaunchStats {
    int64_t launches = 0;
};

// One catalogue of a persistent batched gather deposit (16^3 tiles, cubic order, FP32):
// its sorted records, key table, largest |q| per field, grids and its first global tile.
struct FxJob {
    const Record<float> *rec;
    const uint32_t *offsets;
    const unsigned *qmax;
    float *grids;
    int64_t grid_elems;
    long long first_tile;
    int ng, sshift, list_cap, pad;
};
// The jobs of one launch, passed by value as the kernel's parameter (under 8 KB).
constexpr int kBatchMax = 128;
struct FxBatch {
    FxJob job[kBatchMax];
    int n;
    long long total_tiles;
};

// One catalogue of a persistent batched binning (FP32 grids): its transformed grids,
// moments, shell tables and its own per-item partial sums; its first global item.
struct BinJob {
    const void *grids;
    const double *mom;
    const int *thresh;
    const float *gf, *gh;
    double *partials;
    const uint32_t *order;  // the catalogue's non-empty items (SpectraTables::bin_order)
    long long first_item;   // of this catalogue in the batch's list of non-empty items
    int ng, nbins, nwork;
};
struct BinBatch {
    BinJob job[kBatchMax];
    int n;
    long long total_items;
    unsigned *counter;  // next item of the batch; zeroed before the launch
};

// ---------------------------------------------------------------- assign.cu
cudaError_t launch_hist_moments(const pkmom_catalog &cat, const AssignPlan &pl, double box_L, void *scratch,
                                int *err_flag, cudaStream_t s, LaunchStats &st);
cudaError_t launch_moments_final(const AssignPlan &pl, int64_t n, void *scratch, double *moments_dev,
                                 cudaStream_t s, LaunchStats &st);
cudaError_t launch_scan(const AssignPlan &pl, void *scratch, cudaStream_t s, LaunchStats &st);
cudaError_t launch_scatter(const pkmom_catalog &cat, const AssignPlan &pl, double box_L, void *scratch,
                           cudaStream_t s, LaunchStats &st);
cudaError_t launch_deposit(const AssignPlan &pl, void *scratch, void *grids, cudaStream_t s, LaunchStats &st);
// Whether launch_deposit_batch can take this assignment (16^3 gather tiles, cubic, FP32,
// exact BL kernel), and its FxJob (scratch and grids of that catalogue).
bool batchable_deposit(const AssignPlan &pl);
FxJob deposit_job(const AssignPlan &pl, void *scratch, void *grids);
// One persistent launch over the tiles of jobs[0 .. batch.n); counter: one device word.
cudaError_t launch_deposit_batch(FxBatch &batch, unsigned long long *counter, int num_sms, cudaStream_t s,
                                 LaunchStats &st);
// bytes of the key table (counts, then offsets) for nkeys sort keys
size_t key_table_bytes(int64_t nkeys);
// Tile shapes the deposit kernel is instantiated for (x, y, z nodes).
// Tile kHomeTile (16^3, FP32) deposits each particle once in the tile owning its cell
// (cubic order; it needs home_halo_bytes of scratch); other orders use the 16^3 gather.
constexpr int kHomeTile = 7;
size_t home_halo_bytes(int ng);
int deposit_tile_count();
void deposit_tile_shape(int tile, int prec, int dims[3]);

// ---------------------------------------------------------------- spectra.cu
struct SpectraTables {
    int ng = 0, order = 0, nbins = 0, prec = -1;
    bool direct = false;         // grids assigned with the BL function itself (no Fourier factor)
    double umin = 0, umax = 0;
    int nsq_max = 0;
    uint16_t *bintab = nullptr;  // [nsq_max + 1] shell of |n|^2, 0xFFFF outside
    int *thresh = nullptr;       // [nbins + 1] shell b: thresh[b] <= |n|^2 < thresh[b + 1]
    void *g_full = nullptr;      // [ng] 1/Bhat^2 per full axis (T = float or double)
    void *g_half = nullptr;      // [ng/2+1]
    double *h_full = nullptr;    // [ng] Sigma/Bhat^2 (FP64), for the mode tables
    double *h_half = nullptr;
    double *mode_sums = nullptr; // [kModeVals][nbins]
    double *partials = nullptr;  // [bin_blocks][kModeVals or kBinVals][nbins]
    int bin_blocks = 0;
    double *item_partials = nullptr;  // [ng * nbins][kBinVals] (shell-major binning)
    int shell_blocks = 0;
    // the (slab, shell) items that hold modes, i0 * nbins + b, slabs by increasing |n0|
    // (the larger items first); items missing from it are empty and never written
    uint32_t *bin_order = nullptr;
    int bin_nwork = 0;
    // next entry of bin_order and blocks done: [0, 2) for k_bin_shells, [2, 4) for k_bin_mu
    // (zero between launches)
    unsigned *bin_counter = nullptr;
    size_t bytes = 0;            // device bytes of all the arrays above
};
cudaError_t build_spectra_tables(SpectraTables &t, int ng, int order, bool direct, int nbins, double umin,
                                 double umax, int prec, int num_sms, cudaStream_t s, LaunchStats &st);
void free_spectra_tables(SpectraTables &t);
cudaError_t launch_bin(const SpectraTables &t, const void *grids, const double *moments_dev, cudaStream_t s,
                       LaunchStats &st);
cudaError_t launch_bin_shells(const SpectraTables &t, const void *grids, const double *moments_dev, cudaStream_t s,
                              LaunchStats &st);
// Persistent binning over the non-empty (slab, shell) items of many FP32 catalogues, each
// into its own partials (ng * nbins * kBinVals doubles), then per catalogue the
// fixed-order reduction into sums[kBinVals * nbins] (sums_of[k]) and the finalisation
// into out[k]. batch.counter: 4 bytes of device memory the call zeroes and uses.
cudaError_t launch_bin_batch(BinBatch &batch, const SpectraTables *const *tables, const pkmom_params *const *params,
                             double *const *sums_of, double *const *out, int num_sms, cudaStream_t s,
                             LaunchStats &st);
// sums_ready: the shell sums were already reduced (by launch_bin_shells); otherwise the
// per-block partials of launch_bin are reduced first
cudaError_t launch_finalize(const SpectraTables &t, const pkmom_params &p, const double *moments_dev,
                            double *out, cudaStream_t s, LaunchStats &st, bool sums_ready);

// (|k|, mu)-binned spectra: per-item partials (ng * nbins * nmu items) and cell sums
cudaError_t launch_spectra_mu(const SpectraTables &t, const pkmom_params &p, const void *grids,
                              const double *moments_dev, const double *dir, int nmu, double *partials, double *sums,
                              double *out, cudaStream_t s, LaunchStats &st);
size_t spectra_mu_partial_bytes(int ng, int nbins, int nmu);
size_t spectra_mu_sum_bytes(int nbins, int nmu);

}  // namespace pkmom
