// Steps 1-2 of the estimator on the GPU: catalogue moments and the B-spline
// assignment of mass and momentum to four periodic grids (paper Secs. 2.1-2.2,
// Eq. rawFFTed; the BL kernel's Fourier factor is applied in spectra.cu).
//
// Pipeline (all on one stream):
//   k_hist          the histogram of sort keys (key = x-row, y-row, z-segment of the
//                   cell), from the positions alone.
//   k_scan_*        exclusive scan of the key counts -> segment offsets.
//   k_scatter       writes each particle as a 32-byte record (grid coordinates and the
//                   four deposited values) at the slot an atomic increment of its key's
//                   cursor returns: a counting sort (any order within a key).
//   k_moments       FP64 moments (block partials) and max |q|, from velocities and masses.
//   k_moments_final fixed-order sum of the block partials -> pkmom_moments.
//   k_deposit_home  (FP32, cubic, >= 1/2 particle per cell) each particle deposited
//   + k_home_fixup  once by the tile owning its cell, halos added afterwards; otherwise
//   k_deposit(_fx)  one CTA per output tile gathers the particles of every segment whose
//                   stencils reach the tile, accumulates in shared memory, then writes
//                   each node of the tile exactly once. No global atomics, no zero fill.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <type_traits>
#include <utility>

#include "pkmom_internal.cuh"

namespace pkmom {

// ------------------------------------------------------------------ checked builds
namespace {
#if PKMOM_CHECKED
__device__ unsigned g_check_word;
__device__ __forceinline__ bool check_index(long long i, long long n, unsigned code)
{
    if (i >= 0 && i < n) return true;
    atomicOr(&g_check_word, code);
    return false;
}
#endif
}  // namespace

unsigned take_check_word_assign()
{
#if PKMOM_CHECKED
    unsigned w = 0;
    if (cudaMemcpyFromSymbol(&w, g_check_word, sizeof w) != cudaSuccess) return 0;
    if (w) {
        const unsigned zero = 0;
        cudaMemcpyToSymbol(g_check_word, &zero, sizeof zero);
    }
    return w;
#else
    return 0;
#endif
}

namespace {
// One index test that fails on purpose: index 1 against a bound of 1. The failed test
// records kChkSelf and no access follows it (checked builds; a no-op otherwise).
__global__ void k_check_selftest(int one)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && !PK_IN(one, one, kChkSelf)) return;
}
}  // namespace

cudaError_t launch_check_selftest(cudaStream_t s)
{
    k_check_selftest<<<1, 32, 0, s>>>(1);
    return cudaGetLastError();
}
namespace {

constexpr int kHistThreads = 256;
constexpr int kGroup = 16;  // particles per lane summed in the catalogue precision before a warp reduction

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// floor(u) wrapped into [0, ng); false for non-finite or huge |u|.
template <typename T>
__device__ __forceinline__ bool cell_of(T u, int ng, int &c)
{
    if (!(fabs(u) < T(1 << 30))) return false;
    int ic = static_cast<int>(floor(u));
    if (static_cast<unsigned>(ic) >= static_cast<unsigned>(ng)) {  // outside the box: wrap
        ic %= ng;
        ic = ic < 0 ? ic + ng : ic;
    }
    c = ic;
    return true;
}

// f(std::integral_constant<int, i>) for i = 0 .. N - 1, each i a compile-time constant
template <class F, int... I>
__device__ __forceinline__ void static_for_seq(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    static_for_seq(f, std::make_integer_sequence<int, N>{});
}

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// A record's fourth coordinate holds its wrapped cell (10 bits per axis, ng <= 1024):
// the bit pattern of an FP32 value, or the integer itself as an FP64 value.
template <typename T> __device__ __forceinline__ T pack_cell(int c0, int c1, int c2);
template <> __device__ __forceinline__ float pack_cell<float>(int c0, int c1, int c2)
{
    return __int_as_float(c0 | (c1 << 10) | (c2 << 20));
}
template <> __device__ __forceinline__ double pack_cell<double>(int c0, int c1, int c2)
{
    return static_cast<double>(c0 | (c1 << 10) | (c2 << 20));
}
__device__ __forceinline__ int unpack_cell(float v) { return __float_as_int(v); }
__device__ __forceinline__ int unpack_cell(double v) { return static_cast<int>(v); }

// The histogram of sort keys: positions only (12 bytes per FP32 particle), one
// fire-and-forget atomic increment per particle; non-finite or huge positions raise
// the data error flag. Two particles per iteration keep more loads in flight.
template <typename T>
__global__ void __launch_bounds__(kHistThreads)
k_hist(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z, int64_t stride, int64_t n,
       T scale, int ng, int sshift, uint32_t *__restrict__ counts, int *__restrict__ err)
{
    const int nseg = ng >> sshift;
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
    auto one = [&](int64_t i) {
        const int64_t j = i * stride;
        const T u0 = mul_rn(x[j], scale), u1 = mul_rn(y[j], scale), u2 = mul_rn(z[j], scale);
        int c0, c1, c2;
        if (cell_of(u0, ng, c0) & cell_of(u1, ng, c1) & cell_of(u2, ng, c2)) {
            const int64_t key = (static_cast<int64_t>(c0) * ng + c1) * nseg + (c2 >> sshift);
            if (PK_IN(key, static_cast<int64_t>(ng) * ng * nseg, kChkKey)) atomicAdd(counts + key, 1u);
        } else {
            *err = 1;
        }
    };
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += 2 * step) {
        one(i);
        if (i + step < n) one(i + step);
    }
}

__global__ void k_moments_final(const double *__restrict__ partials, int nblocks, int64_t n_particles,
                                double *__restrict__ out)
{
    // one warp per moment value, fixed summation order
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= kMomentVals) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partials[static_cast<int64_t>(b) * kMomentWords + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[k] = s;
    if (k == 0 && lane == 0) {
        out[kMomentVals] = static_cast<double>(n_particles);
        out[kMomentVals + 1] = 0.0;
    }
}

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 512;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // keys per block

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t &total)
{
    __shared__ uint32_t s_w[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? s_w[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_w[lane] = w;  // inclusive prefix of warp totals
    }
    __syncthreads();
    const uint32_t warp_base = warp ? s_w[warp - 1] : 0u;
    total = s_w[nw - 1];
    __syncthreads();
    return warp_base + inc - v;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t *__restrict__ counts, int64_t nkeys, uint32_t *__restrict__ blocksums)
{
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    uint32_t s = 0;
    if (base + kScanItems <= nkeys) {
        const uint4 *v4 = reinterpret_cast<const uint4 *>(counts + base);
#pragma unroll
        for (int k = 0; k < kScanItems / 4; ++k) {
            const uint4 q = v4[k];
            s += q.x + q.y + q.z + q.w;
        }
    } else {
        for (int k = 0; k < kScanItems; ++k)
            if (base + k < nkeys) s += counts[base + k];
    }
    uint32_t total;
    block_exclusive_scan(s, total);
    if (threadIdx.x == 0) blocksums[blockIdx.x] = total;
}

// One block: exclusive scan of the block sums in place; writes the grand total
// to counts[nkeys] (the end offset).
__global__ void __launch_bounds__(1024)
k_scan_top(uint32_t *__restrict__ blocksums, int64_t nblocks, uint32_t *__restrict__ counts, int64_t nkeys)
{
    const int64_t per = (nblocks + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = static_cast<int64_t>(threadIdx.x) * per;
    uint32_t s = 0;
    for (int64_t k = 0; k < per; ++k)
        if (b0 + k < nblocks) s += blocksums[b0 + k];
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, total);
    for (int64_t k = 0; k < per; ++k)
        if (b0 + k < nblocks) {
            const uint32_t v = blocksums[b0 + k];
            blocksums[b0 + k] = run;
            run += v;
        }
    if (threadIdx.x == 0) counts[nkeys] = total;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(uint32_t *__restrict__ counts, int64_t nkeys, const uint32_t *__restrict__ blocksums)
{
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
    const bool full = base + kScanItems <= nkeys;
    if (full) {
        const uint4 *v4 = reinterpret_cast<const uint4 *>(counts + base);
#pragma unroll
        for (int k = 0; k < kScanItems / 4; ++k) {
            const uint4 q = v4[k];
            v[4 * k] = q.x, v[4 * k + 1] = q.y, v[4 * k + 2] = q.z, v[4 * k + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = base + k < nkeys ? counts[base + k] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, total) + blocksums[blockIdx.x];
    if (full) {
        uint4 *o4 = reinterpret_cast<uint4 *>(counts + base);
#pragma unroll
        for (int k = 0; k < kScanItems / 4; ++k) {
            uint4 q;
            q.x = run, run += v[4 * k];
            q.y = run, run += v[4 * k + 1];
            q.z = run, run += v[4 * k + 2];
            q.w = run, run += v[4 * k + 3];
            o4[k] = q;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
            if (base + k < nkeys) {
                counts[base + k] = run;
                run += v[k];
            }
    }
}

// ------------------------------------------------------------------ moments
// The catalogue moments and the largest |q| of each deposited field, from velocities
// and masses alone: each lane sums kGroup particles in the catalogue precision (four
// per iteration, loads issued first), the warp adds its lanes' group sums (shuffles)
// and lane 0 adds them to FP64 accumulators, so that FP64 work is one add per value
// per 32 * kGroup particles; block sums go to partials[block] (k_moments_final).
template <typename T>
__global__ void __launch_bounds__(256)
k_moments(const T *__restrict__ vx, const T *__restrict__ vy, const T *__restrict__ vz, const T *__restrict__ mass,
          int64_t stride, int64_t n, double *__restrict__ partials, unsigned *__restrict__ qmax_bits)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double s_part[256 / 32][kMomentVals];  // per-warp FP64 sums
    if (lane < kMomentVals) s_part[warp][lane] = 0.0;
    __syncwarp();
    float qmax[4] = {0.f, 0.f, 0.f, 0.f};
    T grp[kMomentVals];
#pragma unroll
    for (int k = 0; k < kMomentVals; ++k) grp[k] = T(0);
    int gcount = 0;
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
    auto flush = [&]() {
#pragma unroll
        for (int k = 0; k < kMomentVals; ++k) {
            T v = grp[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s_part[warp][k] += static_cast<double>(v);
            grp[k] = T(0);
        }
    };
    auto add = [&](T m, T v0, T v1, T v2) {
        const T m2 = m * m;
        qmax[0] = fmaxf(qmax[0], static_cast<float>(fabs(m)));
        qmax[1] = fmaxf(qmax[1], static_cast<float>(fabs(m * v0)));
        qmax[2] = fmaxf(qmax[2], static_cast<float>(fabs(m * v1)));
        qmax[3] = fmaxf(qmax[3], static_cast<float>(fabs(m * v2)));
        grp[0] += m;
        grp[1] += m2;
        grp[2] += m * v0;
        grp[3] += m * v1;
        grp[4] += m * v2;
        grp[5] += m2 * v0;
        grp[6] += m2 * v1;
        grp[7] += m2 * v2;
        grp[8] += m2 * v0 * v0;
        grp[9] += m2 * v1 * v1;
        grp[10] += m2 * v2 * v2;
        grp[11] += m2 * v0 * v1;
        grp[12] += m2 * v0 * v2;
        grp[13] += m2 * v1 * v2;
    };
    // warp-uniform loop: every lane runs the same iterations (shuffles inside)
    for (int64_t wb = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); wb < n; wb += 4 * step) {
        T m[4], a[4], b[4], c[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t i = wb + k * step + lane;
            const bool ok = i < n;
            const int64_t j = ok ? i * stride : 0;
            m[k] = ok ? (mass ? mass[i] : T(1)) : T(0);  // absent particles add nothing
            a[k] = ok ? vx[j] : T(0);
            b[k] = ok ? vy[j] : T(0);
            c[k] = ok ? vz[j] : T(0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) add(m[k], a[k], b[k], c[k]);
        gcount += 4;
        if (gcount >= kGroup) {
            flush();
            gcount = 0;
        }
    }
    flush();
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        // non-negative floats order like their bit patterns
        const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(qmax[f]));
        if (lane == 0) atomicMax(qmax_bits + f, bits);
    }
    __syncthreads();
    if (threadIdx.x < kMomentVals) {
        double sum = 0.0;
        for (int w = 0; w < 256 / 32; ++w) sum += s_part[w][threadIdx.x];
        partials[static_cast<int64_t>(blockIdx.x) * kMomentWords + threadIdx.x] = sum;
    }
}

// FP32 interleaved (n, 3) velocities, 16-byte aligned: four particles per thread read
// as three 128-bit loads ((v0x v0y v0z v1x) (v1y v1z v2x v2y) (v2z v3x v3y v3z)), and
// four masses as one. The same sums as k_moments, kept by each lane in compensated
// (Kahan) FP32 pairs over all of its particles, so that no warp reduction waits inside
// the loop; each lane's pairs go to FP64 once at the end and are summed in a fixed
// order. The n % 4 last particles are added by the first lanes of block 0.
__global__ void __launch_bounds__(256)
k_moments_v3(const float *__restrict__ v, const float *__restrict__ mass, int64_t n,
             double *__restrict__ partials, unsigned *__restrict__ qmax_bits)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double s_part[256 / 32][kMomentVals];
    float qmax[4] = {0.f, 0.f, 0.f, 0.f};
    float sum[kMomentVals], cmp[kMomentVals];  // the sum of a value is sum - cmp
#pragma unroll
    for (int k = 0; k < kMomentVals; ++k) sum[k] = 0.f, cmp[k] = 0.f;
    const int64_t nq = n / 4;
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const float4 *v4 = reinterpret_cast<const float4 *>(v);
    const float4 *m4 = reinterpret_cast<const float4 *>(mass);
    auto kahan = [&](int k, float x) {
        const float y = __fsub_rn(x, cmp[k]);
        const float t = __fadd_rn(sum[k], y);
        cmp[k] = __fsub_rn(__fsub_rn(t, sum[k]), y);
        sum[k] = t;
    };
    auto add = [&](float m, float v0, float v1, float v2) {
        const float m2 = m * m;
        qmax[0] = fmaxf(qmax[0], fabsf(m));
        qmax[1] = fmaxf(qmax[1], fabsf(m * v0));
        qmax[2] = fmaxf(qmax[2], fabsf(m * v1));
        qmax[3] = fmaxf(qmax[3], fabsf(m * v2));
        kahan(0, m);
        kahan(1, m2);
        kahan(2, m * v0);
        kahan(3, m * v1);
        kahan(4, m * v2);
        kahan(5, m2 * v0);
        kahan(6, m2 * v1);
        kahan(7, m2 * v2);
        kahan(8, m2 * v0 * v0);
        kahan(9, m2 * v1 * v1);
        kahan(10, m2 * v2 * v2);
        kahan(11, m2 * v0 * v1);
        kahan(12, m2 * v0 * v2);
        kahan(13, m2 * v1 * v2);
    };
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < nq; q += step) {
        const float4 a = v4[3 * q], b = v4[3 * q + 1], c = v4[3 * q + 2];
        const float4 mm = mass ? m4[q] : make_float4(1.f, 1.f, 1.f, 1.f);
        add(mm.x, a.x, a.y, a.z);
        add(mm.y, a.w, b.x, b.y);
        add(mm.z, b.z, b.w, c.x);
        add(mm.w, c.y, c.z, c.w);
    }
    if (blockIdx.x == 0 && warp == 0) {
        const int64_t i = 4 * nq + lane;
        if (i < n) add(mass ? mass[i] : 1.f, v[3 * i], v[3 * i + 1], v[3 * i + 2]);
    }
#pragma unroll
    for (int k = 0; k < kMomentVals; ++k) {
        double x = static_cast<double>(sum[k]) - static_cast<double>(cmp[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_part[warp][k] = x;
    }
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const unsigned bits = __reduce_max_sync(0xffffffffu, __float_as_uint(qmax[f]));
        if (lane == 0) atomicMax(qmax_bits + f, bits);
    }
    __syncthreads();
    if (threadIdx.x < kMomentVals) {
        double total = 0.0;
        for (int w = 0; w < 256 / 32; ++w) total += s_part[w][threadIdx.x];
        partials[static_cast<int64_t>(blockIdx.x) * kMomentWords + threadIdx.x] = total;
    }
}

// ------------------------------------------------------------------ scatter
// Each particle is written as a 32-byte record at the slot an atomic increment of its
// key's cursor returns: a counting sort (any order within a key).
template <typename T>
__global__ void __launch_bounds__(256)
k_scatter(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z, const T *__restrict__ vx,
          const T *__restrict__ vy, const T *__restrict__ vz, const T *__restrict__ mass, int64_t stride, int64_t n,
          T scale, int ng, int sshift, uint32_t *__restrict__ cursor, Record<T> *__restrict__ rec)
{
    const int nseg = ng >> sshift;
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        const int64_t j = i * stride;
        const T u0 = mul_rn(x[j], scale), u1 = mul_rn(y[j], scale), u2 = mul_rn(z[j], scale);
        int c0, c1, c2;
        if (!(cell_of(u0, ng, c0) & cell_of(u1, ng, c1) & cell_of(u2, ng, c2))) continue;  // reported by k_hist
        const int64_t key = (static_cast<int64_t>(c0) * ng + c1) * nseg + (c2 >> sshift);
        if (!PK_IN(key, static_cast<int64_t>(ng) * ng * nseg, kChkKey)) continue;
        const uint32_t dst = atomicAdd(cursor + key, 1u);
        if (!PK_IN(dst, n, kChkRecord)) continue;
        const T m = mass ? mass[i] : T(1);
        Record<T> r;
        r.u = Vec4<T>{u0 - floor(u0), u1 - floor(u1), u2 - floor(u2), pack_cell<T>(c0, c1, c2)};
        r.q = Vec4<T>{m, m * vx[j], m * vy[j], m * vz[j]};
        rec[dst] = r;
    }
}

// ------------------------------------------------------------------ deposit
// B-spline weights of order M for a particle at fractional offset t = u - floor(u)
// in its cell; `first` receives the first node relative to floor(u).
// Offset from floor(u) of the first of the M nodes the order-M B-spline reaches for a
// particle at offset t in its cell (the convention of bspline_weights below).
template <int M, typename T>
__host__ __device__ constexpr int bspline_first(T t)
{
    if constexpr (M == 5) return t >= T(0.5) ? -1 : -2;
    else if constexpr (M == 4) return -1;
    else if constexpr (M == 3) return t >= T(0.5) ? 0 : -1;
    else if constexpr (M == 2) return 0;
    else return t >= T(0.5) ? 1 : 0;
}

template <int M, typename T>
__device__ __forceinline__ void bspline_weights(T t, T (&w)[M], int &first)
{
    first = bspline_first<M, T>(t);
    if constexpr (M == 4) {
        const T s = T(1) - t, t2 = t * t, t3 = t2 * t;
        const T sixth = T(1) / T(6);
        w[0] = s * s * s * sixth;
        w[1] = (T(3) * t3 - T(6) * t2 + T(4)) * sixth;
        w[2] = (T(-3) * t3 + T(3) * t2 + T(3) * t + T(1)) * sixth;
        w[3] = t3 * sixth;
    } else if constexpr (M == 5) {
        // the centred quartic B-spline at distances d + 2 .. d - 2 from the nearest node
        const bool up = t >= T(0.5);
        const T d = up ? t - T(1) : t;  // offset from the nearest node, in [-1/2, 1/2)
        const T d2 = d * d;
        auto mid = [](T x) {  // 1/2 <= x <= 3/2
            return (T(55) + x * (T(20) + x * (T(-120) + x * (T(80) + x * T(-16))))) / T(96);
        };
        const T lo = T(1) - T(2) * d, hi = T(1) + T(2) * d;
        w[0] = lo * lo * lo * lo / T(384);
        w[1] = mid(T(1) + d);
        w[2] = T(115) / T(192) - T(5) / T(8) * d2 + T(0.25) * d2 * d2;
        w[3] = mid(T(1) - d);
        w[4] = hi * hi * hi * hi / T(384);
    } else if constexpr (M == 3) {
        const bool up = t >= T(0.5);
        const T d = up ? t - T(1) : t;  // offset from the nearest node, in [-1/2, 1/2)
        const T a = T(0.5) - d, b = T(0.5) + d;
        w[0] = T(0.5) * a * a;
        w[1] = T(0.75) - d * d;
        w[2] = T(0.5) * b * b;
    } else if constexpr (M == 2) {
        w[0] = T(1) - t;
        w[1] = t;
    } else {
        w[0] = T(1);
    }
}

// Coefficients c_0..c_7 of the BL function phi = sum_n c_n B_4(. - n), c_{-n} = c_n
// (cubic order), set once per device by set_bl_coefficients.
__constant__ float c_bl_f[8];
__constant__ double c_bl_d[8];
template <typename T> __device__ __forceinline__ T bl_coef(int n);
template <> __device__ __forceinline__ float bl_coef<float>(int n) { return c_bl_f[n < 0 ? -n : n]; }
template <> __device__ __forceinline__ double bl_coef<double>(int n) { return c_bl_d[n < 0 ? -n : n]; }

// Weights of the BL function truncated to |x| < R cells (the direct real-space
// assignment of Sec. 2.4.1) for a particle at offset t in its cell: nodes floor(u) + k,
// k = 1 - R .. R. phi(t - k) = sum_j b_j(t) c_{j-1-k} with b_j the cubic B-spline
// weights of nodes floor(u) - 1 + j; zero where |t - k| >= R.
template <int R, typename T>
__device__ __forceinline__ void bl_weights(T t, T (&w)[2 * R], int &first)
{
    T b[4];
    int f4;
    bspline_weights<4, T>(t, b, f4);
    first = 1 - R;
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) {
        const int k = 1 - R + i;
        T v = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) v += b[j] * bl_coef<T>(j - 1 - k);
        w[i] = fabs(t - T(k)) < T(R) ? v : T(0);
    }
}

template <typename T, int M, int T0, int T1, int T2, int NT>
struct DepositCfg {
    static constexpr int HL = (M % 2 == 0) ? M / 2 : (M + 1) / 2;  // cells below the tile that reach it
    static constexpr int HR = (M % 2 == 0) ? M / 2 - 1 : (M - 1) / 2;
    static constexpr int R0 = T0 + HL + HR, R1 = T1 + HL + HR;
    static constexpr int MAXR = 2 * R0 * R1;  // up to two particle ranges per row
    static constexpr int TN = T0 * T1 * T2;
    static constexpr int IPT = (MAXR + NT - 1) / NT;
    static constexpr size_t smem = 4 * TN * sizeof(T);
};

// Largest product of three B-spline weights of order M: bounds any node value of the
// tile by this times (particles in the tile's reach) times max |q|.
template <int M> constexpr float kMaxWeight3 =
    M == 5 ? 0.2148770f : (M == 4 ? 0.2962963f : (M == 3 ? 0.421875f : 1.0f));
// The same for the BL function: max |phi| = phi(0) = 1.0890, cubed 1.2916.
constexpr float kMaxWeight3BL = 1.2917f;
template <int M, int BLR> constexpr float kMaxW3 = BLR > 0 ? kMaxWeight3BL : kMaxWeight3<M>;

// The particle index ranges of one tile: for every (x, y) cell row within reach of the
// tile, the sort-key segments covering the z cells within reach (one range, or two
// where the reach wraps around the periodic box). Fills s_beg[slot] and the exclusive
// prefix s_pre[slot] of the range lengths; returns the total particle count.
template <class C>
__device__ __forceinline__ uint32_t build_ranges(const uint32_t *__restrict__ offsets, int ng, int sshift, int t0,
                                                 int t1, int t2, int T2, uint32_t *s_beg, uint32_t *s_pre)
{
    const int S = 1 << sshift;
    const int nseg = ng >> sshift;
    const int r0n = C::R0 < ng ? C::R0 : ng;
    const int r1n = C::R1 < ng ? C::R1 : ng;
    const int nrows = r0n * r1n;
    const int zc = (T2 + C::HL + C::HR) < ng ? (T2 + C::HL + C::HR) : ng;
    int slo = 0, shi = nseg - 1;
    bool whole = zc == ng;
    if (!whole) {
        slo = floordiv(t2 - C::HL, S);
        shi = floordiv(t2 - C::HL + zc - 1, S);
        whole = shi - slo + 1 >= nseg;
        if (whole) slo = 0, shi = nseg - 1;
    }
    uint32_t lens[C::IPT];
    uint32_t my = 0;
#pragma unroll
    for (int k = 0; k < C::IPT; ++k) {
        const int slot = threadIdx.x * C::IPT + k;
        uint32_t beg = 0, len = 0;
        if (slot < 2 * nrows) {
            const int r = slot >> 1, second = slot & 1;
            int a0 = t0 - C::HL + r / r1n, a1 = t1 - C::HL + r % r1n;
            a0 = a0 < 0 ? a0 + ng : (a0 >= ng ? a0 - ng : a0);
            a1 = a1 < 0 ? a1 + ng : (a1 >= ng ? a1 - ng : a1);
            const int64_t base = (static_cast<int64_t>(a0) * ng + a1) * nseg;
            int lo = slo, hi = shi;  // segment range of this piece, inclusive
            bool use = !second;
            if (slo < 0) {
                if (second) lo = 0, hi = shi, use = true;
                else lo = slo + nseg, hi = nseg - 1;
            } else if (shi >= nseg) {
                if (second) lo = 0, hi = shi - nseg, use = true;
                else hi = nseg - 1;
            }
            if (use) {
                beg = offsets[base + lo];
                len = offsets[base + hi + 1] - beg;
            }
        }
        if (slot < C::MAXR) s_beg[slot] = beg;
        lens[k] = len;
        my += len;
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(my, total);
#pragma unroll
    for (int k = 0; k < C::IPT; ++k) {
        const int slot = threadIdx.x * C::IPT + k;
        if (slot < C::MAXR) s_pre[slot] = run;
        run += lens[k];
    }
    if (threadIdx.x == 0) s_pre[C::MAXR] = total;
    __syncthreads();
    return total;
}

// Last slot whose range starts at or before p (p < total).
template <int MAXR>
__device__ __forceinline__ int find_slot(const uint32_t *s_pre, uint32_t p)
{
    int lo = 0, hi = MAXR - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_pre[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Weights and tile-local node indices (-1 outside the tile) of one particle.
template <typename T, int M, int BLR = 0>
__device__ __forceinline__ void stencil(const Record<T> &r, int ng, int t0, int t1, int t2, int T0, int T1, int T2,
                                        T (&w)[3][M], int (&li)[3][M])
{
    const T t[3] = {r.u.x, r.u.y, r.u.z};  // offsets within the cells
    const int packed = unpack_cell(r.u.w);
    const int tb[3] = {t0, t1, t2};
    const int td[3] = {T0, T1, T2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int c = (packed >> (10 * a)) & 1023;
        int first;
        if constexpr (BLR > 0) bl_weights<BLR, T>(t[a], w[a], first);
        else bspline_weights<M, T>(t[a], w[a], first);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            int l = c + first + k - tb[a];
            l = l < 0 ? l + ng : (l >= ng ? l - ng : l);
            li[a][k] = l < td[a] ? l : -1;
        }
    }
}

// Weight and tile-local index of x node k0 (node floor(u) + 1 - R + k0) of the truncated
// BL stencil, formed on its own (the rolled x loop of the wide stencils); false if the
// node lies outside the tile or beyond the radius.
template <int R, typename T>
__device__ __forceinline__ bool bl_node_x(const Record<T> &r, int ng, int t0, int T0, int k0, T &w, int &l)
{
    const int k = 1 - R + k0;
    int lx = (unpack_cell(r.u.w) & 1023) + k - t0;
    lx = lx < 0 ? lx + ng : (lx >= ng ? lx - ng : lx);
    if (lx >= T0 || !(fabs(r.u.x - T(k)) < T(R))) return false;
    T b[4];
    int f4;
    bspline_weights<4, T>(r.u.x, b, f4);
    T v = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) v += b[j] * bl_coef<T>(j - 1 - k);
    w = v;
    l = lx;
    return true;
}

// Tile-gather deposit with shared-memory atomics in the grid precision (used for
// FP64 grids, where FP64 accuracy is required).
template <typename T, int M, int T0, int T1, int T2, int NT, int BLR = 0>
__global__ void __launch_bounds__(NT)
k_deposit(const Record<T> *__restrict__ rec, const uint32_t *__restrict__ offsets,
          const unsigned *__restrict__ /*qmax_bits*/, int ng, int sshift, T *__restrict__ grids, int64_t grid_elems,
          int /*list_cap*/)
{
    using C = DepositCfg<T, M, T0, T1, T2, NT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *acc = reinterpret_cast<T *>(smem_raw);  // [4][T0][T1][T2]
    __shared__ uint32_t s_beg[C::MAXR];
    __shared__ uint32_t s_pre[C::MAXR + 1];

    const int ntz = ng / T2, nty = ng / T1;
    int tile = blockIdx.x;
    const int tz = tile % ntz;
    tile /= ntz;
    const int ty = tile % nty;
    const int tx = tile / nty;
    const int t0 = tx * T0, t1 = ty * T1, t2 = tz * T2;
    for (int k = threadIdx.x; k < 4 * C::TN; k += NT) acc[k] = T(0);
    const uint32_t total = build_ranges<C>(offsets, ng, sshift, t0, t1, t2, T2, s_beg, s_pre);

    for (uint32_t p = threadIdx.x; p < total; p += NT) {
        const int slot = find_slot<C::MAXR>(s_pre, p);
        const Record<T> r = rec[s_beg[slot] + (p - s_pre[slot])];
        T w[3][M];
        int li[3][M];
        stencil<T, M, BLR>(r, ng, t0, t1, t2, T0, T1, T2, w, li);
        auto plane = [&](T wx, int lx) {  // the M x M (y, z) nodes of one x node
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                if (li[1][k1] < 0) continue;
                const T w01 = wx * w[1][k1];
                const int b01 = (lx * T1 + li[1][k1]) * T2;
#pragma unroll
                for (int k2 = 0; k2 < M; ++k2) {
                    if (li[2][k2] < 0) continue;
                    const T ww = w01 * w[2][k2];
                    T *a = acc + b01 + li[2][k2];
                    atomicAdd(a, r.q.x * ww);
                    atomicAdd(a + C::TN, r.q.y * ww);
                    atomicAdd(a + 2 * C::TN, r.q.z * ww);
                    atomicAdd(a + 3 * C::TN, r.q.w * ww);
                }
            }
        };
        if constexpr (BLR > 2) {  // wide stencils: rolled x loop (instruction cache)
            T wx;
            int lx;
#pragma unroll 1
            for (int k0 = 0; k0 < M; ++k0)
                if (bl_node_x<BLR, T>(r, ng, t0, T0, k0, wx, lx)) plane(wx, lx);
        } else {
#pragma unroll
            for (int k0 = 0; k0 < M; ++k0)
                if (li[0][k0] >= 0) plane(w[0][k0], li[0][k0]);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < C::TN; k += NT) {
        const int l2 = k % T2, l01 = k / T2;
        const int l1 = l01 % T1, l0 = l01 / T1;
        const int64_t gi = (static_cast<int64_t>(t0 + l0) * ng + (t1 + l1)) * (ng + 2) + t2 + l2;
        if (!PK_IN(gi, grid_elems, kChkGrid)) continue;
#pragma unroll
        for (int f = 0; f < 4; ++f) grids[f * grid_elems + gi] = acc[f * C::TN + k];
    }
}

// Cell-block path of the FP32 deposit for dense tiles (cubic order, per-cell keys): one
// warp per occupied cell of the reach; lane l owns stencil nodes (dx, dy, dz) with
// dz = l & 3, dy = (l >> 2) & 3, dx = (l >> 4) and (l >> 4) + 2, evaluates its weight
// pieces by Horner's rule with lane-constant coefficients, sums up to kCellFlush of the
// cell's particles (records read once, broadcast) in FP32 registers and adds the sums to
// the shared accumulator as fixed-point integers (one rounding per sum).
constexpr int kCellFlush = 256;

__device__ __forceinline__ float horner4(const float (&c)[4], float t) { return c[0] + t * (c[1] + t * (c[2] + t * c[3])); }

// coefficients of the cubic B-spline weight of stencil node k (0..3) in t = u - floor(u)
__device__ __forceinline__ void cubic_piece(int k, float (&c)[4])
{
    const float s = 1.0f / 6.0f;
    if (k == 0) c[0] = s, c[1] = -3 * s, c[2] = 3 * s, c[3] = -s;
    else if (k == 1) c[0] = 4 * s, c[1] = 0.f, c[2] = -6 * s, c[3] = 3 * s;
    else if (k == 2) c[0] = s, c[1] = 3 * s, c[2] = 3 * s, c[3] = -3 * s;
    else c[0] = 0.f, c[1] = 0.f, c[2] = 0.f, c[3] = s;
}

__device__ __forceinline__ int round_shift(int v, int d) { return d > 0 ? (v + (1 << (d - 1))) >> d : v; }

// Weight pieces of a lane's two stencil nodes (dx, dx + 2; dy; dz) in the cell-block paths.
struct CellPieces {
    float xa[4], xb[4], y[4], z[4];
};

// Sums of one chunk (at most kCellFlush particles) of a cell for a lane's two stencil
// nodes. Each contribution is rounded once to the fine scale 2^sf (below 2^22 in
// magnitude: one FFMA against 1.5 * 2^23) and added as an integer; the chunk sum is then
// rounded to the tile scale by a right shift of sf - st bits. Integer sums: the result
// does not depend on the order in which the sort left the cell's particles.
template <int F0 = 0, int NF = 4>
__device__ __forceinline__ void cell_chunk(const Record<float> *__restrict__ rec, uint32_t i0, uint32_t i1,
                                           const CellPieces &pc, const float (&fine)[4], const int (&shift)[4],
                                           int (&a)[NF], int (&b)[NF])
{
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
    constexpr int kMagicBits = 0x4B400000;
    int sa[NF], sb[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) sa[f] = 0, sb[f] = 0;
    auto add = [&](const Record<float> &rc) {
        const float wyz = horner4(pc.y, rc.u.y) * horner4(pc.z, rc.u.z);
        const float wa = horner4(pc.xa, rc.u.x) * wyz, wb = horner4(pc.xb, rc.u.x) * wyz;
        const float qv[4] = {rc.q.x, rc.q.y, rc.q.z, rc.q.w};
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            const float q = qv[F0 + f] * fine[F0 + f];
            sa[f] += __float_as_int(fmaf(q, wa, kMagic)) - kMagicBits;
            sb[f] += __float_as_int(fmaf(q, wb, kMagic)) - kMagicBits;
        }
    };
    uint32_t i = i0;
    for (; i + 4 <= i1; i += 4) {  // four loads in flight
        const Record<float> r0 = rec[i], r1 = rec[i + 1], r2 = rec[i + 2], r3 = rec[i + 3];
        add(r0);
        add(r1);
        add(r2);
        add(r3);
    }
    for (; i < i1; ++i) add(rec[i]);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        a[f] = round_shift(sa[f], shift[F0 + f]);
        b[f] = round_shift(sb[f], shift[F0 + f]);
    }
}

// Fixed-point scales of a tile: 2^st with (bound of any node sum) * 2^st < 2^30, and,
// for the cell-block paths, the fine scale 2^sf with (largest contribution) * 2^sf < 2^22
// and st <= sf. Per-particle paths round at 2^min(st, sf) directly. A node's integer sum
// is then below 2^30 plus half a unit per rounding (fewer than 2^31 particles), which
// fits a signed 32-bit accumulator.
__device__ __forceinline__ void tile_scales(float bound, float cmax, bool cells, float &scale, float &fine, int &shift)
{
    int eb = 0, ec = 0;
    if (bound > 0.f) frexpf(bound, &eb);  // bound < 2^eb
    if (cmax > 0.f) frexpf(cmax, &ec);
    if (!isfinite(bound)) eb = 150;
    if (!isfinite(cmax)) ec = 150;
    auto clampx = [](int e) { return e > 120 ? 120 : (e < -120 ? -120 : e); };
    const int sf = clampx(22 - ec), st = clampx(min(30 - eb, 22 - ec));
    scale = ldexpf(1.0f, st);
    fine = ldexpf(1.0f, sf);
    shift = cells ? min(30, sf - st) : 0;
}

template <int T0, int T1, int T2, int NT>
__device__ __forceinline__ void deposit_cells_path(const Record<float> *__restrict__ rec,
                                                   const uint32_t *__restrict__ offsets, int ng, int t0, int t1, int t2,
                                                   int *acc, int fstride, int px, int rw, const float *s_fine,
                                                   const int *s_shift)
{
    constexpr int HL = 2, R0 = T0 + 3, R1 = T1 + 3, RZ = T2 + 3, NW = NT / 32;
    const float fine[4] = {s_fine[0], s_fine[1], s_fine[2], s_fine[3]};
    const int shift[4] = {s_shift[0], s_shift[1], s_shift[2], s_shift[3]};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int dz = lane & 3, dy = (lane >> 2) & 3, dxl = lane >> 4;
    CellPieces pc;
    cubic_piece(dxl, pc.xa);
    cubic_piece(dxl + 2, pc.xb);
    cubic_piece(dy, pc.y);
    cubic_piece(dz, pc.z);
    auto wrapi = [ng](int a) { return a < 0 ? a + ng : (a >= ng ? a - ng : a); };
    for (int c = warp; c < R0 * R1 * RZ; c += NW) {
        const int r = c / RZ, zz = c % RZ;
        const int cx = r / R1 - HL, cy = r % R1 - HL, cz = zz - HL;  // cell relative to the tile
        const int64_t key =
            (static_cast<int64_t>(wrapi(t0 + cx)) * ng + wrapi(t1 + cy)) * ng + wrapi(t2 + cz);
        const uint32_t beg = offsets[key], end = offsets[key + 1];
        if (beg == end) continue;
        const int lxa = cx - 1 + dxl, lxb = lxa + 2, ly = cy - 1 + dy, lz = cz - 1 + dz;
        const bool yz = ly >= 0 && ly < T1 && lz >= 0 && lz < T2;
        const bool ina = yz && lxa >= 0 && lxa < T0, inb = yz && lxb >= 0 && lxb < T0;
        const int oa = lxa * px + ly * rw + lz, ob = (lxa + 2) * px + ly * rw + lz;
        for (uint32_t i0 = beg; i0 < end; i0 += kCellFlush) {
            int a[4], b[4];
            cell_chunk(rec, i0, min(end, i0 + kCellFlush), pc, fine, shift, a, b);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                if (ina) atomicAdd(acc + f * fstride + oa, a[f]);
                if (inb) atomicAdd(acc + f * fstride + ob, b[f]);
            }
        }
    }
}

// Shared accumulator of the FP32 gather deposit: int[4][T0][PX] per tile, node (x, y, z)
// at x * PX + y * RW + z. The row pitch RW = T2 + 1 is odd; the plane pitch PX = T1 * RW
// + 3 is odd as well, so that the bank of a node, (x PX + y RW + z) mod 32, mixes all
// three coordinates (with PX = 16 mod 32, as T1 * RW alone would give for 16 x 17, x
// would add only its parity).
//
// The listed path adds every stencil node of every particle, with the weights of nodes
// outside the tile set to zero (an add of exactly 0), at an address formed by the same
// linear rule; such a node lies at most 5 nodes below or 4 above the tile on each axis
// (orders 1 to 5), so the allocation has FRONT words of padding before the accumulator
// and at least BACK words after it (the particle list or padding). The zero adds land on
// padding, on other nodes or on list entries, and change none of them.
template <int T0, int T1, int T2>
struct FxLayout {
    static constexpr int RW = T2 + 1;
    static constexpr int PX = T1 * RW + 3;
    static constexpr int TNP = T0 * PX;  // ints per field
    static constexpr int FRONT = (5 * (PX + RW + 1) + 3) / 4 * 4;
    static constexpr int BACK = 4 * PX + (T1 + 4) * RW + T2 + 5;
    static size_t bytes(int list_cap)
    {
        return size_t(FRONT + 4 * TNP + (list_cap > BACK ? list_cap : BACK)) * sizeof(int);
    }
};

// Every node the listed path adds to (weights of nodes outside the tile zero) lies in the
// padded allocation: node coordinates run from -HL + first(0) to (T + HR - 1) + first(1/2)
// + M - 1 on each axis (first is smallest at t = 0 and largest from t = 1/2 on).
template <int M, int T0, int T1, int T2>
constexpr bool fx_pads_cover()
{
    using Lay = FxLayout<T0, T1, T2>;
    constexpr int HL = (M % 2 == 0) ? M / 2 : (M + 1) / 2;
    constexpr int HR = (M % 2 == 0) ? M / 2 - 1 : (M - 1) / 2;
    constexpr int lo = -HL + bspline_first<M, float>(0.0f);
    constexpr int up = HR - 1 + bspline_first<M, float>(0.5f) + M - 1;  // highest coordinate - T
    constexpr long min_lin = static_cast<long>(lo) * (Lay::PX + Lay::RW + 1);
    constexpr long max_lin = static_cast<long>(T0 + up) * Lay::PX + static_cast<long>(T1 + up) * Lay::RW + (T2 + up) +
                             3L * Lay::TNP;
    return min_lin >= -Lay::FRONT && max_lin < 4L * Lay::TNP + Lay::BACK;
}
template <int T0, int T1, int T2>
constexpr bool fx_pads_cover_orders()
{
    return fx_pads_cover<1, T0, T1, T2>() && fx_pads_cover<2, T0, T1, T2>() && fx_pads_cover<3, T0, T1, T2>() &&
           fx_pads_cover<4, T0, T1, T2>() && fx_pads_cover<5, T0, T1, T2>();
}
static_assert(fx_pads_cover_orders<16, 16, 16>() && fx_pads_cover_orders<16, 16, 32>() &&
                  fx_pads_cover_orders<8, 8, 32>() && fx_pads_cover_orders<8, 8, 8>(),
              "the padding of the gather accumulator must cover every node the listed path adds to");

// Four shared-memory adds at byte offsets OFF + f * FS (f = 0..3) from addr (the offsets
// are immediates).
template <int OFF, int FS>
__device__ __forceinline__ void red4(unsigned addr, int v0, int v1, int v2, int v3)
{
    asm volatile(
        "red.shared.add.s32 [%0+%5], %1;\n\t"
        "red.shared.add.s32 [%0+%6], %2;\n\t"
        "red.shared.add.s32 [%0+%7], %3;\n\t"
        "red.shared.add.s32 [%0+%8], %4;" ::"r"(addr),
        "r"(v0), "r"(v1), "r"(v2), "r"(v3), "n"(OFF), "n"(OFF + FS), "n"(OFF + 2 * FS), "n"(OFF + 3 * FS));
}

// Tile-local coordinates of the first stencil node of a particle in the tile's reach,
// where no periodic wrap falls inside the reach (ng >= tile + M cells): the cell offset
// from the tile's corner is taken into [-HL, T + HR).
template <int M, int HL, int HR, int T>
__device__ __forceinline__ int first_node(float t, int cell, int corner, int ng)
{
    int d = cell - corner;
    d = d < -HL ? d + ng : (d >= T + HR ? d - ng : d);
    return d + bspline_first<M, float>(t);
}

// One particle of the reordered list (see k_deposit_fx): its M^3 stencil nodes at
// immediate offsets from the shared-window address of its first node, with the weights of
// nodes outside the tile set to zero (no branch or predicate per node; see FxLayout). The
// contributions of the nodes in the tile are those of the per-node path.
template <int M, int T0, int T1, int T2, int HL, int HR>
__device__ __forceinline__ void banked_particle(const Record<float> &r, int ng, int t0, int t1, int t2, unsigned acc_s,
                                                float sc0, float sc1, float sc2, float sc3)
{
    using Lay = FxLayout<T0, T1, T2>;
    constexpr int RW = Lay::RW, PX = Lay::PX, TNP = Lay::TNP;
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
    constexpr int kMagicBits = 0x4B400000;
    const int packed = unpack_cell(r.u.w);
    float w[3][M];
    int first;
    bspline_weights<M, float>(r.u.x, w[0], first);
    bspline_weights<M, float>(r.u.y, w[1], first);
    bspline_weights<M, float>(r.u.z, w[2], first);
    const int b0 = first_node<M, HL, HR, T0>(r.u.x, packed & 1023, t0, ng);
    const int b1 = first_node<M, HL, HR, T1>(r.u.y, (packed >> 10) & 1023, t1, ng);
    const int b2 = first_node<M, HL, HR, T2>(r.u.z, (packed >> 20) & 1023, t2, ng);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        w[0][k] = static_cast<unsigned>(b0 + k) < static_cast<unsigned>(T0) ? w[0][k] : 0.0f;
        w[1][k] = static_cast<unsigned>(b1 + k) < static_cast<unsigned>(T1) ? w[1][k] : 0.0f;
        w[2][k] = static_cast<unsigned>(b2 + k) < static_cast<unsigned>(T2) ? w[2][k] : 0.0f;
    }
    // (the first node may lie below the accumulator, inside the front padding)
    // the first node where a particle of the tile's reach can have it (cell offset in
    // [-HL, T + HR) plus the first node's offset from the cell), which FxLayout's padding
    // covers (fx_pads_cover)
    constexpr int LO = -HL + bspline_first<M, float>(0.0f), HI = HR - 1 + bspline_first<M, float>(0.5f);
    if (!PK_IN(b0 - LO, T0 + HI - LO + 1, kChkShared) || !PK_IN(b1 - LO, T1 + HI - LO + 1, kChkShared) ||
        !PK_IN(b2 - LO, T2 + HI - LO + 1, kChkShared))
        return;
    const unsigned base = acc_s + 4u * static_cast<unsigned>(b0 * PX + b1 * RW + b2);
    const float q0 = r.q.x * sc0, q1 = r.q.y * sc1, q2 = r.q.z * sc2, q3 = r.q.w * sc3;
    auto row = [&](auto k0c, auto k1c) {
        constexpr int k0 = decltype(k0c)::value, k1 = decltype(k1c)::value;
        const float w01 = w[0][k0] * w[1][k1];
        auto node = [&](auto k2c) {
            constexpr int k2 = decltype(k2c)::value;
            const float ww = w01 * w[2][k2];
            red4<4 * (k0 * PX + k1 * RW + k2), 4 * TNP>(base, __float_as_int(fmaf(q0, ww, kMagic)) - kMagicBits,
                                                        __float_as_int(fmaf(q1, ww, kMagic)) - kMagicBits,
                                                        __float_as_int(fmaf(q2, ww, kMagic)) - kMagicBits,
                                                        __float_as_int(fmaf(q3, ww, kMagic)) - kMagicBits);
        };
        static_for<M>(node);
    };
    static_for<M>([&](auto k0c) { static_for<M>([&](auto k1c) { row(k0c, k1c); }); });
}

// Tile-gather deposit for FP32 grids with 32-bit integer (fixed-point) shared-memory
// atomics (about three times the throughput of FP32 shared atomics on this part).
//
// Work split: tiles whose reach holds few particles (sparse catalogues) list them in
// shared memory, reordered so that 32 consecutive entries have their first stencil nodes
// in different banks, and warps take consecutive chunks of 32 (banked_particle: every
// node at an immediate offset, nodes outside the tile adding exactly 0). Other
// tiles: each warp walks its own contiguous chunk of the tile's particle list 32 at a
// time, lane j taking the j-th particle of each step, node by node; tiles with more than
// two particles per reach cell (cubic order) take the cell-block path. The accumulator
// layout is FxLayout.
//
// Fixed point: field f of the tile uses the scale 2^s_f with
//   B_f 2^s_f < 2^30,   B_f = w3 * min(M^2 * largest row count, particle count) * max |q_f|
// over the tile's reach (w3 = the largest product of three weights; a node receives from
// at most M^2 cell rows, each contributing at most `largest row count` particles, and
// from no more than all of them; max |q_f| over the catalogue), so no node sum can overflow, and also max |q_f| w3 2^s_f < 2^22, so that
// every contribution is rounded to an integer by one FFMA against 1.5 * 2^23 (round to
// nearest even, one rounding of the exact product). The bound depends only on counts
// and maxima, and integer sums do not depend on order: the grids are the same whatever
// order the sort leaves particles of one cell in.
constexpr int kListRankMax = 128;  // largest bank group whose list entries are reordered

// One tile of the FP32 gather deposit (the body of k_deposit_fx, and of each work item
// of its persistent batched form k_deposit_fx_batch). The whole CTA takes part; its
// shared memory is free again when it returns.
template <int M, int T0, int T1, int T2, int NT, int BLR>
__device__ __forceinline__ void fx_tile(const Record<float> *__restrict__ rec, const uint32_t *__restrict__ offsets,
                                        const unsigned *__restrict__ qmax_bits, int ng, int sshift,
                                        float *__restrict__ grids, int64_t grid_elems, int list_cap, int tile)
{
    using C = DepositCfg<float, M, T0, T1, T2, NT>;
    using Lay = FxLayout<T0, T1, T2>;
    constexpr int RW = Lay::RW, PX = Lay::PX, TNP = Lay::TNP;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *acc = reinterpret_cast<int *>(smem_raw) + Lay::FRONT;  // [4][T0][PX], FxLayout
    __shared__ uint32_t s_beg[C::MAXR];
    __shared__ uint32_t s_pre[C::MAXR + 1];
    __shared__ unsigned s_rowmax;
    __shared__ float s_scale[4], s_fine[4];
    __shared__ int s_shift[4];
    __shared__ uint32_t s_bank[33];       // listed path: bank group counts, then the largest
    __shared__ uint32_t s_rbase[kListRankMax];  // entries before rank r of the reordered list
    __shared__ unsigned s_rmask[kListRankMax];  // bank groups with more than r entries

    const int ntz = ng / T2, nty = ng / T1;
    const int tz = tile % ntz;
    tile /= ntz;
    const int ty = tile % nty;
    const int tx = tile / nty;
    const int t0 = tx * T0, t1 = ty * T1, t2 = tz * T2;
    const float qm = threadIdx.x < 4 ? __uint_as_float(qmax_bits[threadIdx.x]) : 0.0f;  // used after the list
    for (int k = threadIdx.x; k < TNP; k += NT) reinterpret_cast<int4 *>(acc)[k] = make_int4(0, 0, 0, 0);
    if (threadIdx.x == 0) s_rowmax = 0;
    const uint32_t total = build_ranges<C>(offsets, ng, sshift, t0, t1, t2, T2, s_beg, s_pre);
    if (BLR > 0 && sshift == 0) {
        // the wide BL stencil: a node receives from M consecutive cells of each of M x M
        // cell rows, so bound with the largest count of M consecutive cells of a row
        // (per-cell keys: each row's offsets are cumulative along z)
        const int r0n = C::R0 < ng ? C::R0 : ng, r1n = C::R1 < ng ? C::R1 : ng;
        const int zc = (T2 + C::HL + C::HR) < ng ? (T2 + C::HL + C::HR) : ng;
        for (int r = threadIdx.x; r < r0n * r1n; r += NT) {
            int a0 = t0 - C::HL + r / r1n, a1 = t1 - C::HL + r % r1n;
            a0 = a0 < 0 ? a0 + ng : (a0 >= ng ? a0 - ng : a0);
            a1 = a1 < 0 ? a1 + ng : (a1 >= ng ? a1 - ng : a1);
            const int64_t base = (static_cast<int64_t>(a0) * ng + a1) * ng;
            uint32_t best = 0;
            for (int w0 = 0; w0 + M <= zc; ++w0) {
                int z = t2 - C::HL + w0;
                z = z < 0 ? z + ng : (z >= ng ? z - ng : z);
                const uint32_t c = z + M <= ng ? offsets[base + z + M] - offsets[base + z]
                                               : (offsets[base + ng] - offsets[base + z]) +
                                                     (offsets[base + z + M - ng] - offsets[base]);
                best = c > best ? c : best;
            }
            if (best) atomicMax(&s_rowmax, best);
        }
    } else {
        // largest row count: a row's two pieces are slots 2r and 2r + 1
        for (int r = threadIdx.x; 2 * r + 1 < C::MAXR + 1; r += NT) {
            const uint32_t c = s_pre[2 * r + 2 <= C::MAXR ? 2 * r + 2 : C::MAXR] - s_pre[2 * r];
            if (c) atomicMax(&s_rowmax, c);
        }
    }

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per_warp = ((total + NW - 1) / NW + 31u) & ~31u;
    const uint32_t wbeg = static_cast<uint32_t>(warp) * per_warp;
    const uint32_t wend = min(wbeg + per_warp, total);
    // flat list of the tile's record indices when it fits in the list_cap slots after
    // the accumulator (sparse catalogues: many short rows; no search per particle)
    uint32_t *s_idx = reinterpret_cast<uint32_t *>(acc + 4 * TNP);
    const bool listed = total <= static_cast<uint32_t>(list_cap);
    if (listed) {
        for (int slot = threadIdx.x; slot < C::MAXR; slot += NT) {
            const uint32_t b = s_beg[slot], p0 = s_pre[slot], p1 = s_pre[slot + 1];
            for (uint32_t p = p0; p < p1; ++p) s_idx[p] = b + (p - p0);
        }
        __syncthreads();
    }
    auto record_index = [&](uint32_t p, int &slot) -> uint32_t {
        if (listed) return s_idx[p];
        while (p >= s_pre[slot + 1]) ++slot;
        return s_beg[slot] + (p - s_pre[slot]);
    };

    // dense tiles (cubic order, more than two particles per reach cell on average) sum
    // each cell's particles in registers first (cell-block path below)
    constexpr int NREACH = C::R0 * C::R1 * (T2 + C::HL + C::HR);
    const bool dense = M == 4 && BLR == 0 && total > 2u * NREACH && sshift == 0 && ng >= C::R0 && ng >= C::R1 &&
                       ng >= T2 + C::HL + C::HR;
    // per-field scale from order-independent bounds only (so that the grids, and the
    // spectra, do not depend on the order in which sorted particles share a cell)
    __syncthreads();
    if (threadIdx.x < 4) {
        const int f = threadIdx.x;
        const float m = qm;  // max |q_f| over the catalogue, loaded at the start
        const float w3 = kMaxW3<M, BLR> * 1.0001f;
        const float reach = fminf(static_cast<float>(M * M) * static_cast<float>(s_rowmax), static_cast<float>(total));
        tile_scales(w3 * reach * m, w3 * m, dense, s_scale[f], s_fine[f], s_shift[f]);
    }
    __syncthreads();
    const float sc0 = s_scale[0], sc1 = s_scale[1], sc2 = s_scale[2], sc3 = s_scale[3];
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
    constexpr int kMagicBits = 0x4B400000;

    // Listed tiles with no periodic wrap inside the reach (ng >= tile + M cells) take the
    // listed path of banked_particle: every stencil node at an immediate offset from the
    // first node, nodes outside the tile adding exactly 0. A node's bank is the
    // first node's plus a constant, so the list is reordered by (rank within its bank
    // group, bank group): 32 consecutive entries then hold distinct first-node banks, or
    // span two ranks (at most two adds per bank), and warps take consecutive chunks of 32
    // (every lane busy). Each contribution is the same rounded integer as on the per-node
    // path, so the grids do not depend on the order.
    constexpr int KP = 8;       // listed particles placed per thread
    const bool banked = BLR == 0 && listed && !dense && total <= static_cast<uint32_t>(KP * NT) && sshift == 0 &&
                        ng >= C::R0 && ng >= C::R1 && ng >= T2 + C::HL + C::HR;
    if (banked) {
        if (threadIdx.x < 32) s_bank[threadIdx.x] = 0;
        __syncthreads();
        Vec4<float> u[KP];
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            const uint32_t p = threadIdx.x + k * NT;
            if (p < total) u[k] = rec[s_idx[p]].u;
        }
        int key[KP];  // bank group | rank << 5, -1 for no particle
#pragma unroll
        for (int k = 0; k < KP; ++k) {
            key[k] = -1;
            if (threadIdx.x + k * NT < total) {
                const int packed = unpack_cell(u[k].w);
                const int b0 = first_node<M, C::HL, C::HR, T0>(u[k].x, packed & 1023, t0, ng);
                const int b1 = first_node<M, C::HL, C::HR, T1>(u[k].y, (packed >> 10) & 1023, t1, ng);
                const int b2 = first_node<M, C::HL, C::HR, T2>(u[k].z, (packed >> 20) & 1023, t2, ng);
                const int g = (b0 * PX + b1 * RW + b2) & 31;
                key[k] = g | static_cast<int>(atomicAdd(&s_bank[g], 1u) << 5);
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const uint32_t mx = __reduce_max_sync(0xffffffffu, s_bank[lane]);
            if (lane == 0) s_bank[32] = mx;
        }
        __syncthreads();
        const uint32_t maxc = s_bank[32];
        if (maxc <= static_cast<uint32_t>(kListRankMax)) {
            // entries before (r, g): sum over groups of min(count, r), then the groups
            // below g with more than r entries
            for (uint32_t r = warp; r < maxc; r += NW) {
                const uint32_t c = s_bank[lane];
                const unsigned m = __ballot_sync(0xffffffffu, c > r);
                const uint32_t below = __reduce_add_sync(0xffffffffu, c < r ? c : r);
                if (lane == 0) s_rmask[r] = m, s_rbase[r] = below;
            }
            uint32_t idx[KP];
#pragma unroll
            for (int k = 0; k < KP; ++k) idx[k] = key[k] >= 0 ? s_idx[threadIdx.x + k * NT] : 0u;
            __syncthreads();
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                if (key[k] < 0) continue;
                const int g = key[k] & 31, r = key[k] >> 5;
                s_idx[s_rbase[r] + __popc(s_rmask[r] & ((1u << g) - 1u))] = idx[k];
            }
            __syncthreads();
        }
    }

    bool cells_done = false;
    if constexpr (BLR == 0) {
        if (banked) {
            const unsigned acc_s = static_cast<unsigned>(__cvta_generic_to_shared(acc));
            uint32_t p = threadIdx.x;  // warp w takes chunks w, w + NW, ... of 32 entries
            Record<float> nxt;
            if (p < total) nxt = rec[s_idx[p]];
            while (p < total) {
                const Record<float> rc = nxt;
                p += NT;
                if (p < total) nxt = rec[s_idx[p]];
                banked_particle<M, T0, T1, T2, C::HL, C::HR>(rc, ng, t0, t1, t2, acc_s, sc0, sc1, sc2, sc3);
            }
            cells_done = true;
        }
    }
    if constexpr (M == 4 && BLR == 0) {  // the cell-block path uses B-spline pieces
        if (dense) {
            deposit_cells_path<T0, T1, T2, NT>(rec, offsets, ng, t0, t1, t2, acc, TNP, PX, RW, s_fine, s_shift);
            cells_done = true;
        }
    }
    // pass 2: deposit, one particle per lane
    if (!cells_done) {
        int slot = (!listed && wbeg + lane < wend) ? find_slot<C::MAXR>(s_pre, wbeg + lane) : 0;
        for (uint32_t p = wbeg + lane; p < wend; p += 32) {
            const Record<float> rc = rec[record_index(p, slot)];
            float w[3][M];
            int li[3][M];
            stencil<float, M, BLR>(rc, ng, t0, t1, t2, T0, T1, T2, w, li);
            const float q0 = rc.q.x * sc0, q1 = rc.q.y * sc1, q2 = rc.q.z * sc2, q3 = rc.q.w * sc3;
            // the M x M (y, z) nodes of one x node
            auto plane = [&](float wx, int lx) {
#pragma unroll
                for (int k1 = 0; k1 < M; ++k1) {
                    if (li[1][k1] < 0) continue;
                    const float w01 = wx * w[1][k1];
                    const int b01 = lx * PX + li[1][k1] * RW;
#pragma unroll
                    for (int k2 = 0; k2 < M; ++k2) {
                        if (li[2][k2] < 0) continue;
                        const float ww = w01 * w[2][k2];
                        if (!PK_IN(b01 + li[2][k2], TNP, kChkShared)) continue;
                        int *a = acc + b01 + li[2][k2];
                        atomicAdd(a, __float_as_int(fmaf(q0, ww, kMagic)) - kMagicBits);
                        atomicAdd(a + TNP, __float_as_int(fmaf(q1, ww, kMagic)) - kMagicBits);
                        atomicAdd(a + 2 * TNP, __float_as_int(fmaf(q2, ww, kMagic)) - kMagicBits);
                        atomicAdd(a + 3 * TNP, __float_as_int(fmaf(q3, ww, kMagic)) - kMagicBits);
                    }
                }
            };
            if constexpr (BLR > 2) {
                // wide stencils: a rolled loop over x nodes keeps the code in the
                // instruction cache; each x weight is formed where it is used
                float wx;
                int lx;
#pragma unroll 1
                for (int k0 = 0; k0 < M; ++k0)
                    if (bl_node_x<BLR, float>(rc, ng, t0, T0, k0, wx, lx)) plane(wx, lx);
            } else {
#pragma unroll
                for (int k0 = 0; k0 < M; ++k0)
                    if (li[0][k0] >= 0) plane(w[0][k0], li[0][k0]);
            }
        }
    }
    __syncthreads();
    const float inv[4] = {1.0f / sc0, 1.0f / sc1, 1.0f / sc2, 1.0f / sc3};  // exact: powers of two
    if ((reinterpret_cast<uintptr_t>(grids) & 7u) == 0) {
        // two z-adjacent cells per thread, one 8-byte store per field (ng, the row pitch
        // ng + 2, t2 and the even l2 keep the pair aligned)
        for (int k = threadIdx.x; k < C::TN / 2; k += NT) {
            const int l2 = 2 * (k % (T2 / 2)), l01 = k / (T2 / 2);
            const int l1 = l01 % T1, l0 = l01 / T1;
            const int64_t gi = (static_cast<int64_t>(t0 + l0) * ng + (t1 + l1)) * (ng + 2) + t2 + l2;
            const int ai = l0 * PX + l1 * RW + l2;
            if (!PK_IN(gi + 1, grid_elems, kChkGrid) || !PK_IN(ai + 1, TNP, kChkShared)) continue;
#pragma unroll
            for (int f = 0; f < 4; ++f)
                *reinterpret_cast<float2 *>(grids + f * grid_elems + gi) =
                    make_float2(static_cast<float>(acc[f * TNP + ai]) * inv[f],
                                static_cast<float>(acc[f * TNP + ai + 1]) * inv[f]);
        }
    } else {
        for (int k = threadIdx.x; k < C::TN; k += NT) {
            const int l2 = k % T2, l01 = k / T2;
            const int l1 = l01 % T1, l0 = l01 / T1;
            const int64_t gi = (static_cast<int64_t>(t0 + l0) * ng + (t1 + l1)) * (ng + 2) + t2 + l2;
            const int ai = l0 * PX + l1 * RW + l2;
            if (!PK_IN(gi, grid_elems, kChkGrid) || !PK_IN(ai, TNP, kChkShared)) continue;
#pragma unroll
            for (int f = 0; f < 4; ++f) grids[f * grid_elems + gi] = static_cast<float>(acc[f * TNP + ai]) * inv[f];
        }
    }
}

// (16^3-cell and larger tiles: up to 128 registers, as shared memory already holds them to
// two per SM; 8^3 tiles: 64, for eight per SM)
template <int M, int T0, int T1, int T2, int NT, int BLR = 0>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : (NT >= 256 ? 2 : 8))
k_deposit_fx(const Record<float> *__restrict__ rec, const uint32_t *__restrict__ offsets,
             const unsigned *__restrict__ qmax_bits, int ng, int sshift, float *__restrict__ grids, int64_t grid_elems,
             int list_cap)
{
    fx_tile<M, T0, T1, T2, NT, BLR>(rec, offsets, qmax_bits, ng, sshift, grids, grid_elems, list_cap,
                                    static_cast<int>(blockIdx.x));
}

// Persistent form of the gather deposit over the tiles of many catalogues (the batched
// estimate): each CTA takes the next (catalogue, tile) item from a global counter until
// none is left. Items are independent (each writes its own tile of its own grids), so
// nothing waits on another item; the order items are taken in does not change any
// result. While a tile is deposited the CTA asks L2 to prefetch the key-table rows of
// the item after it (the rows its range search reads first).
template <int M, int T0, int T1, int T2, int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : (NT >= 256 ? 2 : 8))
k_deposit_fx_batch(const FxBatch jobs, unsigned long long *__restrict__ counter)
{
    __shared__ long long s_item[2];
    using C = DepositCfg<float, M, T0, T1, T2, NT>;
    auto job_of = [&](long long item) {
        int j = 0;
        while (j + 1 < jobs.n && jobs.job[j + 1].first_tile <= item) ++j;
        return j;
    };
    auto prefetch_rows = [&](long long item) {
        if (item >= jobs.total_tiles) return;
        const FxJob &jb = jobs.job[job_of(item)];
        const int ng = jb.ng, ntz = ng / T2, nty = ng / T1;
        int tile = static_cast<int>(item - jb.first_tile);
        const int tz = tile % ntz;
        tile /= ntz;
        const int ty = tile % nty, tx = tile / nty;
        const int nseg = ng >> jb.sshift;
        for (int r = threadIdx.x; r < C::R0 * C::R1; r += NT) {
            int a0 = tx * T0 - C::HL + r / C::R1, a1 = ty * T1 - C::HL + r % C::R1;
            a0 = a0 < 0 ? a0 + ng : (a0 >= ng ? a0 - ng : a0);
            a1 = a1 < 0 ? a1 + ng : (a1 >= ng ? a1 - ng : a1);
            const uint32_t *row = jb.offsets + (static_cast<int64_t>(a0) * ng + a1) * nseg + ((tz * T2) >> jb.sshift);
            asm volatile("prefetch.L2 [%0];" ::"l"(row));
        }
    };
    if (threadIdx.x == 0) s_item[0] = static_cast<long long>(atomicAdd(counter, 1ull));
    __syncthreads();
    long long item = s_item[0];
    int buf = 0;
    while (item < jobs.total_tiles) {
        if (threadIdx.x == 0) s_item[buf ^ 1] = static_cast<long long>(atomicAdd(counter, 1ull));
        __syncthreads();
        const long long next = s_item[buf ^ 1];
        prefetch_rows(next);
        const FxJob &jb = jobs.job[job_of(item)];
        fx_tile<M, T0, T1, T2, NT, 0>(jb.rec, jb.offsets, jb.qmax, jb.ng, jb.sshift, jb.grids, jb.grid_elems,
                                      jb.list_cap, static_cast<int>(item - jb.first_tile));
        __syncthreads();
        item = next;
        buf ^= 1;
    }
}

// ------------------------------------------------------------------ home-tile deposit
// FP32 grids, cubic order, catalogues with about half a particle per cell or more.
//
// Each CTA owns a tile of 16^3 cells and deposits only the particles of those cells
// (each particle once), into a shared buffer of the 19^3 nodes their stencils reach
// (nodes -1 .. 17 of the tile on each axis). The 16^3 nodes the tile owns are written
// to the grid; the 2763 halo nodes go to a per-tile scratch area, and k_home_fixup adds
// each neighbour's halo to the owned nodes it overlaps, in a fixed order (so the grids
// do not depend on scheduling).
//
// Lane mapping: a warp takes a block of 2 x 4 cell columns; lane (x, y, m) takes the
// first particles of cells z = 4m .. 4m + 3 of its column and sums their contributions
// to each node column's 7 z nodes in registers before adding them (home_quad), two
// fields' roundings per paired FMA (fma.rn.f32x2, each half the scalar FMA's result). The
// buffer's x pitch is 16 modulo 32 banks, its y pitch 19 and its z pitch 1, so the 32
// lanes of every add hit 32 different banks (checked at compile time below): one
// wavefront each. Particles beyond the first of a cell go to a per-warp queue and are
// deposited 32 at a time, one per lane.
// Tiles with more than two particles per cell, or 32 in some four consecutive cells of a
// column, take the cell-block path: one warp per cell, each contribution rounded at the
// fine scale (largest contribution < 2^22) and summed exactly, in 64-bit shared
// accumulators (two fields per pass), so that a dense node's error is that of its
// contributions' roundings alone. Tiles with under a quarter particle per cell take one
// particle per lane from the tile's list.
//
// Fixed point as in k_deposit_fx, with bounds over the home tile's own particles (the
// only ones the buffer receives): B_f = w3 * min(16 * largest 4-cell column window count,
// particle count) * max |q_f|.
constexpr int kHomeT = 16;                                      // tile edge in cells (= owned nodes)
constexpr int kHomeB = kHomeT + 3;                              // buffer edge in nodes
constexpr int kHomePY = kHomeB;                                 // buffer y pitch
constexpr int kHomePX = 368;                                    // buffer x pitch
constexpr int kHomeField = kHomeB * kHomePX;                    // ints per field
constexpr int kHomeHalo = kHomeB * kHomeB * kHomeB - kHomeT * kHomeT * kHomeT;  // 2763 halo nodes
constexpr int kHomeNT = 256;                                    // one thread per cell column of the tile
constexpr int kHomeNW = kHomeNT / 32;
constexpr int kHomeQ = 64;                                      // overflow queue entries per warp
constexpr size_t kHomeSmem = size_t(4) * kHomeField * sizeof(int);
static_assert(kHomePX % 32 == 16 && kHomePX >= kHomeB * kHomeB, "x-adjacent cells must be 16 banks apart");
static_assert(kHomeNT == kHomeT * kHomeT, "one thread per cell column");
static_assert(kHomeNW * kHomeQ <= 2 * kHomeNT + 1, "queues share the column-range arrays");

// Banks of the first stencil node of the 32 lanes of a four-cells-per-lane block (2 x 4
// columns, lane (x, y, m) at cells z = 4m .. 4m + 3): all different, so that every add
// of home_quad is one wavefront.
constexpr bool home_quad_banks_distinct()
{
    unsigned seen = 0;
    for (int lane = 0; lane < 32; ++lane) {
        const int m = lane & 3, y = (lane >> 2) & 3, x = lane >> 4;
        const unsigned bit = 1u << ((x * kHomePX + y * kHomePY + 4 * m) & 31);
        if (seen & bit) return false;
        seen |= bit;
    }
    return true;
}
static_assert(home_quad_banks_distinct(), "the 32 lanes of a home_quad add must hit 32 banks");
// home_quad's largest buffer index on each axis: cell 15 + node offset 3 in x and y,
// z = 4 * 3 + 6 (seven z nodes from the lane's first cell); all inside the 19-node edge
static_assert(kHomeT - 1 + 3 < kHomeB && 4 * 3 + 6 < kHomeB && kHomeT % 4 == 0 && kHomeT / 4 == 4,
              "home_quad's nodes must lie in the node buffer");

// Halo index of buffer node (bx, by, bz), at least one coordinate in {0, 17, 18}:
// first the three x planes (19 x 19 each), then the y planes of the inner x range
// (16 x 19), then the z planes of the inner x, y range (16 x 16).
__host__ __device__ constexpr int home_side(int b) { return b == 0 ? 0 : b - kHomeT; }  // 0, 17, 18 -> 0, 1, 2
__host__ __device__ constexpr int home_unside(int s) { return s == 0 ? 0 : s + kHomeT; }
__host__ __device__ constexpr int home_halo_index(int bx, int by, int bz)
{
    if (bx == 0 || bx > kHomeT) return (home_side(bx) * kHomeB + by) * kHomeB + bz;
    if (by == 0 || by > kHomeT) return 3 * kHomeB * kHomeB + ((bx - 1) * 3 + home_side(by)) * kHomeB + bz;
    return 3 * kHomeB * kHomeB + 3 * kHomeT * kHomeB + ((bx - 1) * kHomeT + (by - 1)) * 3 + home_side(bz);
}
__host__ __device__ constexpr void home_halo_node(int k, int &bx, int &by, int &bz)
{
    constexpr int nx = 3 * kHomeB * kHomeB, ny = 3 * kHomeT * kHomeB;
    if (k < nx) {
        bz = k % kHomeB;
        const int r = k / kHomeB;
        by = r % kHomeB;
        bx = home_unside(r / kHomeB);
    } else if (k < nx + ny) {
        k -= nx;
        bz = k % kHomeB;
        const int r = k / kHomeB;
        by = home_unside(r % 3);
        bx = r / 3 + 1;
    } else {
        k -= nx + ny;
        bz = home_unside(k % 3);
        const int r = k / 3;
        by = r % kHomeT + 1;
        bx = r / kHomeT + 1;
    }
}

// home_halo_node inverts home_halo_index over the 2763 halo nodes, and every node it
// gives has a coordinate on the halo (0, 17 or 18)
constexpr bool home_halo_bijective()
{
    for (int k = 0; k < kHomeHalo; ++k) {
        int bx = 0, by = 0, bz = 0;
        home_halo_node(k, bx, by, bz);
        const bool inner = bx >= 1 && bx <= kHomeT && by >= 1 && by <= kHomeT && bz >= 1 && bz <= kHomeT;
        if (inner || bx < 0 || bx >= kHomeB || by < 0 || by >= kHomeB || bz < 0 || bz >= kHomeB ||
            home_halo_index(bx, by, bz) != k)
            return false;
    }
    return true;
}
static_assert(home_halo_bijective(), "the halo scratch layout must be a bijection");

// Shared-memory add without a returned value (the accumulators are read only after a
// barrier): addr is a shared-window byte address.
__device__ __forceinline__ void red_shared_add(unsigned addr, int v)
{
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v));
}

// One particle of home cell (cx, cy, cz) (each 0..15) into the node buffer: node
// c - 1 + k of the tile is buffer index c + k.
__device__ __forceinline__ void home_particle(int *acc, const Record<float> &r, int cx, int cy, int cz, float sc0,
                                              float sc1, float sc2, float sc3)
{
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
    constexpr int kMagicBits = 0x4B400000;
    float wx[4], wy[4], wz[4];
    int first;
    bspline_weights<4, float>(r.u.x, wx, first);
    bspline_weights<4, float>(r.u.y, wy, first);
    bspline_weights<4, float>(r.u.z, wz, first);
    const float q0 = r.q.x * sc0, q1 = r.q.y * sc1, q2 = r.q.z * sc2, q3 = r.q.w * sc3;
    // its last stencil node (3, 3, 3 from the first) must lie in the node buffer
    if (!PK_IN((cx + 3) * kHomePX + (cy + 3) * kHomePY + cz + 3, kHomeField, kChkShared)) return;
    // shared-window byte address of the particle's first stencil node
    const unsigned base = static_cast<unsigned>(__cvta_generic_to_shared(acc)) + 4u * (cx * kHomePX + cy * kHomePY + cz);
#pragma unroll
    for (int k0 = 0; k0 < 4; ++k0) {
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            const float w01 = wx[k0] * wy[k1];
            const unsigned b = base + 4u * (k0 * kHomePX + k1 * kHomePY);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) {
                const float ww = w01 * wz[k2];
                const unsigned a = b + 4 * k2;
                red_shared_add(a, __float_as_int(fmaf(q0, ww, kMagic)) - kMagicBits);
                red_shared_add(a + 4 * kHomeField, __float_as_int(fmaf(q1, ww, kMagic)) - kMagicBits);
                red_shared_add(a + 8 * kHomeField, __float_as_int(fmaf(q2, ww, kMagic)) - kMagicBits);
                red_shared_add(a + 12 * kHomeField, __float_as_int(fmaf(q3, ww, kMagic)) - kMagicBits);
            }
        }
    }
}

// Pairs of FP32 values in one 64-bit register pair for the paired FP32 FMA of sm_100
// and later (fma.rn.f32x2: two correctly rounded FMAs per instruction issued, each the
// same result as the scalar instruction).
using f32x2 = unsigned long long;
__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// The first particles of four z-consecutive home cells (z = 4m .. 4m + 3 of column
// (cx, cy)) of one lane. For each of the 16 (x, y) stencil node columns the lane sums
// the cells' contributions to the 7 z nodes it reaches in registers, then adds the 7
// sums: 28 shared adds per node column instead of 64 for four particles one by one.
// Each contribution is the same rounded integer as in home_particle (same products, one
// FMA against 1.5 * 2^23, here two fields per paired FMA); the raw bit patterns are summed modulo 2^32 and the magic
// constant is taken off once per node (cnt(i) cells reach z node i), so the sums are
// exact. An empty cell has q = 0 and adds exactly the magic constant. With the lanes of
// a warp on 2 x 4 columns (cx, cy) and m = 0..3, the 32 lanes of every add hit 32
// different banks: (16 cx + 19 cy + 4 m) mod 32 is distinct over them.
__device__ __forceinline__ void home_quad(unsigned acc_s, const Record<float> (&r)[4], const bool (&has)[4], int cx,
                                          int cy, int m, float sc0, float sc1, float sc2, float sc3)
{
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
    constexpr unsigned kMagicBits = 0x4B400000u;
    float wx[4][4], wy[4][4], wz[4][4], q[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int first;
        bspline_weights<4, float>(has[j] ? r[j].u.x : 0.0f, wx[j], first);
        bspline_weights<4, float>(has[j] ? r[j].u.y : 0.0f, wy[j], first);
        bspline_weights<4, float>(has[j] ? r[j].u.z : 0.0f, wz[j], first);
        q[j][0] = has[j] ? r[j].q.x * sc0 : 0.0f;
        q[j][1] = has[j] ? r[j].q.y * sc1 : 0.0f;
        q[j][2] = has[j] ? r[j].q.z * sc2 : 0.0f;
        q[j][3] = has[j] ? r[j].q.w * sc3 : 0.0f;
    }
    f32x2 qp[4][2];  // fields (0, 1) and (2, 3) of each cell as pairs
#pragma unroll
    for (int j = 0; j < 4; ++j) qp[j][0] = f2_pack(q[j][0], q[j][1]), qp[j][1] = f2_pack(q[j][2], q[j][3]);
    const f32x2 mg = f2_pack(kMagic, kMagic);
    // buffer index of node (cx - 1 + dx, cy - 1 + dy, 4m - 1 + i) is (cx + dx) PX + (cy + dy) PY + 4m + i.
    // The 4 x 4 node columns are two rolled loops (a short body for the instruction
    // cache); the weights of the current dx and dy are kept in slot 0 by rotating them.
    // the lane's last node (3, 3 node columns on, z node 4m + 6) must lie in the buffer
    if (!PK_IN((cx + 3) * kHomePX + (cy + 3) * kHomePY + 4 * m + 6, kHomeField, kChkShared)) return;
    unsigned base = acc_s + 4u * static_cast<unsigned>(cx * kHomePX + cy * kHomePY + 4 * m);
#pragma unroll 1
    for (int dx = 0; dx < 4; ++dx) {
#pragma unroll 1
        for (int dy = 0; dy < 4; ++dy) {
            unsigned a[7][4];
            static_for<7>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr unsigned cnt = static_cast<unsigned>((i < 3 ? i : 3) - (i > 3 ? i - 3 : 0) + 1);
#pragma unroll
                for (int f = 0; f < 4; ++f) a[i][f] = 0u - cnt * kMagicBits;
            });
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float w01 = wx[j][0] * wy[j][0];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float ww = w01 * wz[j][k];
                    const f32x2 w2 = f2_pack(ww, ww);
                    const f32x2 t01 = f2_fma(qp[j][0], w2, mg), t23 = f2_fma(qp[j][1], w2, mg);
                    a[j + k][0] += static_cast<unsigned>(t01);
                    a[j + k][1] += static_cast<unsigned>(t01 >> 32);
                    a[j + k][2] += static_cast<unsigned>(t23);
                    a[j + k][3] += static_cast<unsigned>(t23 >> 32);
                }
            }
            const unsigned b = base + 4u * static_cast<unsigned>(dy * kHomePY);
            static_for<7>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                red4<4 * i, 4 * kHomeField>(b, static_cast<int>(a[i][0]), static_cast<int>(a[i][1]),
                                            static_cast<int>(a[i][2]), static_cast<int>(a[i][3]));
            });
#pragma unroll
            for (int j = 0; j < 4; ++j) {  // next dy in slot 0
                const float t = wy[j][0];
                wy[j][0] = wy[j][1], wy[j][1] = wy[j][2], wy[j][2] = wy[j][3], wy[j][3] = t;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // next dx in slot 0
            const float t = wx[j][0];
            wx[j][0] = wx[j][1], wx[j][1] = wx[j][2], wx[j][2] = wx[j][3], wx[j][3] = t;
        }
        base += 4u * kHomePX;
    }
}

// A sorted particle of this tile (its cell read from the record); skipped if the record
// does not lie in the tile. One copy for its three call sites (instruction cache).
__device__ __noinline__ void home_listed(int *acc, const Record<float> *__restrict__ rec, uint32_t idx, int t0, int t1,
                                         int t2, float sc0, float sc1, float sc2, float sc3)
{
    const Record<float> r = rec[idx];
    const int c = unpack_cell(r.u.w);
    const unsigned cx = static_cast<unsigned>((c & 1023) - t0), cy = static_cast<unsigned>(((c >> 10) & 1023) - t1),
                   cz = static_cast<unsigned>(((c >> 20) & 1023) - t2);
    if (cx < kHomeT && cy < kHomeT && cz < kHomeT)
        home_particle(acc, r, static_cast<int>(cx), static_cast<int>(cy), static_cast<int>(cz), sc0, sc1, sc2, sc3);
}

// Dense home tiles: one warp per occupied cell; lane l owns stencil nodes (dx, dy, dz)
// with dz = l & 3, dy = (l >> 2) & 3, dx = (l >> 4) and (l >> 4) + 2, sums up to
// kCellFlush of the cell's particles in FP32 registers and adds the rounded sums.
template <int F0>
__device__ __forceinline__ void home_cells_path(const Record<float> *__restrict__ rec,
                                                const uint32_t *__restrict__ offsets, int ng, int t0, int t1, int t2,
                                                unsigned long long *acc, const float *s_fine)
{
    const float fine[4] = {s_fine[0], s_fine[1], s_fine[2], s_fine[3]};
    const int noshift[4] = {0, 0, 0, 0};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int dz = lane & 3, dy = (lane >> 2) & 3, dxl = lane >> 4;
    CellPieces pc;
    cubic_piece(dxl, pc.xa);
    cubic_piece(dxl + 2, pc.xb);
    cubic_piece(dy, pc.y);
    cubic_piece(dz, pc.z);
    for (int c = warp; c < kHomeT * kHomeT * kHomeT; c += kHomeNW) {
        const int cx = c >> 8, cy = (c >> 4) & 15, cz = c & 15;
        const int64_t key = (static_cast<int64_t>(t0 + cx) * ng + (t1 + cy)) * ng + (t2 + cz);
        const uint32_t beg = offsets[key], end = offsets[key + 1];
        if (beg == end) continue;
        const int oa = (cx + dxl) * kHomePX + (cy + dy) * kHomePY + cz + dz, ob = oa + 2 * kHomePX;
        if (!PK_IN(ob, kHomeField, kChkShared)) continue;
        for (uint32_t i0 = beg; i0 < end; i0 += kCellFlush) {
            int a[2], b[2];
            cell_chunk<F0, 2>(rec, i0, min(end, i0 + kCellFlush), pc, fine, noshift, a, b);
#pragma unroll
            for (int f = 0; f < 2; ++f) {  // two's complement sums
                atomicAdd(acc + f * kHomeField + oa, static_cast<unsigned long long>(static_cast<long long>(a[f])));
                atomicAdd(acc + f * kHomeField + ob, static_cast<unsigned long long>(static_cast<long long>(b[f])));
            }
        }
    }
}

__global__ void __launch_bounds__(kHomeNT, 2)
k_deposit_home(const Record<float> *__restrict__ rec, const uint32_t *__restrict__ offsets,
               const unsigned *__restrict__ qmax_bits, int ng, float *__restrict__ grids, int64_t grid_elems,
               float *__restrict__ halo)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *acc = reinterpret_cast<int *>(smem_raw);  // [4][kHomeB][kHomePX] (x, y, z of the node buffer)
    // column ranges of the tile (sparse path), reused as the per-warp queues (medium path)
    __shared__ uint32_t s_cols[2 * kHomeNT + 1];
    uint32_t *s_beg = s_cols, *s_pre = s_cols + kHomeNT;
    __shared__ unsigned s_rowmax;
    __shared__ float s_scale[4], s_fine[4];
    __shared__ int s_shift[4];

    const int nt = ng / kHomeT;
    const int tz = blockIdx.x % nt, ty = (blockIdx.x / nt) % nt, tx = blockIdx.x / (nt * nt);
    const int t0 = tx * kHomeT, t1 = ty * kHomeT, t2 = tz * kHomeT;
    const float qm = threadIdx.x < 4 ? __uint_as_float(qmax_bits[threadIdx.x]) : 0.0f;  // used after the scan
    {
        int4 *a4 = reinterpret_cast<int4 *>(acc);
        for (int k = threadIdx.x; k < kHomeField; k += kHomeNT) a4[k] = make_int4(0, 0, 0, 0);  // 4 fields / 4 ints
    }
    if (threadIdx.x == 0) s_rowmax = 0;
    __syncthreads();
    // thread = cell column (x, y) of the tile: its particles are one range of the sort
    uint32_t total;
    {
        const int x = threadIdx.x >> 4, y = threadIdx.x & 15;
        const int64_t key = (static_cast<int64_t>(t0 + x) * ng + (t1 + y)) * ng + t2;
        uint32_t o[kHomeT + 1];
#pragma unroll
        for (int z = 0; z <= kHomeT; ++z) o[z] = offsets[key + z];
        const uint32_t b = o[0], cnt = o[kHomeT] - b;
        // the column's records are read later, cell by cell: ask L2 for them now (128-byte
        // lines covering the column's contiguous range, at most 32 lines per column)
        {
            const char *r0 = reinterpret_cast<const char *>(rec + b);
            const uint32_t lines = cnt ? min((cnt * 32u + 127u) / 128u + 1u, 32u) : 0u;
            for (uint32_t l = 0; l < lines; ++l) asm volatile("prefetch.L2 [%0];" ::"l"(r0 + 128 * l));
        }
        // a node receives from 4 consecutive cells of a column: the largest such count
        uint32_t win = 0;
#pragma unroll
        for (int z = 0; z + 4 <= kHomeT; ++z) win = max(win, o[z + 4] - o[z]);
        const uint32_t pre = block_exclusive_scan(cnt, total);
        s_beg[threadIdx.x] = b;
        s_pre[threadIdx.x] = pre;
        if (threadIdx.x == 0) s_pre[kHomeNT] = total;
        if (win) atomicMax(&s_rowmax, win);
    }
    __syncthreads();
    constexpr uint32_t kCells = kHomeT * kHomeT * kHomeT;
    // dense somewhere (32 particles in four consecutive cells) or on average: sum each
    // cell in registers and round once per cell, instead of once per particle
    const bool dense = s_rowmax >= 32u || total > 2u * kCells;
    const bool sparse = !dense && total < kCells / 4u;
    if (threadIdx.x < 4) {
        const int f = threadIdx.x;
        const float m = qm;  // max |q_f| over the catalogue, loaded at the start
        const float w3 = kMaxWeight3<4> * 1.0001f;
        // a node receives from 4 consecutive cells of at most 4 x 4 columns of the tile
        const float reach = fminf(16.0f * static_cast<float>(s_rowmax), static_cast<float>(total));
        tile_scales(w3 * reach * m, w3 * m, dense, s_scale[f], s_fine[f], s_shift[f]);
    }
    __syncthreads();
    const float sc0 = s_scale[0], sc1 = s_scale[1], sc2 = s_scale[2], sc3 = s_scale[3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // owned nodes to the grid, halo nodes to this tile's scratch; value(f, buffer index).
    // Owned rows: eight lanes per (x, y) row, two z nodes each (8-byte stores: the rows
    // start at even offsets, ng + 2 and the tile corner being even, and the grids are
    // 16-byte aligned).
    float *h = halo + static_cast<int64_t>(blockIdx.x) * 4 * kHomeHalo;
    auto emit = [&](int f, auto value) {
        float *gf = grids + f * grid_elems;
#pragma unroll 2
        for (int pass = 0; pass < kHomeT * kHomeT * 8 / kHomeNT; ++pass) {
            const int rowi = pass * (kHomeNT / 8) + (threadIdx.x >> 3), zp = 2 * (threadIdx.x & 7);
            const int x = rowi >> 4, y = rowi & 15;
            const int ab = (x + 1) * kHomePX + (y + 1) * kHomePY + zp + 1;
            const int64_t gi = (static_cast<int64_t>(t0 + x) * ng + (t1 + y)) * (ng + 2) + t2 + zp;
            if (PK_IN(gi + 1, grid_elems, kChkGrid) && PK_IN(ab + 1, kHomeField, kChkShared))
                *reinterpret_cast<float2 *>(gf + gi) = make_float2(value(ab), value(ab + 1));
        }
        for (int k = threadIdx.x; k < kHomeHalo; k += kHomeNT) {
            int bx, by, bz;
            home_halo_node(k, bx, by, bz);
            const int ai = bx * kHomePX + by * kHomePY + bz;
            if (PK_IN(static_cast<int64_t>(blockIdx.x) * 4 * kHomeHalo + f * kHomeHalo + k,
                      static_cast<int64_t>(gridDim.x) * 4 * kHomeHalo, kChkHalo) &&
                PK_IN(ai, kHomeField, kChkShared))
                h[f * kHomeHalo + k] = value(ai);
        }
    };

    if (dense) {
        // 64-bit sums of the fine-scale contributions, two fields per pass in the same buffer
        auto *acc64 = reinterpret_cast<unsigned long long *>(smem_raw);  // [2][kHomeB][kHomePX]
#pragma unroll
        for (int pass = 0; pass < 2; ++pass) {
            if (pass) {
                __syncthreads();
                int4 *a4 = reinterpret_cast<int4 *>(smem_raw);
                for (int k = threadIdx.x; k < kHomeField; k += kHomeNT) a4[k] = make_int4(0, 0, 0, 0);
                __syncthreads();
            }
            if (pass == 0) home_cells_path<0>(rec, offsets, ng, t0, t1, t2, acc64, s_fine);
            else home_cells_path<2>(rec, offsets, ng, t0, t1, t2, acc64, s_fine);
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int f = 2 * pass + k;
                const float inv = 1.0f / s_fine[f];  // exact: a power of two
                const unsigned long long *a = acc64 + k * kHomeField;
                emit(f, [&](int ai) { return static_cast<float>(static_cast<long long>(a[ai])) * inv; });
            }
        }
        return;
    }
    if (sparse) {
        // one particle per lane, warp-contiguous chunks of the tile's list
        const uint32_t per_warp = ((total + kHomeNW - 1) / kHomeNW + 31u) & ~31u;
        const uint32_t wbeg = static_cast<uint32_t>(warp) * per_warp, wend = min(wbeg + per_warp, total);
        int slot = wbeg + lane < wend ? find_slot<kHomeNT>(s_pre, wbeg + lane) : 0;
        for (uint32_t p = wbeg + lane; p < wend; p += 32) {
            while (p >= s_pre[slot + 1]) ++slot;
            home_listed(acc, rec, s_beg[slot] + (p - s_pre[slot]), t0, t1, t2, sc0, sc1, sc2, sc3);
        }
    } else {
        uint32_t *q = s_cols + warp * kHomeQ;  // the column ranges are no longer needed
        __syncthreads();
        int qn = 0;  // warp-uniform queue length
        const unsigned acc_s = static_cast<unsigned>(__cvta_generic_to_shared(acc));
        // a block is 2 x 4 cell columns; lane (xl, yl, m) takes cells z = 4m .. 4m + 3
        const int m = lane & 3, yl = (lane >> 2) & 3, xl = lane >> 4;
        constexpr int kBlocks = (kHomeT / 2) * (kHomeT / 4);
        auto cell_offsets = [&](int blk, uint32_t(&o)[5]) {  // the five offsets of the four cells
            if (blk >= kBlocks) {
#pragma unroll
                for (int k = 0; k < 5; ++k) o[k] = 0;
                return;
            }
            const int cx = 2 * (blk >> 2) + xl, cy = 4 * (blk & 3) + yl;
            const int64_t key = (static_cast<int64_t>(t0 + cx) * ng + (t1 + cy)) * ng + (t2 + 4 * m);
#pragma unroll
            for (int k = 0; k < 5; ++k) o[k] = offsets[key + k];
        };
        uint32_t on[5];
        cell_offsets(warp, on);  // loads run one block ahead
        for (int blk = warp; blk < kBlocks; blk += kHomeNW) {
            const int cx = 2 * (blk >> 2) + xl, cy = 4 * (blk & 3) + yl;
            uint32_t o[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) o[k] = on[k];
            cell_offsets(blk + kHomeNW, on);
            Record<float> r[4];
            bool has[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                has[k] = o[k + 1] > o[k];
                r[k] = has[k] ? rec[o[k]] : Record<float>{};
            }
            home_quad(acc_s, r, has, cx, cy, m, sc0, sc1, sc2, sc3);
            // second and later particles of the four cells: the per-warp queue, 32 at a time
#pragma unroll 1
            for (int k = 0; k < 4; ++k) {
                uint32_t next = o[k] + 1, extra = has[k] ? o[k + 1] - o[k] - 1 : 0u;
                while (__any_sync(0xffffffffu, extra > 0u)) {
                    const bool more = extra > 0u;
                    const unsigned mk = __ballot_sync(0xffffffffu, more);
                    if (more) {
                        q[qn + __popc(mk & ((1u << lane) - 1u))] = next;
                        ++next;
                        --extra;
                    }
                    qn += __popc(mk);
                    __syncwarp();
                    if (qn >= 32) {
                        home_listed(acc, rec, q[lane], t0, t1, t2, sc0, sc1, sc2, sc3);
                        __syncwarp();
                        if (lane < qn - 32) q[lane] = q[lane + 32];
                        qn -= 32;
                        __syncwarp();
                    }
                }
            }
        }
        if (lane < qn) home_listed(acc, rec, q[lane], t0, t1, t2, sc0, sc1, sc2, sc3);
    }
    __syncthreads();
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const float inv = 1.0f / s_scale[f];  // exact: a power of two
        const int *a = acc + f * kHomeField;
        emit(f, [&](int ai) { return static_cast<float>(a[ai]) * inv; });
    }
}

// Owned nodes within reach of a neighbouring tile's particles (local index 0, 1 or 15
// on some axis) receive that neighbour's halo values, added in a fixed order. Threads
// take only those 1899 nodes of a tile: the x faces (x in {0, 1, 15}), then the y faces
// of the other x, then the z faces of the rest, z fastest where a face allows.
constexpr int kHomeEdge = 3 * kHomeT * kHomeT + (kHomeT - 3) * 3 * kHomeT + (kHomeT - 3) * (kHomeT - 3) * 3;
__device__ __forceinline__ int home_face(int s) { return s == 2 ? kHomeT - 1 : s; }  // 0, 1, 15

__global__ void __launch_bounds__(256)
k_home_fixup(const float *__restrict__ halo, int ng, float *__restrict__ grids, int64_t grid_elems)
{
    const int nt = ng / kHomeT;
    const int tz = blockIdx.x % nt, ty = (blockIdx.x / nt) % nt, tx = blockIdx.x / (nt * nt);
    auto wrap = [nt](int a) { return a < 0 ? a + nt : (a >= nt ? a - nt : a); };
    // the neighbour offset on one axis whose halo covers local index l (0 if none)
    auto side = [](int l) { return l <= 1 ? -1 : (l == kHomeT - 1 ? 1 : 0); };
    constexpr int nx = 3 * kHomeT * kHomeT, ny = (kHomeT - 3) * 3 * kHomeT;
    for (int k = threadIdx.x; k < kHomeEdge; k += blockDim.x) {
        int x, y, z;
        if (k < nx) {
            x = home_face(k / (kHomeT * kHomeT));
            y = (k / kHomeT) % kHomeT;
            z = k % kHomeT;
        } else if (k < nx + ny) {
            const int r = k - nx;
            x = 2 + r / (3 * kHomeT);
            y = home_face((r / kHomeT) % 3);
            z = r % kHomeT;
        } else {
            const int r = k - nx - ny;
            x = 2 + r / (3 * (kHomeT - 3));
            y = 2 + (r / 3) % (kHomeT - 3);
            z = home_face(r % 3);
        }
        const int64_t gi = (static_cast<int64_t>(tx * kHomeT + x) * ng + (ty * kHomeT + y)) * (ng + 2) + tz * kHomeT + z;
        if (!PK_IN(gi, grid_elems, kChkGrid)) continue;
        float v[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) v[f] = grids[f * grid_elems + gi];
        const int sx = side(x), sy = side(y), sz = side(z);
        // neighbours (dx, dy, dz), each 0 or the axis' side, in a fixed order
#pragma unroll
        for (int c = 1; c < 8; ++c) {
            const int dx = (c & 4) ? sx : 0, dy = (c & 2) ? sy : 0, dz = (c & 1) ? sz : 0;
            if (((c & 4) && !sx) || ((c & 2) && !sy) || ((c & 1) && !sz)) continue;
            const int nb = (wrap(tx + dx) * nt + wrap(ty + dy)) * nt + wrap(tz + dz);
            const int hi = home_halo_index(x - kHomeT * dx + 1, y - kHomeT * dy + 1, z - kHomeT * dz + 1);
            if (!PK_IN(static_cast<int64_t>(nb) * 4 * kHomeHalo + 3 * kHomeHalo + hi,
                       static_cast<int64_t>(gridDim.x) * 4 * kHomeHalo, kChkHalo))
                continue;
            const float *hp = halo + static_cast<int64_t>(nb) * 4 * kHomeHalo + hi;
#pragma unroll
            for (int f = 0; f < 4; ++f) v[f] += hp[f * kHomeHalo];
        }
#pragma unroll
        for (int f = 0; f < 4; ++f) grids[f * grid_elems + gi] = v[f];
    }
}

cudaError_t launch_home(const AssignPlan &pl, const uint32_t *offsets, const unsigned *qmax, const Record<float> *rec,
                        void *grids, float *halo, cudaStream_t s)
{
    constexpr int kMaxDev = 64;
    static bool configured[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev || !configured[dev]) {
        e = cudaFuncSetAttribute(k_deposit_home, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kHomeSmem));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_deposit_home, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < kMaxDev) configured[dev] = true;
    }
    const int ng = pl.ng;
    const unsigned tiles = static_cast<unsigned>((ng / kHomeT) * (ng / kHomeT) * (ng / kHomeT));
    const int64_t grid_elems = static_cast<int64_t>(ng) * ng * (ng + 2);
    auto *g = static_cast<float *>(grids);
    k_deposit_home<<<tiles, kHomeNT, kHomeSmem, s>>>(rec, offsets, qmax, ng, g, grid_elems, halo);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_home_fixup<<<tiles, 256, 0, s>>>(halo, ng, g, grid_elems);
    return cudaGetLastError();
}

struct TileDesc {
    int prec;
    int d[3];
};
constexpr TileDesc kTiles[] = {
    {PKMOM_F32, {16, 16, 16}},  // 0
    {PKMOM_F32, {16, 16, 32}},  // 1
    {PKMOM_F32, {8, 8, 32}},    // 2
    {PKMOM_F32, {8, 8, 8}},     // 3
    {PKMOM_F64, {8, 8, 16}},    // 4
    {PKMOM_F64, {16, 16, 16}},  // 5
    {PKMOM_F64, {8, 8, 8}},     // 6
    {PKMOM_F32, {16, 16, 16}},  // 7: home tiles (cubic order; other orders use tile 0)
};

template <typename T, int M, int T0, int T1, int T2, int NT, int BLR = 0>
cudaError_t launch_deposit_t(const AssignPlan &pl, const uint32_t *offsets, const unsigned *qmax, const Record<T> *rec,
                             void *grids, cudaStream_t s)
{
    using C = DepositCfg<T, M, T0, T1, T2, NT>;
    void (*kern)(const Record<T> *, const uint32_t *, const unsigned *, int, int, T *, int64_t, int);
    size_t smem = C::smem;
    int list_cap = 0;
    if constexpr (sizeof(T) == 4) {
        kern = k_deposit_fx<M, T0, T1, T2, NT, BLR>;
        list_cap = pl.list_cap;
        smem = FxLayout<T0, T1, T2>::bytes(list_cap);
    } else {
        kern = k_deposit<T, M, T0, T1, T2, NT, BLR>;
    }
    // the attribute is per device and only needs raising: remember the largest value set
    constexpr int kMaxDev = 64;
    static size_t configured[kMaxDev] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev || configured[dev] < smem) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < kMaxDev) configured[dev] = smem;
    }
    const int ng = pl.ng;
    const int64_t tiles = static_cast<int64_t>(ng / T0) * (ng / T1) * (ng / T2);
    const int64_t grid_elems = static_cast<int64_t>(ng) * ng * (ng + 2);
    kern<<<static_cast<unsigned>(tiles), NT, smem, s>>>(rec, offsets, qmax, ng, pl.sshift, static_cast<T *>(grids),
                                                           grid_elems, list_cap);
    return cudaGetLastError();
}

template <int M>
cudaError_t launch_deposit_m(const AssignPlan &pl, const uint32_t *offsets, const unsigned *q, const void *rec,
                             void *grids, float *halo, cudaStream_t s)
{
    const auto *rf = static_cast<const Record<float> *>(rec);
    const auto *rd = static_cast<const Record<double> *>(rec);
    switch (pl.tile) {
    case 0: return launch_deposit_t<float, M, 16, 16, 16, 256>(pl, offsets, q, rf, grids, s);
    case 1: return launch_deposit_t<float, M, 16, 16, 32, 512>(pl, offsets, q, rf, grids, s);
    case 2: return launch_deposit_t<float, M, 8, 8, 32, 128>(pl, offsets, q, rf, grids, s);
    case 3: return launch_deposit_t<float, M, 8, 8, 8, 128>(pl, offsets, q, rf, grids, s);
    case 4: return launch_deposit_t<double, M, 8, 8, 16, 256>(pl, offsets, q, rd, grids, s);
    case 5: return launch_deposit_t<double, M, 16, 16, 16, 256>(pl, offsets, q, rd, grids, s);
    case 6: return launch_deposit_t<double, M, 8, 8, 8, 128>(pl, offsets, q, rd, grids, s);
    case 7:
        if constexpr (M == 4) return launch_home(pl, offsets, q, rf, grids, halo, s);
        else return launch_deposit_t<float, M, 16, 16, 16, 256>(pl, offsets, q, rf, grids, s);
    default: return cudaErrorInvalidValue;
    }
}

// The direct truncated-BL deposit (gather tiles 16^3 / 8^3 in FP32, 8x8x16 / 8^3 in FP64).
template <int R>
cudaError_t launch_deposit_bl(const AssignPlan &pl, const uint32_t *offsets, const unsigned *q, const void *rec,
                              void *grids, cudaStream_t s)
{
    constexpr int M = 2 * R;
    const auto *rf = static_cast<const Record<float> *>(rec);
    const auto *rd = static_cast<const Record<double> *>(rec);
    switch (pl.tile) {
    case 0: return launch_deposit_t<float, M, 16, 16, 16, 256, R>(pl, offsets, q, rf, grids, s);
    case 3: return launch_deposit_t<float, M, 8, 8, 8, 128, R>(pl, offsets, q, rf, grids, s);
    case 4: return launch_deposit_t<double, M, 8, 8, 16, 256, R>(pl, offsets, q, rd, grids, s);
    case 6: return launch_deposit_t<double, M, 8, 8, 8, 128, R>(pl, offsets, q, rd, grids, s);
    default: return cudaErrorInvalidValue;
    }
}

// c_n = (1/2 pi) int Sigma_4(w)^{-1/2} e^{i n w} dw by the periodic trapezoid rule on 4096
// points (spectrally accurate for this smooth periodic integrand), with
// Sigma_4(w) = (2416 + 2382 cos w + 240 cos 2w + 2 cos 3w) / 5040 from the integer samples
// of the order-8 B-spline; copied to constant memory once per device.
cudaError_t set_bl_coefficients()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    constexpr int N = 4096;
    constexpr double kPi = 3.14159265358979323846;
    double c[8] = {};
    for (int k = 0; k < N; ++k) {
        const double w = 2.0 * kPi * k / N;
        const double sig = (2416.0 + 2382.0 * std::cos(w) + 240.0 * std::cos(2 * w) + 2.0 * std::cos(3 * w)) / 5040.0;
        const double f = 1.0 / std::sqrt(sig);
        for (int n = 0; n < 8; ++n) c[n] += f * std::cos(n * w);
    }
    float cf[8];
    for (int n = 0; n < 8; ++n) {
        c[n] /= N;
        cf[n] = static_cast<float>(c[n]);
    }
    if ((e = cudaMemcpyToSymbol(c_bl_f, cf, sizeof cf)) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_bl_d, c, sizeof c)) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) done[dev] = true;
    return cudaSuccess;
}

template <typename T>
const T *tp(const void *p) { return static_cast<const T *>(p); }

}  // namespace

int deposit_tile_count() { return static_cast<int>(sizeof(kTiles) / sizeof(kTiles[0])); }

size_t home_halo_bytes(int ng)
{
    const size_t tiles = size_t(ng / kHomeT) * (ng / kHomeT) * (ng / kHomeT);
    return tiles * 4 * kHomeHalo * sizeof(float);
}

void deposit_tile_shape(int tile, int prec, int dims[3])
{
    dims[0] = dims[1] = dims[2] = 0;
    if (tile < 0 || tile >= deposit_tile_count() || kTiles[tile].prec != prec) return;
    for (int a = 0; a < 3; ++a) dims[a] = kTiles[tile].d[a];
}

// The key table: counts at C = P + 4 words (P = scratch + off_counts; 16-byte aligned
// for the scan's vector accesses). The histogram counts into C[key], the scan turns the
// counts into exclusive offsets in place, and the scatter advances C[key] once per
// particle it places, leaving C[key] = offset[key + 1]. P[3] stays zero, so C - 1 is the
// table offset[0..nkeys] the deposit reads.
size_t key_table_bytes(int64_t nkeys) { return static_cast<size_t>(nkeys + 5) * sizeof(uint32_t); }
uint32_t *key_table(const AssignPlan &pl, void *scratch)
{
    return reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + pl.off_counts) + 4;
}

cudaError_t launch_hist_moments(const pkmom_catalog &cat, const AssignPlan &pl, double box_L, void *scratch,
                                int *err_flag, cudaStream_t s, LaunchStats &st)
{
    char *sc = static_cast<char *>(scratch);
    uint32_t *counts = key_table(pl, scratch);
    auto *qmax = reinterpret_cast<unsigned *>(sc + pl.off_qmax);
    cudaError_t e = cudaMemsetAsync(sc + pl.off_counts, 0, key_table_bytes(pl.nkeys), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(qmax, 0, 4 * sizeof(unsigned), s);  // maxima taken by the scatter
    if (e != cudaSuccess) return e;
    const double scale = static_cast<double>(pl.ng) / box_L;
    if (pl.prec == PKMOM_F32) {
        k_hist<float><<<pl.hist_blocks, kHistThreads, 0, s>>>(tp<float>(cat.x), tp<float>(cat.y), tp<float>(cat.z),
                                                            cat.stride, cat.n, static_cast<float>(scale), pl.ng,
                                                            pl.sshift, counts, err_flag);
    } else {
        k_hist<double><<<pl.hist_blocks, kHistThreads, 0, s>>>(tp<double>(cat.x), tp<double>(cat.y),
                                                             tp<double>(cat.z), cat.stride, cat.n, scale, pl.ng,
                                                             pl.sshift, counts, err_flag);
    }
    st.launches++;
    return cudaGetLastError();
}

cudaError_t launch_moments_final(const AssignPlan &pl, int64_t n, void *scratch, double *moments_dev,
                                 cudaStream_t s, LaunchStats &st)
{
    char *sc = static_cast<char *>(scratch);
    auto *partials = reinterpret_cast<const double *>(sc + pl.off_partials);
    k_moments_final<<<1, 32 * kMomentVals, 0, s>>>(partials, pl.hist_blocks, n, moments_dev);
    st.launches++;
    return cudaGetLastError();
}

cudaError_t launch_scan(const AssignPlan &pl, void *scratch, cudaStream_t s, LaunchStats &st)
{
    char *sc = static_cast<char *>(scratch);
    uint32_t *counts = key_table(pl, scratch);
    auto *bsum = reinterpret_cast<uint32_t *>(sc + pl.off_blocksums);
    const unsigned nb = static_cast<unsigned>(pl.scan_blocks);
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(counts, pl.nkeys, bsum);
    k_scan_top<<<1, 1024, 0, s>>>(bsum, pl.scan_blocks, counts, pl.nkeys);
    k_scan_apply<<<nb, kScanThreads, 0, s>>>(counts, pl.nkeys, bsum);
    st.launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_scatter(const pkmom_catalog &cat, const AssignPlan &pl, double box_L, void *scratch,
                           cudaStream_t s, LaunchStats &st)
{
    char *sc = static_cast<char *>(scratch);
    uint32_t *cursor = key_table(pl, scratch);
    auto *partials = reinterpret_cast<double *>(sc + pl.off_partials);
    auto *qmax = reinterpret_cast<unsigned *>(sc + pl.off_qmax);
    const double scale = static_cast<double>(pl.ng) / box_L;
    const unsigned blocks = pl.hist_blocks;  // k_moments: one partial per block
    if (pl.prec == PKMOM_F32) {
        k_scatter<float><<<blocks, 256, 0, s>>>(tp<float>(cat.x), tp<float>(cat.y), tp<float>(cat.z),
                                                tp<float>(cat.vx), tp<float>(cat.vy), tp<float>(cat.vz),
                                                tp<float>(cat.mass), cat.stride, cat.n, static_cast<float>(scale),
                                                pl.ng, pl.sshift, cursor,
                                                reinterpret_cast<Record<float> *>(sc + pl.off_records));
        const char *bv = static_cast<const char *>(cat.vx);
        const bool v3 = cat.stride == 3 && static_cast<const char *>(cat.vy) == bv + 4 &&
                        static_cast<const char *>(cat.vz) == bv + 8 && reinterpret_cast<uintptr_t>(bv) % 16 == 0 &&
                        (!cat.mass || reinterpret_cast<uintptr_t>(cat.mass) % 16 == 0);
        if (v3)
            k_moments_v3<<<blocks, 256, 0, s>>>(tp<float>(cat.vx), tp<float>(cat.mass), cat.n, partials, qmax);
        else
            k_moments<float><<<blocks, 256, 0, s>>>(tp<float>(cat.vx), tp<float>(cat.vy), tp<float>(cat.vz),
                                                    tp<float>(cat.mass), cat.stride, cat.n, partials, qmax);
    } else {
        k_scatter<double><<<blocks, 256, 0, s>>>(tp<double>(cat.x), tp<double>(cat.y), tp<double>(cat.z),
                                                 tp<double>(cat.vx), tp<double>(cat.vy), tp<double>(cat.vz),
                                                 tp<double>(cat.mass), cat.stride, cat.n, scale, pl.ng, pl.sshift,
                                                 cursor, reinterpret_cast<Record<double> *>(sc + pl.off_records));
        k_moments<double><<<blocks, 256, 0, s>>>(tp<double>(cat.vx), tp<double>(cat.vy), tp<double>(cat.vz),
                                                 tp<double>(cat.mass), cat.stride, cat.n, partials, qmax);
    }
    st.launches++;
    st.launches++;
    return cudaGetLastError();
}

bool batchable_deposit(const AssignPlan &pl)
{
    return pl.prec == PKMOM_F32 && pl.order == 4 && pl.bl_radius == 0 && pl.tile == 0;
}

FxJob deposit_job(const AssignPlan &pl, void *scratch, void *grids)
{
    char *sc = static_cast<char *>(scratch);
    FxJob j{};
    j.rec = reinterpret_cast<const Record<float> *>(sc + pl.off_records);
    j.offsets = key_table(pl, scratch) - 1;
    j.qmax = reinterpret_cast<const unsigned *>(sc + pl.off_qmax);
    j.grids = static_cast<float *>(grids);
    j.grid_elems = static_cast<int64_t>(pl.ng) * pl.ng * (pl.ng + 2);
    j.ng = pl.ng;
    j.sshift = pl.sshift;
    j.list_cap = pl.list_cap;
    return j;
}

cudaError_t launch_deposit_batch(FxBatch &batch, unsigned long long *counter, int num_sms, cudaStream_t s,
                                 LaunchStats &st)
{
    constexpr int T = 16, NT = 256;
    auto kern = k_deposit_fx_batch<4, T, T, T, NT>;
    long long first = 0;
    int cap = 0;
    for (int k = 0; k < batch.n; ++k) {
        batch.job[k].first_tile = first;
        first += static_cast<long long>(batch.job[k].ng / T) * (batch.job[k].ng / T) * (batch.job[k].ng / T);
        cap = std::max(cap, batch.job[k].list_cap);
    }
    batch.total_tiles = first;
    if (first == 0) return cudaSuccess;
    const size_t smem = FxLayout<T, T, T>::bytes(cap);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess) return e;
    const long long ctas = std::min<long long>(first, static_cast<long long>(std::max(1, per_sm)) * num_sms);
    if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(ctas), NT, smem, s>>>(batch, counter);
    st.launches++;
    return cudaGetLastError();
}

cudaError_t launch_deposit(const AssignPlan &pl, void *scratch, void *grids, cudaStream_t s, LaunchStats &st)
{
    char *sc = static_cast<char *>(scratch);
    const uint32_t *offsets = key_table(pl, scratch) - 1;  // offset[0..nkeys] after the scatter
    auto *qmax = reinterpret_cast<const unsigned *>(sc + pl.off_qmax);
    const void *rec = sc + pl.off_records;
    float *halo = pl.off_halo ? reinterpret_cast<float *>(sc + pl.off_halo) : nullptr;
    cudaError_t e;
    if (pl.bl_radius > 0) {
        if ((e = set_bl_coefficients()) != cudaSuccess) return e;
        switch (pl.bl_radius) {
        case 2: e = launch_deposit_bl<2>(pl, offsets, qmax, rec, grids, s); break;
        case 3: e = launch_deposit_bl<3>(pl, offsets, qmax, rec, grids, s); break;
        case 4: e = launch_deposit_bl<4>(pl, offsets, qmax, rec, grids, s); break;
        default: return cudaErrorInvalidValue;
        }
        st.launches++;
        return e;
    }
    switch (pl.order) {
    case 1: e = launch_deposit_m<1>(pl, offsets, qmax, rec, grids, halo, s); break;
    case 2: e = launch_deposit_m<2>(pl, offsets, qmax, rec, grids, halo, s); break;
    case 3: e = launch_deposit_m<3>(pl, offsets, qmax, rec, grids, halo, s); break;
    case 4: e = launch_deposit_m<4>(pl, offsets, qmax, rec, grids, halo, s); break;
    case 5: e = launch_deposit_m<5>(pl, offsets, qmax, rec, grids, halo, s); break;
    default: return cudaErrorInvalidValue;
    }
    st.launches += (pl.tile == kHomeTile && pl.order == 4) ? 2 : 1;
    return e;
}

}  // namespace pkmom
