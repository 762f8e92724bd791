// Steps 1-2 of the estimator on the GPU: catalogue moments and the B-spline
// assignment of mass and momentum to four periodic grids (paper Secs. 2.1-2.2,
// Eq. rawFFTed; the BL kernel's Fourier factor is applied in spectra.cu).
//
// Pipeline (all on one stream):
//   k_hist_moments  one pass over the catalogue: FP64 moments (block partials) and a
//                   histogram of sort keys (key = x-row, y-row, z-segment of the cell);
//                   each particle keeps the rank its atomic increment returned.
//   k_moments_final fixed-order sum of the block partials -> pkmom_moments.
//   k_scan_*        exclusive scan of the key counts -> segment offsets.
//   k_scatter       writes each particle as a 32-byte record (grid coordinates and the
//                   four deposited values) at offset[key] + rank: a counting sort.
//   k_deposit       one CTA per output tile of grid nodes: gathers the particles of
//                   every segment whose stencils reach the tile (tile + halo, located
//                   through the offsets), accumulates B-spline weights x values in
//                   shared memory, then writes each node of the tile exactly once.
//                   No global atomics, no zero-fill pass.
#include <cfloat>

#include "pkmom_internal.cuh"

namespace pkmom {
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
    int ic = static_cast<int>(floor(u)) % ng;
    c = ic < 0 ? ic + ng : ic;
    return true;
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

// One pass over the catalogue: the histogram of sort keys (each particle keeps the
// rank its atomic increment returned) and the moments. Each lane sums kGroup
// particles in the catalogue precision; the warp then adds its lanes' group sums
// (shuffles) and lane 0 adds the result to FP64 accumulators, so that FP64 work is
// one add per value per 32 * kGroup particles. Two particles per iteration keep more
// loads and atomics in flight.
template <typename T>
__global__ void __launch_bounds__(kHistThreads, 4)
k_hist_moments(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z,
               const T *__restrict__ vx, const T *__restrict__ vy, const T *__restrict__ vz,
               const T *__restrict__ mass, int64_t stride, int64_t n, T scale, int ng, int sshift,
               uint32_t *__restrict__ counts, uint32_t *__restrict__ ranks, double *__restrict__ partials,
               unsigned *__restrict__ qmax_bits, int *__restrict__ err)
{
    const int nseg = ng >> sshift;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double s_part[kHistThreads / 32][kMomentVals];  // per-warp FP64 sums
    if (lane < kMomentVals) s_part[warp][lane] = 0.0;
    __syncwarp();
    float qmax[4] = {0.f, 0.f, 0.f, 0.f};
    T grp[kMomentVals];
#pragma unroll
    for (int k = 0; k < kMomentVals; ++k) grp[k] = T(0);
    int gcount = 0;
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t wbase0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31);

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
    auto one = [&](int64_t i) {
        const int64_t j = i * stride;
        const T u0 = mul_rn(x[j], scale), u1 = mul_rn(y[j], scale), u2 = mul_rn(z[j], scale);
        const T m = mass ? mass[i] : T(1);
        const T v0 = vx[j], v1 = vy[j], v2 = vz[j];
        int c0, c1, c2;
        const bool ok = cell_of(u0, ng, c0) & cell_of(u1, ng, c1) & cell_of(u2, ng, c2);
        uint32_t rank = 0xffffffffu;
        if (ok) {
            const int64_t key = (static_cast<int64_t>(c0) * ng + c1) * nseg + (c2 >> sshift);
            rank = atomicAdd(counts + key, 1u);
        } else {
            *err = 1;
        }
        ranks[i] = rank;
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
    for (int64_t wb = wbase0; wb < n; wb += 2 * step) {
        const int64_t i0 = wb + lane, i1 = wb + step + lane;
        if (i0 < n) one(i0);
        if (i1 < n) one(i1);
        gcount += 2;
        if (gcount >= kGroup) {
            flush();
            gcount = 0;
        }
    }
    flush();

#pragma unroll
    for (int f = 0; f < 4; ++f) {
        // non-negative floats order like their bit patterns
        const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(qmax[f]));
        if (lane == 0) atomicMax(qmax_bits + f, b);
    }
    __syncthreads();
    if (threadIdx.x < kMomentVals) {
        double s = 0.0;
        for (int w = 0; w < kHistThreads / 32; ++w) s += s_part[w][threadIdx.x];
        partials[static_cast<int64_t>(blockIdx.x) * kMomentWords + threadIdx.x] = s;
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

// ------------------------------------------------------------------ scatter
template <typename T>
__global__ void __launch_bounds__(256)
k_scatter(const T *__restrict__ x, const T *__restrict__ y, const T *__restrict__ z, const T *__restrict__ vx,
          const T *__restrict__ vy, const T *__restrict__ vz, const T *__restrict__ mass, int64_t stride, int64_t n,
          T scale, int ng, int sshift, const uint32_t *__restrict__ offsets, const uint32_t *__restrict__ ranks,
          Record<T> *__restrict__ rec)
{
    const int nseg = ng >> sshift;
    const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += step) {
        const uint32_t rank = ranks[i];
        if (rank == 0xffffffffu) continue;
        const int64_t j = i * stride;
        const T u0 = mul_rn(x[j], scale), u1 = mul_rn(y[j], scale), u2 = mul_rn(z[j], scale);
        int c0, c1, c2;
        cell_of(u0, ng, c0);
        cell_of(u1, ng, c1);
        cell_of(u2, ng, c2);
        const int64_t key = (static_cast<int64_t>(c0) * ng + c1) * nseg + (c2 >> sshift);
        const uint32_t dst = offsets[key] + rank;
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
template <int M, typename T>
__device__ __forceinline__ void bspline_weights(T t, T (&w)[M], int &first)
{
    if constexpr (M == 4) {
        const T s = T(1) - t, t2 = t * t, t3 = t2 * t;
        const T sixth = T(1) / T(6);
        w[0] = s * s * s * sixth;
        w[1] = (T(3) * t3 - T(6) * t2 + T(4)) * sixth;
        w[2] = (T(-3) * t3 + T(3) * t2 + T(3) * t + T(1)) * sixth;
        w[3] = t3 * sixth;
        first = -1;
    } else if constexpr (M == 3) {
        const bool up = t >= T(0.5);
        const T d = up ? t - T(1) : t;  // offset from the nearest node, in [-1/2, 1/2)
        const T a = T(0.5) - d, b = T(0.5) + d;
        w[0] = T(0.5) * a * a;
        w[1] = T(0.75) - d * d;
        w[2] = T(0.5) * b * b;
        first = up ? 0 : -1;
    } else if constexpr (M == 2) {
        w[0] = T(1) - t;
        w[1] = t;
        first = 0;
    } else {
        w[0] = T(1);
        first = t >= T(0.5) ? 1 : 0;
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
template <int M> constexpr float kMaxWeight3 = M == 4 ? 0.2962963f : (M == 3 ? 0.421875f : 1.0f);

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
template <typename T, int M>
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
        bspline_weights<M, T>(t[a], w[a], first);
#pragma unroll
        for (int k = 0; k < M; ++k) {
            int l = c + first + k - tb[a];
            l = l < 0 ? l + ng : (l >= ng ? l - ng : l);
            li[a][k] = l < td[a] ? l : -1;
        }
    }
}

// Tile-gather deposit with shared-memory atomics in the grid precision (used for
// FP64 grids, where FP64 accuracy is required).
template <typename T, int M, int T0, int T1, int T2, int NT>
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
        stencil<T, M>(r, ng, t0, t1, t2, T0, T1, T2, w, li);
#pragma unroll
        for (int k0 = 0; k0 < M; ++k0) {
            if (li[0][k0] < 0) continue;
#pragma unroll
            for (int k1 = 0; k1 < M; ++k1) {
                if (li[1][k1] < 0) continue;
                const T w01 = w[0][k0] * w[1][k1];
                const int b01 = (li[0][k0] * T1 + li[1][k1]) * T2;
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
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < C::TN; k += NT) {
        const int l2 = k % T2, l01 = k / T2;
        const int l1 = l01 % T1, l0 = l01 / T1;
        const int64_t gi = (static_cast<int64_t>(t0 + l0) * ng + (t1 + l1)) * (ng + 2) + t2 + l2;
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

template <int T0, int T1, int T2, int NT>
__device__ __forceinline__ void deposit_cells_path(const Record<float> *__restrict__ rec,
                                                   const uint32_t *__restrict__ offsets, int ng, int t0, int t1, int t2,
                                                   int *acc, int fstride, int rw, const float *s_scale)
{
    constexpr int HL = 2, R0 = T0 + 3, R1 = T1 + 3, RZ = T2 + 3, NW = NT / 32;
    const float sc[4] = {s_scale[0], s_scale[1], s_scale[2], s_scale[3]};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int dz = lane & 3, dy = (lane >> 2) & 3, dxl = lane >> 4;
    float cxa[4], cxb[4], cyy[4], czz[4];
    cubic_piece(dxl, cxa);
    cubic_piece(dxl + 2, cxb);
    cubic_piece(dy, cyy);
    cubic_piece(dz, czz);
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
        const int oa = (lxa * T1 + ly) * rw + lz, ob = ((lxa + 2) * T1 + ly) * rw + lz;
        for (uint32_t i0 = beg; i0 < end; i0 += kCellFlush) {
            const uint32_t i1 = min(end, i0 + kCellFlush);
            float a[4] = {0.f, 0.f, 0.f, 0.f}, b[4] = {0.f, 0.f, 0.f, 0.f};
            auto add = [&](const Record<float> &rc) {
                const float wyz = horner4(cyy, rc.u.y) * horner4(czz, rc.u.z);
                const float wa = horner4(cxa, rc.u.x) * wyz, wb = horner4(cxb, rc.u.x) * wyz;
                a[0] += rc.q.x * wa, b[0] += rc.q.x * wb;
                a[1] += rc.q.y * wa, b[1] += rc.q.y * wb;
                a[2] += rc.q.z * wa, b[2] += rc.q.z * wb;
                a[3] += rc.q.w * wa, b[3] += rc.q.w * wb;
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
            for (int f = 0; f < 4; ++f) {
                if (ina) atomicAdd(acc + f * fstride + oa, __float2int_rn(a[f] * sc[f]));
                if (inb) atomicAdd(acc + f * fstride + ob, __float2int_rn(b[f] * sc[f]));
            }
        }
    }
}

// Tile-gather deposit for FP32 grids with 32-bit integer (fixed-point) shared-memory
// atomics (about three times the throughput of FP32 shared atomics on this part).
//
// Work split: each warp walks its own contiguous chunk of the tile's particle list 32
// at a time, lane j taking the j-th particle of each step. Sorted neighbours lie in
// neighbouring cells, so for one stencil offset the lanes mostly hit different nodes
// (particles that share a cell still collide). Rows of the shared accumulator are
// padded to an odd length.
//
// Fixed point: field f of the tile uses the scale 2^s_f with
//   B_f 2^s_f < 2^29,   B_f = w3 * min(M^2 * largest row count, particle count) * max |q_f|
// over the tile's reach (w3 = the largest product of three weights; a node receives from
// at most M^2 cell rows, each contributing at most `largest row count` particles, and
// from no more than all of them; max |q_f| over the catalogue), so no node sum can overflow, and also max |q_f| w3 2^s_f < 2^22, so that
// every contribution is rounded to an integer by one FFMA against 1.5 * 2^23 (round to
// nearest even, one rounding of the exact product). The bound depends only on counts
// and maxima, and integer sums do not depend on order: the grids are the same whatever
// order the sort leaves particles of one cell in.
template <int M, int T0, int T1, int T2, int NT>
__global__ void __launch_bounds__(NT)
k_deposit_fx(const Record<float> *__restrict__ rec, const uint32_t *__restrict__ offsets,
             const unsigned *__restrict__ qmax_bits, int ng, int sshift, float *__restrict__ grids, int64_t grid_elems,
             int list_cap)
{
    using C = DepositCfg<float, M, T0, T1, T2, NT>;
    constexpr int RW = T2 + 1;  // odd row pitch
    constexpr int TNP = T0 * T1 * RW;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *acc = reinterpret_cast<int *>(smem_raw);  // [4][T0 * T1][RW]
    __shared__ uint32_t s_beg[C::MAXR];
    __shared__ uint32_t s_pre[C::MAXR + 1];
    __shared__ unsigned s_rowmax;
    __shared__ float s_scale[4];

    const int ntz = ng / T2, nty = ng / T1;
    int tile = blockIdx.x;
    const int tz = tile % ntz;
    tile /= ntz;
    const int ty = tile % nty;
    const int tx = tile / nty;
    const int t0 = tx * T0, t1 = ty * T1, t2 = tz * T2;
    for (int k = threadIdx.x; k < 4 * TNP; k += NT) acc[k] = 0;
    if (threadIdx.x == 0) s_rowmax = 0;
    const uint32_t total = build_ranges<C>(offsets, ng, sshift, t0, t1, t2, T2, s_beg, s_pre);
    // largest row count: a row's two pieces are slots 2r and 2r + 1
    for (int r = threadIdx.x; 2 * r + 1 < C::MAXR + 1; r += NT) {
        const uint32_t c = s_pre[2 * r + 2 <= C::MAXR ? 2 * r + 2 : C::MAXR] - s_pre[2 * r];
        if (c) atomicMax(&s_rowmax, c);
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
    const bool dense = M == 4 && total > 2u * NREACH && sshift == 0 && ng >= C::R0 && ng >= C::R1 &&
                       ng >= T2 + C::HL + C::HR;
    // per-field scale from order-independent bounds only (so that the grids, and the
    // spectra, do not depend on the order in which sorted particles share a cell)
    __syncthreads();
    if (threadIdx.x < 4) {
        const int f = threadIdx.x;
        const float m = __uint_as_float(qmax_bits[f]);  // max |q_f| over the catalogue
        const float w3 = kMaxWeight3<M> * 1.0001f;
        const float reach = fminf(static_cast<float>(M * M) * static_cast<float>(s_rowmax), static_cast<float>(total));
        const float bound = w3 * reach * m;
        const float cmax = w3 * m;  // largest single contribution
        int eb = 0, ec = 0;
        if (bound > 0.f) frexpf(bound, &eb);  // bound < 2^eb
        if (cmax > 0.f) frexpf(cmax, &ec);
        if (!isfinite(bound)) eb = 150;
        if (!isfinite(cmax)) ec = 150;
        int sexp = dense ? 29 - eb : min(29 - eb, 22 - ec);  // cell sums round with cvt, not FFMA
        sexp = sexp > 120 ? 120 : (sexp < -120 ? -120 : sexp);
        s_scale[f] = ldexpf(1.0f, sexp);
    }
    __syncthreads();
    const float sc0 = s_scale[0], sc1 = s_scale[1], sc2 = s_scale[2], sc3 = s_scale[3];
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
    constexpr int kMagicBits = 0x4B400000;

    bool cells_done = false;
    if constexpr (M == 4) {
        if (dense) {
            deposit_cells_path<T0, T1, T2, NT>(rec, offsets, ng, t0, t1, t2, acc, TNP, RW, s_scale);
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
            stencil<float, M>(rc, ng, t0, t1, t2, T0, T1, T2, w, li);
            const float q0 = rc.q.x * sc0, q1 = rc.q.y * sc1, q2 = rc.q.z * sc2, q3 = rc.q.w * sc3;
#pragma unroll
            for (int k0 = 0; k0 < M; ++k0) {
                if (li[0][k0] < 0) continue;
#pragma unroll
                for (int k1 = 0; k1 < M; ++k1) {
                    if (li[1][k1] < 0) continue;
                    const float w01 = w[0][k0] * w[1][k1];
                    const int b01 = (li[0][k0] * T1 + li[1][k1]) * RW;
#pragma unroll
                    for (int k2 = 0; k2 < M; ++k2) {
                        if (li[2][k2] < 0) continue;
                        const float ww = w01 * w[2][k2];
                        int *a = acc + b01 + li[2][k2];
                        atomicAdd(a, __float_as_int(fmaf(q0, ww, kMagic)) - kMagicBits);
                        atomicAdd(a + TNP, __float_as_int(fmaf(q1, ww, kMagic)) - kMagicBits);
                        atomicAdd(a + 2 * TNP, __float_as_int(fmaf(q2, ww, kMagic)) - kMagicBits);
                        atomicAdd(a + 3 * TNP, __float_as_int(fmaf(q3, ww, kMagic)) - kMagicBits);
                    }
                }
            }
        }
    }
    __syncthreads();
    const float inv[4] = {1.0f / sc0, 1.0f / sc1, 1.0f / sc2, 1.0f / sc3};  // exact: powers of two
    for (int k = threadIdx.x; k < C::TN; k += NT) {
        const int l2 = k % T2, l01 = k / T2;
        const int l1 = l01 % T1, l0 = l01 / T1;
        const int64_t gi = (static_cast<int64_t>(t0 + l0) * ng + (t1 + l1)) * (ng + 2) + t2 + l2;
        const int ai = l01 * RW + l2;
#pragma unroll
        for (int f = 0; f < 4; ++f) grids[f * grid_elems + gi] = static_cast<float>(acc[f * TNP + ai]) * inv[f];
    }
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
};

template <typename T, int M, int T0, int T1, int T2, int NT>
cudaError_t launch_deposit_t(const AssignPlan &pl, const uint32_t *offsets, const unsigned *qmax, const Record<T> *rec,
                             void *grids, cudaStream_t s)
{
    using C = DepositCfg<T, M, T0, T1, T2, NT>;
    void (*kern)(const Record<T> *, const uint32_t *, const unsigned *, int, int, T *, int64_t, int);
    size_t smem = C::smem;
    int list_cap = 0;
    if constexpr (sizeof(T) == 4) {
        kern = k_deposit_fx<M, T0, T1, T2, NT>;
        list_cap = pl.list_cap;
        smem = size_t(4) * T0 * T1 * (T2 + 1) * sizeof(int) + size_t(list_cap) * sizeof(uint32_t);
    } else {
        kern = k_deposit<T, M, T0, T1, T2, NT>;
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
                             void *grids, cudaStream_t s)
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
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
const T *tp(const void *p) { return static_cast<const T *>(p); }

}  // namespace

int deposit_tile_count() { return static_cast<int>(sizeof(kTiles) / sizeof(kTiles[0])); }

void deposit_tile_shape(int tile, int prec, int dims[3])
{
    dims[0] = dims[1] = dims[2] = 0;
    if (tile < 0 || tile >= deposit_tile_count() || kTiles[tile].prec != prec) return;
    for (int a = 0; a < 3; ++a) dims[a] = kTiles[tile].d[a];
}

cudaError_t launch_hist_moments(const pkmom_catalog &cat, const AssignPlan &pl, double box_L, void *scratch,
                                int *err_flag, cudaStream_t s, LaunchStats &st)
{
    char *sc = static_cast<char *>(scratch);
    auto *counts = reinterpret_cast<uint32_t *>(sc + pl.off_counts);
    auto *ranks = reinterpret_cast<uint32_t *>(sc + pl.off_ranks);
    auto *partials = reinterpret_cast<double *>(sc + pl.off_partials);
    auto *qmax = reinterpret_cast<unsigned *>(sc + pl.off_qmax);
    cudaError_t e = cudaMemsetAsync(counts, 0, static_cast<size_t>(pl.nkeys + 1) * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(qmax, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const double scale = static_cast<double>(pl.ng) / box_L;
    if (pl.prec == PKMOM_F32) {
        k_hist_moments<float><<<pl.hist_blocks, kHistThreads, 0, s>>>(
            tp<float>(cat.x), tp<float>(cat.y), tp<float>(cat.z), tp<float>(cat.vx), tp<float>(cat.vy),
            tp<float>(cat.vz), tp<float>(cat.mass), cat.stride, cat.n, static_cast<float>(scale), pl.ng, pl.sshift,
            counts, ranks, partials, qmax, err_flag);
    } else {
        k_hist_moments<double><<<pl.hist_blocks, kHistThreads, 0, s>>>(
            tp<double>(cat.x), tp<double>(cat.y), tp<double>(cat.z), tp<double>(cat.vx), tp<double>(cat.vy),
            tp<double>(cat.vz), tp<double>(cat.mass), cat.stride, cat.n, scale, pl.ng, pl.sshift, counts, ranks,
            partials, qmax, err_flag);
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
    auto *counts = reinterpret_cast<uint32_t *>(sc + pl.off_counts);
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
    auto *offsets = reinterpret_cast<const uint32_t *>(sc + pl.off_counts);
    auto *ranks = reinterpret_cast<const uint32_t *>(sc + pl.off_ranks);
    const double scale = static_cast<double>(pl.ng) / box_L;
    const unsigned blocks = pl.hist_blocks;
    if (pl.prec == PKMOM_F32) {
        k_scatter<float><<<blocks, 256, 0, s>>>(tp<float>(cat.x), tp<float>(cat.y), tp<float>(cat.z),
                                                tp<float>(cat.vx), tp<float>(cat.vy), tp<float>(cat.vz),
                                                tp<float>(cat.mass), cat.stride, cat.n, static_cast<float>(scale),
                                                pl.ng, pl.sshift, offsets, ranks,
                                                reinterpret_cast<Record<float> *>(sc + pl.off_records));
    } else {
        k_scatter<double><<<blocks, 256, 0, s>>>(tp<double>(cat.x), tp<double>(cat.y), tp<double>(cat.z),
                                                 tp<double>(cat.vx), tp<double>(cat.vy), tp<double>(cat.vz),
                                                 tp<double>(cat.mass), cat.stride, cat.n, scale, pl.ng, pl.sshift,
                                                 offsets, ranks,
                                                 reinterpret_cast<Record<double> *>(sc + pl.off_records));
    }
    st.launches++;
    return cudaGetLastError();
}

cudaError_t launch_deposit(const AssignPlan &pl, void *scratch, void *grids, cudaStream_t s, LaunchStats &st)
{
    char *sc = static_cast<char *>(scratch);
    auto *offsets = reinterpret_cast<const uint32_t *>(sc + pl.off_counts);
    auto *qmax = reinterpret_cast<const unsigned *>(sc + pl.off_qmax);
    const void *rec = sc + pl.off_records;
    cudaError_t e;
    switch (pl.order) {
    case 1: e = launch_deposit_m<1>(pl, offsets, qmax, rec, grids, s); break;
    case 2: e = launch_deposit_m<2>(pl, offsets, qmax, rec, grids, s); break;
    case 3: e = launch_deposit_m<3>(pl, offsets, qmax, rec, grids, s); break;
    case 4: e = launch_deposit_m<4>(pl, offsets, qmax, rec, grids, s); break;
    default: return cudaErrorInvalidValue;
    }
    st.launches++;
    return e;
}

}  // namespace pkmom
