// Step 4 of the estimator on the GPU: window deconvolution, shot-noise
// subtraction and |k|-shell averages of the density, momentum, momentum-
// divergence and cross spectra, with and without the bulk flow (paper Sec. 2,
// Eqs. psn, rawPp, rawPtheta, rawPx; Sec. 3, Eqs. bfpp, bfpdpx).
//
// Per mode n (integer wave vector, k = k_f n) the four transformed B-spline
// grids F_d, F_p give the BL-assigned fields times C(n) = prod Sigma_m^{-1/2};
// dividing by the BL window W = prod Bhat_m Sigma_m^{-1/2} leaves
//     P_raw / W^2 = g(n) |F|^2,   g = 1 / prod_a Bhat_m(2 pi n_a / ng)^2,
// and the shot noise times sum_J W^2(k + 2 k_N J) (= 1 for the orthonormal BL
// function) divided by W^2 is SN * h(n), h = prod Sigma_m / prod Bhat_m^2.
//
// k_bin accumulates, per shell, sum w g |F_d|^2, sum w g |F_p|^2,
// sum w g |n.F_p|^2 and sum w g Im(conj F_d  n.F_p) for F_p and for
// F_p' = F_p - v_b F_d, with the half-spectrum weight w (1 on the planes n_z = 0
// and ng/2, else 2). Per-mode values are formed in the grid precision, combined
// across the lanes of a warp that fall in the same shell, and added into FP64
// per-CTA shell sums in shared memory; the CTA sums go to a partial array that
// a fixed-order reduction combines. The data-independent sums (mode counts,
// sum w |n|, sum w h, sum w h n n^T) are built once per grid/shell layout by
// k_mode_sums in FP64. k_finalize subtracts the shot noise at the shell level in
// FP64, where the cancellation against large shot noise is harmless.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

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

unsigned take_check_word_spectra()
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

template <typename T> struct Cx { T x, y; };

constexpr int kBinThreads = 256;
constexpr double kTwoPi = 6.283185307179586476925286766559;

// Add the values of the lanes of each run of equal `bin` (runs are contiguous in
// lane order) and let the first lane of each run add them to s_bins[k * nbins + bin].
template <int NV, typename V>
__device__ __forceinline__ void flush_runs(int bin, V (&v)[NV], double *s_bins, int nbins)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int prev = __shfl_up_sync(full, bin, 1);
    const bool head = lane == 0 || prev != bin;
    const unsigned heads = __ballot_sync(full, head);
    const int run = __popc(heads & (full >> (31 - lane)));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int orun = __shfl_down_sync(full, run, d);
        const bool take = lane + d < 32 && orun == run;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const V o = __shfl_down_sync(full, v[k], d);
            if (take) v[k] += o;
        }
    }
    if (head && bin >= 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) atomicAdd(s_bins + k * nbins + bin, static_cast<double>(v[k]));
    }
}

// Mode of lane `lane` in chunk `ch` (32 consecutive half-spectrum modes): row and z index.
__device__ __forceinline__ void chunk_mode(uint32_t ch, int lane, int ng, int nh, int &i0, int &i1, int &l)
{
    const uint32_t m0 = ch * 32u;
    const uint32_t row0 = m0 / static_cast<uint32_t>(nh);
    int ll = static_cast<int>(m0 - row0 * nh) + lane;
    int drow = 0;
    while (ll >= nh) ll -= nh, ++drow;
    const int r0 = static_cast<int>(row0 / static_cast<uint32_t>(ng));
    int r1 = static_cast<int>(row0 - static_cast<uint32_t>(r0) * ng) + drow;
    int rr0 = r0;
    while (r1 >= ng) r1 -= ng, ++rr0;
    i0 = rr0;
    i1 = r1;
    l = ll;
}

template <typename T>
__global__ void __launch_bounds__(kBinThreads)
k_bin(const Cx<T> *__restrict__ F, int64_t gstride, int ng, uint32_t nmodes, const uint16_t *__restrict__ bintab,
      int nsq_max, const T *__restrict__ gf, const T *__restrict__ gh, const double *__restrict__ mom, int nbins,
      double *__restrict__ partials)
{
    extern __shared__ double s_bins[];  // [kBinVals][nbins]
    for (int k = threadIdx.x; k < kBinVals * nbins; k += blockDim.x) s_bins[k] = 0.0;
    __syncthreads();
    const int nh = ng / 2 + 1;
    const double Mtot = mom[0];
    const T vb0 = static_cast<T>(mom[2] / Mtot), vb1 = static_cast<T>(mom[3] / Mtot), vb2 = static_cast<T>(mom[4] / Mtot);
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = (nmodes + 31u) / 32u;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < nchunks; ch += nwarps) {
        const uint32_t mode = ch * 32u + lane;
        int bin = -1;
        T v[kBinVals];
#pragma unroll
        for (int k = 0; k < kBinVals; ++k) v[k] = T(0);
        if (mode < nmodes) {
            int i0, i1, l;
            chunk_mode(ch, lane, ng, nh, i0, i1, l);
            const int n0 = i0 < ng / 2 ? i0 : i0 - ng;
            const int n1 = i1 < ng / 2 ? i1 : i1 - ng;
            const int nsq = n0 * n0 + n1 * n1 + l * l;
            const int b = nsq <= nsq_max ? static_cast<int>(bintab[nsq]) : 0xffff;
            if (b != 0xffff) {
                bin = b;
                const T g = gf[i0] * gf[i1] * gh[l] * ((l == 0 || l == nh - 1) ? T(1) : T(2));
                const Cx<T> d = F[mode], p0 = F[gstride + mode], p1 = F[2 * gstride + mode],
                            p2 = F[3 * gstride + mode];
                const T fn0 = static_cast<T>(n0), fn1 = static_cast<T>(n1), fn2 = static_cast<T>(l);
                // n . F_p
                const T kr = fn0 * p0.x + fn1 * p1.x + fn2 * p2.x;
                const T ki = fn0 * p0.y + fn1 * p1.y + fn2 * p2.y;
                const T d2 = d.x * d.x + d.y * d.y;
                v[0] = g * d2;
                v[1] = g * (p0.x * p0.x + p0.y * p0.y + p1.x * p1.x + p1.y * p1.y + p2.x * p2.x + p2.y * p2.y);
                v[2] = g * (kr * kr + ki * ki);
                v[3] = g * (d.x * ki - d.y * kr);  // Im(conj(F_d) * (n.F_p))
                // bulk flow removed: F_p' = F_p - v_b F_d
                const Cx<T> q0{p0.x - vb0 * d.x, p0.y - vb0 * d.y};
                const Cx<T> q1{p1.x - vb1 * d.x, p1.y - vb1 * d.y};
                const Cx<T> q2{p2.x - vb2 * d.x, p2.y - vb2 * d.y};
                const T jr = fn0 * q0.x + fn1 * q1.x + fn2 * q2.x;
                const T ji = fn0 * q0.y + fn1 * q1.y + fn2 * q2.y;
                v[4] = g * (q0.x * q0.x + q0.y * q0.y + q1.x * q1.x + q1.y * q1.y + q2.x * q2.x + q2.y * q2.y);
                v[5] = g * (jr * jr + ji * ji);
                v[6] = g * (d.x * ji - d.y * jr);
            }
        }
        flush_runs<kBinVals, T>(bin, v, s_bins, nbins);
    }
    __syncthreads();
    double *out = partials + static_cast<int64_t>(blockIdx.x) * kBinVals * nbins;
    for (int k = threadIdx.x; k < kBinVals * nbins; k += blockDim.x) out[k] = s_bins[k];
}

// (hi, lo) += (bh, bl) for unevaluated float pairs: a two-sum of the high parts, then
// the low parts and the rounding error added and renormalised.
__device__ __forceinline__ void pair_add(float &hi, float &lo, float bh, float bl)
{
    const float sh = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(sh, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(sh, bb)), __fsub_rn(bh, bb));
    const float t = __fadd_rn(se, __fadd_rn(lo, bl));
    hi = __fadd_rn(sh, t);
    lo = __fsub_rn(t, __fsub_rn(hi, sh));
}
__device__ __forceinline__ void pair_add(double &hi, double &lo, double bh, double bl)
{
    hi = (hi + lo) + (bh + bl);  // FP64: plain adds
    lo = 0.0;
}

// Warp sums of 8 values per lane (value k as the pair hi[k] + lo[k]) by reduce-scatter:
// at the steps across lanes 16, 8 and 4 apart each lane keeps half of the values it
// still holds and adds its partner's copy of them, then the lanes 2 and 1 apart add their
// single values. Lane L ends with the sum of value ((L >> 2) & 7) over the warp, the
// same in lanes 4k..4k+3; 9 pair additions per lane instead of 40 for eight butterflies.
// Returned as FP64; fixed order.
template <typename T>
__device__ __forceinline__ double warp_scatter_sum8(T (&hi)[8], T (&lo)[8])
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int half = 4, o = 16; half >= 1; half >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;  // keeps the upper half of its values
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const T mh = up ? hi[j + half] : hi[j], ml = up ? lo[j + half] : lo[j];
            const T sh = up ? hi[j] : hi[j + half], sl = up ? lo[j] : lo[j + half];
            const T rh = __shfl_xor_sync(full, sh, o), rl = __shfl_xor_sync(full, sl, o);
            hi[j] = mh, lo[j] = ml;
            pair_add(hi[j], lo[j], rh, rl);
        }
    }
#pragma unroll
    for (int o = 2; o >= 1; o >>= 1) {
        const T rh = __shfl_xor_sync(full, hi[0], o), rl = __shfl_xor_sync(full, lo[0], o);
        pair_add(hi[0], lo[0], rh, rl);
    }
    return static_cast<double>(hi[0]) + static_cast<double>(lo[0]);
}

// floor(sqrt(x)) for 0 <= x < 2^24, exact
__device__ __forceinline__ int isqrt_floor(int x)
{
    int r = static_cast<int>(sqrtf(static_cast<float>(x)));
    while (r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return r;
}

// Shell-major binning. Work item (n0, b): all modes of shell b in the slab n_x = n0,
// one warp per item, so each lane keeps one set of sums for the whole item. Items are
// taken slab by slab, so the items running together read the same few slabs (which
// stay in L2); items that hold no mode are not run. The shell is the integer interval
// thresh[b] <= |n|^2 < thresh[b + 1]; in each row (n0, n1) its modes form one run of l,
// found with exact integer square roots (no mode is tested against a table). The runs
// of 32 rows are laid end to end and the warp walks the joined list in windows of 32
// modes, two windows per pass (lane j takes the j-th mode of each), so all lanes work
// and consecutive lanes read consecutive modes of a row. The seven per-mode
// values are summed with Kahan-compensated adds in the grid precision; one warp
// reduce-scatter per item (float pairs for FP32) writes partials[item][kBinVals] in FP64,
// and k_reduce_items adds the items of each shell in a fixed order.
// Per-warp staging of the rows of one item (k_bin_shells, k_bin_batch): the non-empty
// rows of a group of 32, in order, each as (first mode's index in the joined list, first
// l, n1, then for FP32 the bits of the row's factor g0 * gf[i1], for FP64 i1), one
// 16-byte load.
struct BinWarpStage {
    int4 rows[32];
};

// One item (n0 = slab i0, shell b) of the shell-major binning, by one warp: writes
// partials[item][kBinVals] (item = i0 * nbins + b).
template <typename T>
__device__ __forceinline__ void bin_item(const Cx<T> *__restrict__ F, int64_t gstride, int ng, int nbins,
                                         const int *__restrict__ thresh, const T *__restrict__ gf,
                                         const T *__restrict__ gh, T vb0, T vb1, T vb2, double *__restrict__ partials,
                                         int item, BinWarpStage &st)
{
    const int nh = ng / 2 + 1;
    const int lane = threadIdx.x & 31;
    if (!PK_IN(item, static_cast<int64_t>(ng) * nbins, kChkBin)) return;  // warp-uniform
    const int b = item % nbins;
    const int i0 = item / nbins;
    const int n0 = i0 < ng / 2 ? i0 : i0 - ng;
    const int lo2 = thresh[b], hi2 = thresh[b + 1];  // lo2 <= |n|^2 < hi2
    T s[kBinVals], c[kBinVals];
#pragma unroll
    for (int k = 0; k < kBinVals; ++k) s[k] = T(0), c[k] = T(0);
    const int rem = hi2 - 1 - n0 * n0;
    if (hi2 <= lo2 || rem < 0) {  // the shell misses this slab: zero sums, no reduction
        if (lane < kBinVals) partials[static_cast<int64_t>(item) * kBinVals + lane] = 0.0;
        return;
    }
    {
        const int R1 = isqrt_floor(rem);
        const int n1lo = max(-ng / 2, -R1), n1hi = min(ng / 2 - 1, R1);
        const T g0 = gf[i0];
        for (int r0 = n1lo; r0 <= n1hi; r0 += 32) {
            const int n1 = r0 + lane;
            const bool row = n1 <= n1hi;
            int l_lo = 0, len = 0;
            if (row) {
                const int r2 = n0 * n0 + n1 * n1;
                const int top = hi2 - 1 - r2;  // l^2 <= top
                if (top >= 0) {
                    const int lh = min(isqrt_floor(top), nh - 1);
                    const int need = lo2 - r2;  // l^2 >= need
                    const int ll = need <= 0 ? 0 : isqrt_floor(need - 1) + 1;
                    if (lh >= ll) l_lo = ll, len = lh - ll + 1;
                }
            }
            int inc = len;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += t;
            }
            const int total = __shfl_sync(0xffffffffu, inc, 31);
            if (total == 0) continue;
            const int pre = inc - len;
            const unsigned nonempty = __ballot_sync(0xffffffffu, len > 0);
            if (len > 0) {  // compacted: the k-th non-empty row at index k
                const int i1 = n1 < 0 ? n1 + ng : n1;
                int w;
                if constexpr (sizeof(T) == 4) w = static_cast<int>(__float_as_uint(g0 * gf[i1]));
                else w = i1;
                st.rows[__popc(nonempty & ((1u << lane) - 1u))] = make_int4(pre, l_lo, n1, w);
            }
            __syncwarp();
            for (int m0 = 0; m0 < total; m0 += 64) {
                // two windows of 32 modes per pass (8 loads in flight per lane); the row
                // holding mode m = w0 + lane: non-empty rows start at increasing positions,
                // so it is the last one starting at or before m: count the rows started
                // before the window and the starts in it up to m
                int mm[2], mlo[2], mn1[2];
                int64_t mi[2];
                bool ok[2];
                T grow[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int w0 = m0 + 32 * h;
                    const bool in_win = len > 0 && pre >= w0 && pre < w0 + 32;
                    const unsigned starts = __reduce_or_sync(0xffffffffu, in_win ? 1u << (pre - w0) : 0u);
                    const int before = __popc(__ballot_sync(0xffffffffu, len > 0 && pre < w0));
                    mm[h] = w0 + lane;
                    ok[h] = mm[h] < total;
                    const int q = before + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
                    const int4 rw = st.rows[ok[h] ? q : 0];
                    mlo[h] = rw.y + (mm[h] - rw.x);
                    mn1[h] = rw.z;
                    const int ri1 = rw.z < 0 ? rw.z + ng : rw.z;
                    mi[h] = (static_cast<int64_t>(i0) * ng + ri1) * nh + mlo[h];
                    if (ok[h] && (!PK_IN(mi[h], gstride, kChkMode) || !PK_IN(mlo[h], nh, kChkMode))) ok[h] = false;
                    if constexpr (sizeof(T) == 4) grow[h] = __uint_as_float(static_cast<unsigned>(rw.w));
                    else grow[h] = g0 * gf[ri1];
                }
                Cx<T> dd[2], pp0[2], pp1[2], pp2[2];
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (ok[h]) {
                        dd[h] = F[mi[h]], pp0[h] = F[gstride + mi[h]], pp1[h] = F[2 * gstride + mi[h]],
                        pp2[h] = F[3 * gstride + mi[h]];
                    }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!ok[h]) continue;
                    const int l = mlo[h];
                    const Cx<T> d = dd[h], p0 = pp0[h], p1 = pp1[h], p2 = pp2[h];
                    const T g = grow[h] * gh[l] * ((l == 0 || l == nh - 1) ? T(1) : T(2));
                    const T fn0 = static_cast<T>(n0), fn1 = static_cast<T>(mn1[h]), fn2 = static_cast<T>(l);
                    const T kr = fn0 * p0.x + fn1 * p1.x + fn2 * p2.x;
                    const T ki = fn0 * p0.y + fn1 * p1.y + fn2 * p2.y;
                    const Cx<T> q0{p0.x - vb0 * d.x, p0.y - vb0 * d.y};
                    const Cx<T> q1{p1.x - vb1 * d.x, p1.y - vb1 * d.y};
                    const Cx<T> q2{p2.x - vb2 * d.x, p2.y - vb2 * d.y};
                    const T jr = fn0 * q0.x + fn1 * q1.x + fn2 * q2.x;
                    const T ji = fn0 * q0.y + fn1 * q1.y + fn2 * q2.y;
                    T v[kBinVals];
                    v[0] = g * (d.x * d.x + d.y * d.y);
                    v[1] = g * (p0.x * p0.x + p0.y * p0.y + p1.x * p1.x + p1.y * p1.y + p2.x * p2.x + p2.y * p2.y);
                    v[2] = g * (kr * kr + ki * ki);
                    v[3] = g * (d.x * ki - d.y * kr);  // Im(conj(F_d) * (n.F_p))
                    v[4] = g * (q0.x * q0.x + q0.y * q0.y + q1.x * q1.x + q1.y * q1.y + q2.x * q2.x + q2.y * q2.y);
                    v[5] = g * (jr * jr + ji * ji);
                    v[6] = g * (d.x * ji - d.y * jr);
#pragma unroll
                    for (int k = 0; k < kBinVals; ++k) {  // Kahan: s - c carries the sum
                        const T y = v[k] - c[k];
                        const T t = s[k] + y;
                        c[k] = (t - s[k]) - y;
                        s[k] = t;
                    }
                }
            }
            __syncwarp();
        }
    }
    static_assert(kBinVals <= 8, "the reduce-scatter sums 8 values");
    T hi[8], lo[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) hi[k] = k < kBinVals ? s[k] : T(0), lo[k] = k < kBinVals ? -c[k] : T(0);
    const double dsum = warp_scatter_sum8(hi, lo);
    const int k = (lane >> 2) & 7;
    if ((lane & 3) == 0 && k < kBinVals) partials[static_cast<int64_t>(item) * kBinVals + k] = dsum;
}

// Warps draw items from a device counter, one at a time (taking the next index before
// finishing the current item measured slower), in the order of the table's list of
// non-empty items, so the large items of the central slabs are spread first and the
// small ones fill the tail. Which warp takes an item does not change its result. The
// last block to finish sets the counter back to zero for the next launch.
template <typename T>
__global__ void __launch_bounds__(kBinThreads, sizeof(T) == 4 ? 4 : 2)
k_bin_shells(const Cx<T> *__restrict__ F, int64_t gstride, int ng, int nbins, const int *__restrict__ thresh,
             const T *__restrict__ gf, const T *__restrict__ gh, const double *__restrict__ mom,
             const uint32_t *__restrict__ order, int nwork, unsigned *__restrict__ counter,
             double *__restrict__ partials)
{
    constexpr int NW = kBinThreads / 32;
    __shared__ BinWarpStage s_st[NW];
    const double Mtot = mom[0];
    const T vb0 = static_cast<T>(mom[2] / Mtot), vb1 = static_cast<T>(mom[3] / Mtot), vb2 = static_cast<T>(mom[4] / Mtot);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned j = 0;
        if (lane == 0) j = atomicAdd(counter, 1u);
        j = __shfl_sync(0xffffffffu, j, 0);
        if (j >= static_cast<unsigned>(nwork)) break;
        bin_item<T>(F, gstride, ng, nbins, thresh, gf, gh, vb0, vb1, vb2, partials, static_cast<int>(order[j]),
                    s_st[w]);
    }
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(counter + 1, 1u) == gridDim.x - 1) counter[0] = 0u, counter[1] = 0u;
}

// Persistent form over the non-empty items of many FP32 catalogues (the batched
// estimate), drawn from one counter in catalogue order; each item is written to its own
// catalogue's partials, so the results do not depend on which warp took it.
__global__ void __launch_bounds__(kBinThreads, 4)
k_bin_batch(const BinBatch jobs)
{
    constexpr int NW = kBinThreads / 32;
    __shared__ BinWarpStage s_st[NW];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int jj = 0;
    for (;;) {
        unsigned nx = 0;
        if (lane == 0) nx = atomicAdd(jobs.counter, 1u);
        const long long item = __shfl_sync(0xffffffffu, nx, 0);
        if (item >= jobs.total_items) break;
        while (jj + 1 < jobs.n && jobs.job[jj + 1].first_item <= item) ++jj;  // items only grow
        const BinJob &jb = jobs.job[jj];
        const double Mtot = jb.mom[0];
        const float vb0 = static_cast<float>(jb.mom[2] / Mtot), vb1 = static_cast<float>(jb.mom[3] / Mtot),
                    vb2 = static_cast<float>(jb.mom[4] / Mtot);
        const int nh = jb.ng / 2 + 1;
        const int64_t gstride = static_cast<int64_t>(jb.ng) * jb.ng * nh;
        bin_item<float>(static_cast<const Cx<float> *>(jb.grids), gstride, jb.ng, jb.nbins, jb.thresh, jb.gf, jb.gh,
                        vb0, vb1, vb2, jb.partials, static_cast<int>(jb.order[item - jb.first_item]), s_st[w]);
    }
}

// out[k * nbins + b] = sum over slabs j of partials[(j * nbins + b) * NV + k], fixed order.
// With thresh: column b belongs to shell b / per_shell, and the slabs that shell misses
// hold no modes and are skipped (their partials are never written).
template <int NV>
__global__ void __launch_bounds__(256)
k_reduce_items(const double *__restrict__ partials, int nslabs, int nbins, double *__restrict__ out,
               const int *__restrict__ thresh = nullptr, int per_shell = 1)
{
    const int b = blockIdx.x;
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = 0.0;
    const int sh = b / per_shell;
    const int hi2 = thresh ? thresh[sh + 1] : 0, lo2 = thresh ? thresh[sh] : 0;
    for (int j = threadIdx.x; j < nslabs; j += blockDim.x) {
        const int n0 = j < nslabs / 2 ? j : j - nslabs;
        if (thresh && (hi2 <= lo2 || hi2 - 1 - n0 * n0 < 0)) continue;
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] += partials[(static_cast<int64_t>(j) * nbins + b) * NV + k];
    }
    __shared__ double red[NV][256];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < NV; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < NV) out[threadIdx.x * nbins + b] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(kBinThreads)
k_mode_sums(int ng, uint32_t nmodes, const uint16_t *__restrict__ bintab, int nsq_max, const double *__restrict__ hf,
            const double *__restrict__ hh, int nbins, double *__restrict__ partials)
{
    extern __shared__ double s_bins[];  // [kModeVals][nbins]
    for (int k = threadIdx.x; k < kModeVals * nbins; k += blockDim.x) s_bins[k] = 0.0;
    __syncthreads();
    const int nh = ng / 2 + 1;
    const int lane = threadIdx.x & 31;
    const uint32_t nchunks = (nmodes + 31u) / 32u;
    const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t ch = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ch < nchunks; ch += nwarps) {
        const uint32_t mode = ch * 32u + lane;
        int bin = -1;
        double v[kModeVals];
#pragma unroll
        for (int k = 0; k < kModeVals; ++k) v[k] = 0.0;
        if (mode < nmodes) {
            int i0, i1, l;
            chunk_mode(ch, lane, ng, nh, i0, i1, l);
            const int n0 = i0 < ng / 2 ? i0 : i0 - ng;
            const int n1 = i1 < ng / 2 ? i1 : i1 - ng;
            const int nsq = n0 * n0 + n1 * n1 + l * l;
            const int b = nsq <= nsq_max ? static_cast<int>(bintab[nsq]) : 0xffff;
            if (b != 0xffff) {
                bin = b;
                const double w = (l == 0 || l == nh - 1) ? 1.0 : 2.0;
                const double h = w * hf[i0] * hf[i1] * hh[l];
                const double a0 = n0, a1 = n1, a2 = l;
                v[0] = w;
                v[1] = w * sqrt(static_cast<double>(nsq));
                v[2] = h;
                v[3] = h * a0 * a0;
                v[4] = h * a1 * a1;
                v[5] = h * a2 * a2;
                v[6] = h * a0 * a1;
                v[7] = h * a0 * a2;
                v[8] = h * a1 * a2;
            }
        }
        flush_runs<kModeVals, double>(bin, v, s_bins, nbins);
    }
    __syncthreads();
    double *out = partials + static_cast<int64_t>(blockIdx.x) * kModeVals * nbins;
    for (int k = threadIdx.x; k < kModeVals * nbins; k += blockDim.x) out[k] = s_bins[k];
}

// One block per shell: out[k * nbins + b] = sum_j partials[j][k][b], fixed order.
template <int NV>
__global__ void __launch_bounds__(256)
k_reduce_partials(const double *__restrict__ partials, int nblk, int nbins, double *__restrict__ out)
{
    const int b = blockIdx.x;
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = 0.0;
    for (int j = threadIdx.x; j < nblk; j += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] += partials[(static_cast<int64_t>(j) * NV + k) * nbins + b];
    __shared__ double red[NV][256];
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < NV; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < NV) out[threadIdx.x * nbins + b] = red[threadIdx.x][0];
}

struct FinalParams {
    double V, kf, ts;
    int sub, bulk, iso, nbins;
};

// sum_ab Q_ab H_ab for symmetric Q, H stored as xx, yy, zz, xy, xz, yz
__device__ __forceinline__ double qdot(const double *Q, const double *H)
{
    return Q[0] * H[0] + Q[1] * H[1] + Q[2] * H[2] + 2.0 * (Q[3] * H[3] + Q[4] * H[4] + Q[5] * H[5]);
}

__global__ void k_finalize(const double *__restrict__ sums /*[kBinVals][nbins]*/,
                           const double *__restrict__ modes /*[kModeVals][nbins]*/, const double *__restrict__ mom,
                           FinalParams fp, double *__restrict__ out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int nb = fp.nbins;
    if (b >= nb) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const double n = modes[b];
    auto put = [&](int row, double v) { out[row * nb + b] = v; };
    put(PKMOM_ROW_NMODES, n);
    if (!(n > 0.0)) {
        for (int r = 0; r < PKMOM_NROWS; ++r)
            if (r != PKMOM_ROW_NMODES) put(r, nan);
        return;
    }
    const double M = mom[0], S2 = mom[1];
    const double vb[3] = {mom[2] / M, mom[3] / M, mom[4] / M};
    const double R[3] = {mom[5], mom[6], mom[7]};
    const double *Q = mom + 8;
    const double H = modes[2 * nb + b];
    double H2[6];
    for (int k = 0; k < 6; ++k) H2[k] = modes[(3 + k) * nb + b];
    const double c = fp.V / (M * M * n);
    const double ct = c * fp.ts * fp.ts * fp.kf * fp.kf;
    const double cx = c * fp.ts * fp.kf;
    const double sub = fp.sub ? 1.0 : 0.0;
    const double trH2 = H2[0] + H2[1] + H2[2];

    put(PKMOM_ROW_K, fp.kf * modes[nb + b] / n);
    const double sn_dd = c * S2 * H;
    put(PKMOM_ROW_PDD, c * sums[0 * nb + b] - sub * sn_dd);
    put(PKMOM_ROW_SNDD, sn_dd);

    const double trQ = Q[0] + Q[1] + Q[2];
    const double sn_pp = c * trQ * H;
    const double sn_tt = ct * (fp.iso ? trQ * trH2 / 3.0 : qdot(Q, H2));
    put(PKMOM_ROW_PPP, c * sums[1 * nb + b] - sub * sn_pp);
    put(PKMOM_ROW_PTT, ct * sums[2 * nb + b] - sub * sn_tt);
    put(PKMOM_ROW_PDT, cx * sums[3 * nb + b]);
    put(PKMOM_ROW_SNPP, sn_pp);
    put(PKMOM_ROW_SNTT, sn_tt);

    if (fp.bulk) {
        // Q' = sum m^2 (v - v_b)(v - v_b)^T = Q - v_b R^T - R v_b^T + v_b v_b^T S2 (Sec. 3.1)
        const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
        double Qb[6];
        for (int k = 0; k < 6; ++k)
            Qb[k] = Q[k] - vb[ia[k]] * R[ib[k]] - R[ia[k]] * vb[ib[k]] + vb[ia[k]] * vb[ib[k]] * S2;
        const double trQb = Qb[0] + Qb[1] + Qb[2];
        const double sn_ppb = c * trQb * H;
        const double sn_ttb = ct * (fp.iso ? trQb * trH2 / 3.0 : qdot(Qb, H2));
        put(PKMOM_ROW_PPP_B, c * sums[4 * nb + b] - sub * sn_ppb);
        put(PKMOM_ROW_PTT_B, ct * sums[5 * nb + b] - sub * sn_ttb);
        put(PKMOM_ROW_PDT_B, cx * sums[6 * nb + b]);
        put(PKMOM_ROW_SNPP_B, sn_ppb);
        put(PKMOM_ROW_SNTT_B, sn_ttb);
    } else {
        const int rows[5] = {PKMOM_ROW_PPP_B, PKMOM_ROW_PTT_B, PKMOM_ROW_PDT_B, PKMOM_ROW_SNPP_B, PKMOM_ROW_SNTT_B};
        for (int r = 0; r < 5; ++r) put(rows[r], nan);
    }
}

// ---------------------------------------------------------------- host tables
// B_{2m}(n) at the integers, n = 0..m (textbook values of the centred cardinal
// B-splines of even order 2, 4, 6, 8), giving Sigma_m(w) = sum_n B_2m(n) cos(n w).
const double *euler_frobenius(int m)
{
    static const double b2[] = {1.0};
    static const double b4[] = {2.0 / 3.0, 1.0 / 6.0};
    static const double b6[] = {11.0 / 20.0, 13.0 / 60.0, 1.0 / 120.0};
    static const double b8[] = {151.0 / 315.0, 397.0 / 1680.0, 1.0 / 42.0, 1.0 / 5040.0};
    static const double b10[] = {15619.0 / 36288.0, 44117.0 / 181440.0, 913.0 / 22680.0, 251.0 / 181440.0,
                                 1.0 / 362880.0};
    switch (m) {
    case 1: return b2;
    case 2: return b4;
    case 3: return b6;
    case 4: return b8;
    case 5: return b10;
    default: return nullptr;
    }
}

double sigma_m(double w, int m)
{
    const double *c = euler_frobenius(m);
    double s = c[0];
    for (int n = 1; n < m; ++n) s += 2.0 * c[n] * std::cos(n * w);
    return s;
}

double bhat2(double w, int m)
{
    const double x = 0.5 * w;
    const double sx = x == 0.0 ? 1.0 : std::sin(x) / x;
    double r = 1.0;
    for (int k = 0; k < m; ++k) r *= sx;
    return r * r;
}

template <typename T>
cudaError_t upload(void **dst, const std::vector<T> &src)
{
    cudaError_t e = cudaMalloc(dst, src.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

void free_spectra_tables(SpectraTables &t)
{
    cudaFree(t.bintab);
    cudaFree(t.thresh);
    cudaFree(t.g_full);
    cudaFree(t.g_half);
    cudaFree(t.h_full);
    cudaFree(t.h_half);
    cudaFree(t.mode_sums);
    cudaFree(t.partials);
    cudaFree(t.item_partials);
    cudaFree(t.bin_order);
    cudaFree(t.bin_counter);
    t = SpectraTables{};
}

cudaError_t build_spectra_tables(SpectraTables &t, int ng, int order, bool direct, int nbins, double umin,
                                 double umax, int prec, int num_sms, cudaStream_t s, LaunchStats &st)
{
    t.ng = ng;
    t.order = order;
    t.direct = direct;
    t.nbins = nbins;
    t.umin = umin;
    t.umax = umax;
    t.prec = prec;
    const int nh = ng / 2 + 1;
    std::vector<uint16_t> bintab;
    std::vector<int> thresh;
    t.nsq_max = shell_tables(nbins, umin, umax, bintab, thresh);
    std::vector<double> gfd(ng), ghd(nh), hfd(ng), hhd(nh);
    for (int i = 0; i < ng; ++i) {
        const int ni = i < ng / 2 ? i : i - ng;
        const double w = kTwoPi * ni / ng;
        hfd[i] = sigma_m(w, order) / bhat2(w, order);
        // B-spline grids carry the BL field times prod Sigma^{-1/2}: 1/W^2 of the BL field
        // is then 1/Bhat^2 per axis; grids assigned with the BL function itself take
        // 1/W^2 = Sigma/Bhat^2
        gfd[i] = direct ? hfd[i] : 1.0 / bhat2(w, order);
    }
    for (int i = 0; i < nh; ++i) {
        const double w = kTwoPi * i / ng;
        hhd[i] = sigma_m(w, order) / bhat2(w, order);
        ghd[i] = direct ? hhd[i] : 1.0 / bhat2(w, order);
    }
    cudaError_t e;
    if ((e = upload(reinterpret_cast<void **>(&t.bintab), bintab)) != cudaSuccess) return e;
    if ((e = upload(reinterpret_cast<void **>(&t.thresh), thresh)) != cudaSuccess) return e;
    if (prec == PKMOM_F32) {
        std::vector<float> gf(gfd.begin(), gfd.end()), gh(ghd.begin(), ghd.end());
        if ((e = upload(&t.g_full, gf)) != cudaSuccess) return e;
        if ((e = upload(&t.g_half, gh)) != cudaSuccess) return e;
    } else {
        if ((e = upload(&t.g_full, gfd)) != cudaSuccess) return e;
        if ((e = upload(&t.g_half, ghd)) != cudaSuccess) return e;
    }
    if ((e = upload(reinterpret_cast<void **>(&t.h_full), hfd)) != cudaSuccess) return e;
    if ((e = upload(reinterpret_cast<void **>(&t.h_half), hhd)) != cudaSuccess) return e;

    const uint32_t nmodes = static_cast<uint32_t>(static_cast<int64_t>(ng) * ng * nh);
    const uint32_t nchunks = (nmodes + 31u) / 32u;
    const int warps_per_block = kBinThreads / 32;
    int64_t want = (nchunks + warps_per_block - 1) / warps_per_block;
    const int64_t cap = static_cast<int64_t>(num_sms) * 8;
    t.bin_blocks = static_cast<int>(want < cap ? want : cap);
    if (t.bin_blocks < 1) t.bin_blocks = 1;
    if ((e = cudaMalloc(reinterpret_cast<void **>(&t.partials),
                        static_cast<size_t>(t.bin_blocks) * kModeVals * nbins * sizeof(double))) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(reinterpret_cast<void **>(&t.mode_sums), static_cast<size_t>(kModeVals + kBinVals) * nbins *
                                                                       sizeof(double))) != cudaSuccess)
        return e;
    if ((e = cudaMalloc(reinterpret_cast<void **>(&t.item_partials),
                        static_cast<size_t>(ng) * nbins * kBinVals * sizeof(double))) != cudaSuccess)
        return e;
    // the non-empty (slab, shell) items (the same test as bin_item's)
    std::vector<uint32_t> work = bin_item_list(thresh, ng, nbins);
    t.bin_nwork = static_cast<int>(work.size());
    if (work.empty()) work.push_back(0);  // keep a valid allocation
    if ((e = upload(reinterpret_cast<void **>(&t.bin_order), work)) != cudaSuccess) return e;
    if ((e = cudaMalloc(reinterpret_cast<void **>(&t.bin_counter), 4 * sizeof(unsigned))) != cudaSuccess) return e;
    if ((e = cudaMemset(t.bin_counter, 0, 4 * sizeof(unsigned))) != cudaSuccess) return e;
    t.shell_blocks = num_sms * 4;  // resident blocks (56 registers, 256 threads)
    t.bytes = work.size() * sizeof(uint32_t) + 4 * sizeof(unsigned) + bintab.size() * sizeof(uint16_t) +
              thresh.size() * sizeof(int) +
              static_cast<size_t>(ng + nh) * (prec == PKMOM_F32 ? sizeof(float) : sizeof(double)) +
              static_cast<size_t>(ng + nh) * sizeof(double) +
              static_cast<size_t>(t.bin_blocks) * kModeVals * nbins * sizeof(double) +
              static_cast<size_t>(kModeVals + kBinVals) * nbins * sizeof(double) +
              static_cast<size_t>(ng) * nbins * kBinVals * sizeof(double);
    const size_t smem = static_cast<size_t>(kModeVals) * nbins * sizeof(double);
    if ((e = cudaFuncSetAttribute(k_mode_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem))) !=
        cudaSuccess)
        return e;
    k_mode_sums<<<t.bin_blocks, kBinThreads, smem, s>>>(ng, nmodes, t.bintab, t.nsq_max, t.h_full, t.h_half, nbins,
                                                        t.partials);
    k_reduce_partials<kModeVals><<<nbins, 256, 0, s>>>(t.partials, t.bin_blocks, nbins, t.mode_sums);
    st.launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t launch_bin(const SpectraTables &t, const void *grids, const double *moments_dev, cudaStream_t s,
                       LaunchStats &st)
{
    const int ng = t.ng, nh = ng / 2 + 1;
    const uint32_t nmodes = static_cast<uint32_t>(static_cast<int64_t>(ng) * ng * nh);
    const int64_t gstride = static_cast<int64_t>(ng) * ng * nh;  // complex elements per grid
    const size_t smem = static_cast<size_t>(kBinVals) * t.nbins * sizeof(double);
    cudaError_t e;
    if (t.prec == PKMOM_F32) {
        if (smem > 48 * 1024 && (e = cudaFuncSetAttribute(k_bin<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          static_cast<int>(smem))) != cudaSuccess)
            return e;
        k_bin<float><<<t.bin_blocks, kBinThreads, smem, s>>>(
            static_cast<const Cx<float> *>(grids), gstride, ng, nmodes, t.bintab, t.nsq_max,
            static_cast<const float *>(t.g_full), static_cast<const float *>(t.g_half), moments_dev, t.nbins,
            t.partials);
    } else {
        if (smem > 48 * 1024 && (e = cudaFuncSetAttribute(k_bin<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          static_cast<int>(smem))) != cudaSuccess)
            return e;
        k_bin<double><<<t.bin_blocks, kBinThreads, smem, s>>>(
            static_cast<const Cx<double> *>(grids), gstride, ng, nmodes, t.bintab, t.nsq_max,
            static_cast<const double *>(t.g_full), static_cast<const double *>(t.g_half), moments_dev, t.nbins,
            t.partials);
    }
    st.launches++;
    return cudaGetLastError();
}

cudaError_t launch_bin_shells(const SpectraTables &t, const void *grids, const double *moments_dev, cudaStream_t s,
                              LaunchStats &st)
{
    const int ng = t.ng, nh = ng / 2 + 1;
    const int64_t gstride = static_cast<int64_t>(ng) * ng * nh;
    const unsigned blocks = static_cast<unsigned>(t.shell_blocks);
    if (t.prec == PKMOM_F32)
        k_bin_shells<float><<<blocks, kBinThreads, 0, s>>>(
            static_cast<const Cx<float> *>(grids), gstride, ng, t.nbins, t.thresh,
            static_cast<const float *>(t.g_full), static_cast<const float *>(t.g_half), moments_dev, t.bin_order,
            t.bin_nwork, t.bin_counter, t.item_partials);
    else
        k_bin_shells<double><<<blocks, kBinThreads, 0, s>>>(
            static_cast<const Cx<double> *>(grids), gstride, ng, t.nbins, t.thresh,
            static_cast<const double *>(t.g_full), static_cast<const double *>(t.g_half), moments_dev, t.bin_order,
            t.bin_nwork, t.bin_counter, t.item_partials);
    double *sums = t.mode_sums + static_cast<size_t>(kModeVals) * t.nbins;
    k_reduce_items<kBinVals><<<t.nbins, 256, 0, s>>>(t.item_partials, ng, t.nbins, sums, t.thresh);
    st.launches += 2;
    return cudaGetLastError();
}

namespace {
// k_finalize of shell sums `sums` ([kBinVals][nbins]) with the table's mode sums.
cudaError_t finalize_sums(const SpectraTables &t, const pkmom_params &p, const double *moments_dev,
                          const double *sums, double *out, cudaStream_t s, LaunchStats &st)
{
    FinalParams fp;
    fp.V = p.box_L * p.box_L * p.box_L;
    fp.kf = kTwoPi / p.box_L;
    fp.ts = p.theta_scale;
    fp.sub = p.subtract_shot_noise;
    fp.bulk = p.bulk;
    fp.iso = p.theta_sn_mode == 1;
    fp.nbins = t.nbins;
    k_finalize<<<(t.nbins + 127) / 128, 128, 0, s>>>(sums, t.mode_sums, moments_dev, fp, out);
    st.launches++;
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_bin_batch(BinBatch &batch, const SpectraTables *const *tables, const pkmom_params *const *params,
                             double *const *sums_of, double *const *out, int num_sms, cudaStream_t s,
                             LaunchStats &st)
{
    long long first = 0;
    for (int k = 0; k < batch.n; ++k) {
        batch.job[k].order = tables[k]->bin_order;
        batch.job[k].nwork = tables[k]->bin_nwork;
        batch.job[k].first_item = first;
        first += tables[k]->bin_nwork;
    }
    batch.total_items = first;
    cudaError_t e;
    if (first > 0) {
        const long long want = (first + kBinThreads / 32 - 1) / (kBinThreads / 32);
        const unsigned blocks = static_cast<unsigned>(std::min<long long>(want, static_cast<long long>(num_sms) * 4));
        if ((e = cudaMemsetAsync(batch.counter, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
        k_bin_batch<<<blocks, kBinThreads, 0, s>>>(batch);
        st.launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int k = 0; k < batch.n; ++k) {
        const BinJob &jb = batch.job[k];
        k_reduce_items<kBinVals><<<jb.nbins, 256, 0, s>>>(jb.partials, jb.ng, jb.nbins, sums_of[k], jb.thresh);
        st.launches++;
        if ((e = finalize_sums(*tables[k], *params[k], jb.mom, sums_of[k], out[k], s, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_finalize(const SpectraTables &t, const pkmom_params &p, const double *moments_dev, double *out,
                            cudaStream_t s, LaunchStats &st, bool sums_ready)
{
    double *sums = t.mode_sums + static_cast<size_t>(kModeVals) * t.nbins;
    if (!sums_ready) {
        k_reduce_partials<kBinVals><<<t.nbins, 256, 0, s>>>(t.partials, t.bin_blocks, t.nbins, sums);
        st.launches++;
    }
    FinalParams fp;
    fp.V = p.box_L * p.box_L * p.box_L;
    fp.kf = kTwoPi / p.box_L;
    fp.ts = p.theta_scale;
    fp.sub = p.subtract_shot_noise;
    fp.bulk = p.bulk;
    fp.iso = p.theta_sn_mode == 1;
    fp.nbins = t.nbins;
    k_finalize<<<(t.nbins + 127) / 128, 128, 0, s>>>(sums, t.mode_sums, moments_dev, fp, out);
    st.launches++;
    return cudaGetLastError();
}

}  // namespace pkmom

// ---------------------------------------------------------------------------
// pkmom_spectra_static: step 4 without any device allocation.
//
// Some callers cannot allocate device memory while they run: a host process that
// owns a fixed memory pool and forbids allocator calls, or a plug-in that must not
// grow the device footprint of the program it runs in after start-up. For them this entry point keeps all of its
// scratch (shell table, window tables, per-block partial sums, shell sums) in one
// file-scope device array of kStaticScratchBytes. Every GPU that loads the library
// holds that array until the process exits. The caller passes the transformed grids,
// the moments and the output, as for pkmom_spectra.
//
// The first call on a device looks up the array's device address for that device
// (cudaGetSymbolAddress) with the device current; make that first call before any
// stream capture. All calls share the one array and each call overwrites what it
// uses (the previous call's contents remain until then, and everything that must
// start at zero is cleared by the call itself), so calls whose work overlaps on the
// GPU (different streams without ordering, or several host threads) race with each
// other.
namespace pkmom {
namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr int kStaticMaxBins = 256;
constexpr int kStaticBlocks = 64;  // CTAs of the binning kernels on this path

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

__device__ const double kEF1[1] = {1.0};
__device__ const double kEF2[2] = {2.0 / 3.0, 1.0 / 6.0};
__device__ const double kEF3[3] = {11.0 / 20.0, 13.0 / 60.0, 1.0 / 120.0};
__device__ const double kEF4[4] = {151.0 / 315.0, 397.0 / 1680.0, 1.0 / 42.0, 1.0 / 5040.0};
__device__ const double kEF5[5] = {15619.0 / 36288.0, 44117.0 / 181440.0, 913.0 / 22680.0, 251.0 / 181440.0,
                                   1.0 / 362880.0};

// The shell table and the per-axis window factors, built on the device in FP64 with
// the same expressions as build_spectra_tables (correctly rounded sqrt and division,
// so the shell of every |n|^2 is the same).
template <typename T>
__global__ void k_static_tables(int ng, int order, bool direct, int nbins, double umin, double umax, int nsq_max,
                                uint16_t *__restrict__ bintab, T *__restrict__ gf, T *__restrict__ gh,
                                double *__restrict__ hf, double *__restrict__ hh)
{
    const double *ef = order == 1 ? kEF1 : order == 2 ? kEF2 : order == 3 ? kEF3 : order == 4 ? kEF4 : kEF5;
    const int nh = ng / 2 + 1;
    const int stride = gridDim.x * blockDim.x;
    for (int nsq = blockIdx.x * blockDim.x + threadIdx.x; nsq <= nsq_max; nsq += stride) {
        uint16_t b = 0xffff;
        if (nsq > 0) {
            const double u = sqrt(static_cast<double>(nsq));
            if (u >= umin && u <= umax) {
                double tb = floor(((u - umin) * nbins) / (umax - umin));
                if (tb > nbins - 1) tb = nbins - 1;
                b = static_cast<uint16_t>(tb);
            }
        }
        bintab[nsq] = b;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ng + nh; i += stride) {
        const bool full = i < ng;
        const int j = full ? i : i - ng;
        const int nj = full ? (j < ng / 2 ? j : j - ng) : j;
        const double w = kTwoPi * nj / ng;
        double s = ef[0];
        for (int n = 1; n < order; ++n) s += 2.0 * ef[n] * cos(n * w);
        const double x = 0.5 * w;
        const double sx = x == 0.0 ? 1.0 : sin(x) / x;
        double b2 = 1.0;
        for (int k = 0; k < order; ++k) b2 *= sx;
        b2 *= b2;
        if (full) {
            gf[j] = static_cast<T>(direct ? s / b2 : 1.0 / b2);
            hf[j] = s / b2;
        } else {
            gh[j] = static_cast<T>(direct ? s / b2 : 1.0 / b2);
            hh[j] = s / b2;
        }
    }
}

size_t static_align(size_t v) { return (v + 255) / 256 * 256; }

struct StaticLayout {
    size_t bintab, gf, gh, hf, hh, partials, sums, total;
};

StaticLayout static_layout(int ng, int nbins, int nsq_max, size_t elem)
{
    StaticLayout L{};
    const int nh = ng / 2 + 1;
    size_t off = 0;
    L.bintab = off;
    off = static_align(off + size_t(nsq_max + 1) * sizeof(uint16_t));
    L.gf = off;
    off = static_align(off + size_t(ng) * elem);
    L.gh = off;
    off = static_align(off + size_t(nh) * elem);
    L.hf = off;
    off = static_align(off + size_t(ng) * sizeof(double));
    L.hh = off;
    off = static_align(off + size_t(nh) * sizeof(double));
    L.partials = off;
    off = static_align(off + size_t(kStaticBlocks) * kModeVals * nbins * sizeof(double));
    L.sums = off;
    off = static_align(off + size_t(kModeVals + kBinVals) * nbins * sizeof(double));
    L.total = off;
    return L;
}

// Device address of g_static_scratch, looked up once per device (under a lock, so that
// host threads making their first calls at the same time do not race on the cache).
constexpr int kMaxDevices = 64;
unsigned char *g_static_ptr[kMaxDevices] = {};
std::mutex g_static_ptr_lock;

cudaError_t static_scratch_ptr(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_static_ptr_lock);
    if (!g_static_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_ptr[dev] = static_cast<unsigned char *>(ptr);
    }
    *out = g_static_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace pkmom

extern "C" pkmom_status pkmom_spectra_static(const pkmom_params *p, const void *grids, const void *moments_dev,
                                             double *out_dev, void *stream)
{
    using namespace pkmom;
    if (!p || !grids || !moments_dev || !out_dev) return PKMOM_EINVAL;
    if (!(p->box_L > 0) || !std::isfinite(p->box_L) || !std::isfinite(p->theta_scale) || p->ng < 16 ||
        p->ng > 1024 || p->ng % 8 || p->order < 1 || p->order > 5 ||
        (p->precision != PKMOM_F32 && p->precision != PKMOM_F64) || p->nbins < 1 || p->theta_sn_mode < 0 ||
        p->theta_sn_mode > 1 || (p->bl_radius != 0 && (p->bl_radius < 2 || p->bl_radius > 4 || p->order != 4)))
        return PKMOM_EINVAL;
    if (p->nbins > kStaticMaxBins) return PKMOM_EUNSUPPORTED;  // beyond the static scratch's shell limit
    const double umin = p->kmin_kf > 0 ? p->kmin_kf : 1.0;
    const double umax = p->kmax_kf > 0 ? p->kmax_kf : 0.5 * p->ng;
    if (!(umax <= 0.5 * p->ng) || !(umin < umax)) return PKMOM_EINVAL;
    const int ng = p->ng, nh = ng / 2 + 1, nbins = p->nbins;
    const int nsq_max = static_cast<int>(std::floor(umax * umax)) + 1;
    const size_t elem = p->precision == PKMOM_F32 ? sizeof(float) : sizeof(double);
    const StaticLayout L = static_layout(ng, nbins, nsq_max, elem);
    if (L.total > kStaticScratchBytes) return PKMOM_EUNSUPPORTED;  // does not fit the static scratch
    unsigned char *base = nullptr;
    if (static_scratch_ptr(&base) != cudaSuccess) return PKMOM_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    SpectraTables t;
    t.ng = ng;
    t.order = p->order;
    t.direct = p->bl_radius != 0;
    t.nbins = nbins;
    t.prec = p->precision;
    t.umin = umin;
    t.umax = umax;
    t.nsq_max = nsq_max;
    t.bintab = reinterpret_cast<uint16_t *>(base + L.bintab);
    t.g_full = base + L.gf;
    t.g_half = base + L.gh;
    t.h_full = reinterpret_cast<double *>(base + L.hf);
    t.h_half = reinterpret_cast<double *>(base + L.hh);
    t.partials = reinterpret_cast<double *>(base + L.partials);
    t.mode_sums = reinterpret_cast<double *>(base + L.sums);
    t.bin_blocks = kStaticBlocks;

    const int tb = 256, tg = (nsq_max + 1 + tb - 1) / tb < 256 ? (nsq_max + 1 + tb - 1) / tb : 256;
    if (p->precision == PKMOM_F32)
        k_static_tables<float><<<tg, tb, 0, s>>>(ng, p->order, p->bl_radius != 0, nbins, umin, umax, nsq_max, t.bintab,
                                                 static_cast<float *>(t.g_full), static_cast<float *>(t.g_half),
                                                 t.h_full, t.h_half);
    else
        k_static_tables<double><<<tg, tb, 0, s>>>(ng, p->order, p->bl_radius != 0, nbins, umin, umax, nsq_max, t.bintab,
                                                  static_cast<double *>(t.g_full), static_cast<double *>(t.g_half),
                                                  t.h_full, t.h_half);
    const uint32_t nmodes = static_cast<uint32_t>(static_cast<int64_t>(ng) * ng * nh);
    const size_t msmem = static_cast<size_t>(kModeVals) * nbins * sizeof(double);
    if (cudaFuncSetAttribute(k_mode_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(msmem)) !=
        cudaSuccess)
        return PKMOM_ECUDA;
    // every partial slot is written by its block, so nothing here needs clearing
    k_mode_sums<<<kStaticBlocks, kBinThreads, msmem, s>>>(ng, nmodes, t.bintab, t.nsq_max, t.h_full, t.h_half, nbins,
                                                          t.partials);
    k_reduce_partials<kModeVals><<<nbins, 256, 0, s>>>(t.partials, kStaticBlocks, nbins, t.mode_sums);
    LaunchStats st;
    if (cudaGetLastError() != cudaSuccess) return PKMOM_ECUDA;
    if (launch_bin(t, grids, static_cast<const double *>(moments_dev), s, st) != cudaSuccess) return PKMOM_ECUDA;
    if (launch_finalize(t, *p, static_cast<const double *>(moments_dev), out_dev, s, st, false) != cudaSuccess)
        return PKMOM_ECUDA;
    return PKMOM_OK;
}

// ---------------------------------------------------------------- spectra in (|k|, mu) bins
// Shells of |k| split into nmu linear bins of mu = n.e / |n| in [-1, 1] (e: a given
// direction, or the bulk flow), for the direction-dependent parts of Sec. 2.2 (Eq.
// thetanoise) and Sec. 3.2 (Eq. bfpdpx): the imaginary density x momentum-divergence
// cross spectrum -i k mu_b (v_b/Haf) P and the mu_b-dependent shot noise, which shell
// averages cancel. A stored half-spectrum mode n with 0 < n_z < ng/2 stands for n and -n:
// it is added at mu(n) and, mirrored (odd terms negated), at mu(-n) = -mu(n). Modes with
// a Nyquist component have no direction sign and are left out. The mu bin is decided in
// FP32 with correctly rounded operations in a fixed order:
// m = floor(((n0 e0 + n1 e1) + n2 e2) / sqrt(|n|^2) + 1) * nmu/2), clipped.
namespace pkmom {
namespace {

// Per-item sums (each times the mode weight; data values also times g = 1/W^2):
//  0 |F_d|^2  1 |F_p|^2  2 |F_p'|^2  3 |n.F_p|^2  4 |n.F_p'|^2
//  5 Im z  6 Re z  (z = conj(F_d) n.F_p)   7 Im z'  8 Re z'  (F_p')   9 Re conj(F_d) e_b.F_p'
//  10 count  11 |n|  12 mu  13 h  14-19 h n_a n_b (xx yy zz xy xz yz)  20-22 h n_a
constexpr int kMuVals = 23;
__device__ __forceinline__ bool mu_odd(int k) { return k == 6 || k == 8 || k == 12 || k >= 20; }

__device__ __forceinline__ int mu_bin(float n0, float n1, float n2, float e0, float e1, float e2, float r, int nmu)
{
    const float d = __fadd_rn(__fadd_rn(__fmul_rn(n0, e0), __fmul_rn(n1, e1)), __fmul_rn(n2, e2));
    const float mu = __fdiv_rn(d, r);
    const int m = static_cast<int>(floorf(__fmul_rn(__fadd_rn(mu, 1.0f), 0.5f * static_cast<float>(nmu))));
    return m < 0 ? 0 : (m >= nmu ? nmu - 1 : m);
}

template <typename T>
__global__ void __launch_bounds__(kBinThreads, 2)
k_bin_mu(const Cx<T> *__restrict__ F, int64_t gstride, int ng, int nbins, int nmu, const int *__restrict__ thresh,
         const T *__restrict__ gf, const T *__restrict__ gh, const double *__restrict__ hf,
         const double *__restrict__ hh, const double *__restrict__ mom, double ge0, double ge1, double ge2,
         int bulk_dir, const uint32_t *__restrict__ order, int nwork, unsigned *__restrict__ counter,
         double *__restrict__ partials)
{
    constexpr int NW = kBinThreads / 32;
    __shared__ int s_lo[NW][32], s_pre[NW][32], s_n1[NW][32];
    __shared__ int64_t s_row[NW][32];
    __shared__ T s_g[NW][32];
    __shared__ T s_h[NW][32];
    const int nh = ng / 2 + 1;
    const double Mtot = mom[0];
    const double vbd[3] = {mom[2] / Mtot, mom[3] / Mtot, mom[4] / Mtot};
    const double vbn = sqrt(vbd[0] * vbd[0] + vbd[1] * vbd[1] + vbd[2] * vbd[2]);
    const T vb0 = static_cast<T>(vbd[0]), vb1 = static_cast<T>(vbd[1]), vb2 = static_cast<T>(vbd[2]);
    const T eb0 = vbn > 0 ? static_cast<T>(vbd[0] / vbn) : T(0), eb1 = vbn > 0 ? static_cast<T>(vbd[1] / vbn) : T(0),
            eb2 = vbn > 0 ? static_cast<T>(vbd[2] / vbn) : T(0);
    double ed0 = ge0, ed1 = ge1, ed2 = ge2;  // unit direction in FP64
    if (bulk_dir) {
        ed0 = vbn > 0 ? vbd[0] / vbn : 0.0;
        ed1 = vbn > 0 ? vbd[1] / vbn : 0.0;
        ed2 = vbn > 0 ? vbd[2] / vbn : 0.0;
    }
    // the bin decision in FP32; the mean mu in the grid precision
    const float e0 = static_cast<float>(ed0), e1 = static_cast<float>(ed1), e2 = static_cast<float>(ed2);
    const T et0 = static_cast<T>(ed0), et1 = static_cast<T>(ed1), et2 = static_cast<T>(ed2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // items (slab, shell, mu bin) of the (slab, shell) pairs that hold modes, drawn from a
    // device counter; the last block sets it back to zero
    const unsigned nitems = static_cast<unsigned>(nwork) * static_cast<unsigned>(nmu);
    for (;;) {
        unsigned jw = 0;
        if (lane == 0) jw = atomicAdd(counter, 1u);
        jw = __shfl_sync(0xffffffffu, jw, 0);
        if (jw >= nitems) break;
        const int item = static_cast<int>(order[jw / nmu]) * nmu + static_cast<int>(jw % nmu);
        const int m = item % nmu;
        const int b = (item / nmu) % nbins;
        const int i0 = item / (nmu * nbins);
        const int n0 = i0 < ng / 2 ? i0 : i0 - ng;
        const int lo2 = thresh[b], hi2 = thresh[b + 1];  // lo2 <= |n|^2 < hi2
        T s[kMuVals], c[kMuVals];
#pragma unroll
        for (int k = 0; k < kMuVals; ++k) s[k] = T(0), c[k] = T(0);
        const int rem = hi2 - 1 - n0 * n0;
        if (i0 == ng / 2 || hi2 <= lo2 || rem < 0) {  // no mode: zero sums, no reduction
            if (lane < kMuVals) partials[static_cast<int64_t>(item) * kMuVals + lane] = 0.0;
            continue;
        }
        {
            const int R1 = isqrt_floor(rem);
            const int n1lo = max(1 - ng / 2, -R1), n1hi = min(ng / 2 - 1, R1);
            const T g0 = gf[i0];
            const double h0 = hf[i0];
            for (int r0 = n1lo; r0 <= n1hi; r0 += 32) {
                const int n1 = r0 + lane;
                const bool row = n1 <= n1hi;
                int l_lo = 0, len = 0;
                if (row) {
                    const int r2 = n0 * n0 + n1 * n1;
                    const int top = hi2 - 1 - r2;
                    if (top >= 0) {
                        const int lh = min(isqrt_floor(top), nh - 2);  // no Nyquist plane
                        const int need = lo2 - r2;
                        const int ll = need <= 0 ? 0 : isqrt_floor(need - 1) + 1;
                        if (lh >= ll) l_lo = ll, len = lh - ll + 1;
                    }
                }
                int inc = len;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, inc, d);
                    if (lane >= d) inc += t;
                }
                const int total = __shfl_sync(0xffffffffu, inc, 31);
                if (total == 0) continue;
                const int i1 = row ? (n1 < 0 ? n1 + ng : n1) : 0;
                s_lo[w][lane] = l_lo;
                s_pre[w][lane] = inc - len;
                s_n1[w][lane] = n1;
                s_row[w][lane] = (static_cast<int64_t>(i0) * ng + i1) * nh;
                s_g[w][lane] = row ? g0 * gf[i1] : T(0);
                s_h[w][lane] = row ? static_cast<T>(h0 * hf[i1]) : T(0);
                __syncwarp();
                for (int mm = lane; mm < total; mm += 32) {
                    int j = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1)
                        if (s_pre[w][j + step] <= mm) j += step;
                    const int l = s_lo[w][j] + (mm - s_pre[w][j]);
                    const int nn1 = s_n1[w][j];
                    const int nsq = n0 * n0 + nn1 * nn1 + l * l;
                    const float rn = __fsqrt_rn(static_cast<float>(nsq));
                    const float fn0 = static_cast<float>(n0), fn1 = static_cast<float>(nn1), fl = static_cast<float>(l);
                    const bool fwd = mu_bin(fn0, fn1, fl, e0, e1, e2, rn, nmu) == m;
                    const bool mir = l > 0 && mu_bin(-fn0, -fn1, -fl, e0, e1, e2, rn, nmu) == m;
                    if (!fwd && !mir) continue;
                    const int64_t mi = s_row[w][j] + l;
                    if (!PK_IN(mi, gstride, kChkMode) || !PK_IN(l, nh, kChkMode)) continue;
                    const T g = s_g[w][j] * gh[l];
                    const T th = s_h[w][j] * static_cast<T>(hh[l]);
                    const Cx<T> dd = F[mi], p0 = F[gstride + mi], p1 = F[2 * gstride + mi], p2 = F[3 * gstride + mi];
                    const T a0 = static_cast<T>(n0), a1 = static_cast<T>(nn1), a2 = static_cast<T>(l);
                    const T kr = a0 * p0.x + a1 * p1.x + a2 * p2.x, ki = a0 * p0.y + a1 * p1.y + a2 * p2.y;
                    const Cx<T> q0{p0.x - vb0 * dd.x, p0.y - vb0 * dd.y};
                    const Cx<T> q1{p1.x - vb1 * dd.x, p1.y - vb1 * dd.y};
                    const Cx<T> q2{p2.x - vb2 * dd.x, p2.y - vb2 * dd.y};
                    const T jr = a0 * q0.x + a1 * q1.x + a2 * q2.x, ji = a0 * q0.y + a1 * q1.y + a2 * q2.y;
                    const T br = eb0 * q0.x + eb1 * q1.x + eb2 * q2.x, bi = eb0 * q0.y + eb1 * q1.y + eb2 * q2.y;
                    T v[kMuVals];
                    v[0] = g * (dd.x * dd.x + dd.y * dd.y);
                    v[1] = g * (p0.x * p0.x + p0.y * p0.y + p1.x * p1.x + p1.y * p1.y + p2.x * p2.x + p2.y * p2.y);
                    v[2] = g * (q0.x * q0.x + q0.y * q0.y + q1.x * q1.x + q1.y * q1.y + q2.x * q2.x + q2.y * q2.y);
                    v[3] = g * (kr * kr + ki * ki);
                    v[4] = g * (jr * jr + ji * ji);
                    v[5] = g * (dd.x * ki - dd.y * kr);  // Im(conj(F_d) n.F_p)
                    v[6] = g * (dd.x * kr + dd.y * ki);  // Re(conj(F_d) n.F_p)
                    v[7] = g * (dd.x * ji - dd.y * jr);
                    v[8] = g * (dd.x * jr + dd.y * ji);
                    v[9] = g * (dd.x * br + dd.y * bi);
                    const T rt = sqrt(static_cast<T>(nsq));
                    v[10] = T(1);
                    v[11] = rt;
                    v[12] = (a0 * et0 + a1 * et1 + a2 * et2) / rt;
                    v[13] = th;
                    v[14] = th * a0 * a0;
                    v[15] = th * a1 * a1;
                    v[16] = th * a2 * a2;
                    v[17] = th * a0 * a1;
                    v[18] = th * a0 * a2;
                    v[19] = th * a1 * a2;
                    v[20] = th * a0;
                    v[21] = th * a1;
                    v[22] = th * a2;
#pragma unroll
                    for (int k = 0; k < kMuVals; ++k) {
                        // forward and mirrored contributions (the mirror negates odd terms)
                        const T x = (fwd ? v[k] : T(0)) + (mir ? (mu_odd(k) ? -v[k] : v[k]) : T(0));
                        const T y = x - c[k];
                        const T t = s[k] + y;
                        c[k] = (t - s[k]) - y;
                        s[k] = t;
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int g = 0; g < (kMuVals + 7) / 8; ++g) {  // reduce-scatter, 8 sums at a time
            T hi[8], lo[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int v = 8 * g + k;
                hi[k] = v < kMuVals ? s[v] : T(0);
                lo[k] = v < kMuVals ? -c[v] : T(0);
            }
            const double dsum = warp_scatter_sum8(hi, lo);
            const int v = 8 * g + ((lane >> 2) & 7);
            if ((lane & 3) == 0 && v < kMuVals) partials[static_cast<int64_t>(item) * kMuVals + v] = dsum;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(counter + 1, 1u) == gridDim.x - 1) counter[0] = 0u, counter[1] = 0u;
}

struct MuParams {
    double V, kf, ts;
    int ncells;
};

// One thread per (shell, mu) cell: the sums of k_bin_mu -> spectra with the shot noise
// subtracted in FP64 (the same algebra as k_finalize, with the odd terms kept).
__global__ void k_finalize_mu(const double *__restrict__ sums /*[kMuVals][ncells]*/, const double *__restrict__ mom,
                              MuParams fp, double *__restrict__ out /*[PKMOM_MU_NROWS][ncells]*/)
{
    const int cidx = blockIdx.x * blockDim.x + threadIdx.x;
    const int nc = fp.ncells;
    if (cidx >= nc) return;
    auto S = [&](int k) { return sums[k * nc + cidx]; };
    auto put = [&](int row, double v) { out[row * nc + cidx] = v; };
    const double n = S(10);
    put(PKMOM_MU_ROW_NMODES, n);
    if (!(n > 0.0)) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        for (int r = 0; r < PKMOM_MU_NROWS; ++r)
            if (r != PKMOM_MU_ROW_NMODES) put(r, nan);
        return;
    }
    const double M = mom[0], S2 = mom[1];
    const double vb[3] = {mom[2] / M, mom[3] / M, mom[4] / M};
    const double R[3] = {mom[5], mom[6], mom[7]};
    const double *Q = mom + 8;
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
    double Qb[6], Rb[3];
    for (int k = 0; k < 6; ++k)
        Qb[k] = Q[k] - vb[ia[k]] * R[ib[k]] - R[ia[k]] * vb[ib[k]] + vb[ia[k]] * vb[ib[k]] * S2;
    for (int a = 0; a < 3; ++a) Rb[a] = R[a] - S2 * vb[a];
    const double vbn = sqrt(vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]);
    const double ebR = vbn > 0 ? (vb[0] * Rb[0] + vb[1] * Rb[1] + vb[2] * Rb[2]) / vbn : 0.0;
    const double H = S(13);
    double H2[6];
    for (int k = 0; k < 6; ++k) H2[k] = S(14 + k);
    const double H1[3] = {S(20), S(21), S(22)};
    const double c = fp.V / (M * M * n);
    const double ct = c * fp.ts * fp.ts * fp.kf * fp.kf, cx = c * fp.ts * fp.kf;
    put(PKMOM_MU_ROW_K, fp.kf * S(11) / n);
    put(PKMOM_MU_ROW_MU, S(12) / n);
    const double sn_dd = c * S2 * H;
    put(PKMOM_MU_ROW_PDD, c * S(0) - sn_dd);
    put(PKMOM_MU_ROW_SNDD, sn_dd);
    put(PKMOM_MU_ROW_PPP, c * (S(1) - (Q[0] + Q[1] + Q[2]) * H));
    put(PKMOM_MU_ROW_PPP_B, c * (S(2) - (Qb[0] + Qb[1] + Qb[2]) * H));
    const double sn_tt = ct * qdot(Q, H2);
    put(PKMOM_MU_ROW_PTT, ct * S(3) - sn_tt);
    put(PKMOM_MU_ROW_SNTT, sn_tt);
    put(PKMOM_MU_ROW_PTT_B, ct * S(4) - ct * qdot(Qb, H2));
    // X = -i ts conj(F_d) k.F_p: Re X = ts Im z, Im X = -ts Re z; its shot noise
    // -i ts (k.R) h is imaginary (Eq. rawPx)
    const double im_sn = -cx * (R[0] * H1[0] + R[1] * H1[1] + R[2] * H1[2]);
    const double im_sn_b = -cx * (Rb[0] * H1[0] + Rb[1] * H1[1] + Rb[2] * H1[2]);
    put(PKMOM_MU_ROW_RE_DT, cx * S(5));
    put(PKMOM_MU_ROW_IM_DT, -cx * S(6) - im_sn);
    put(PKMOM_MU_ROW_IM_SNDT, im_sn);
    put(PKMOM_MU_ROW_RE_DT_B, cx * S(7));
    put(PKMOM_MU_ROW_IM_DT_B, -cx * S(8) - im_sn_b);
    put(PKMOM_MU_ROW_RE_DPB_B, c * (S(9) - ebR * H));
}

}  // namespace

cudaError_t launch_spectra_mu(const SpectraTables &t, const pkmom_params &p, const void *grids,
                              const double *moments_dev, const double *dir /* unit, or nullptr */, int nmu,
                              double *partials, double *sums, double *out, cudaStream_t s, LaunchStats &st)
{
    const int ng = t.ng, nh = ng / 2 + 1;
    const int64_t gstride = static_cast<int64_t>(ng) * ng * nh;
    const unsigned blocks = static_cast<unsigned>(t.shell_blocks) / 2u;  // resident: 2 blocks per SM
    const double d0 = dir ? dir[0] : 0.0, d1 = dir ? dir[1] : 0.0, d2 = dir ? dir[2] : 0.0;
    const int bulk_dir = dir ? 0 : 1;
    if (t.prec == PKMOM_F32)
        k_bin_mu<float><<<blocks, kBinThreads, 0, s>>>(
            static_cast<const Cx<float> *>(grids), gstride, ng, t.nbins, nmu, t.thresh,
            static_cast<const float *>(t.g_full), static_cast<const float *>(t.g_half), t.h_full, t.h_half,
            moments_dev, d0, d1, d2, bulk_dir, t.bin_order, t.bin_nwork, t.bin_counter + 2, partials);
    else
        k_bin_mu<double><<<blocks, kBinThreads, 0, s>>>(
            static_cast<const Cx<double> *>(grids), gstride, ng, t.nbins, nmu, t.thresh,
            static_cast<const double *>(t.g_full), static_cast<const double *>(t.g_half), t.h_full, t.h_half,
            moments_dev, d0, d1, d2, bulk_dir, t.bin_order, t.bin_nwork, t.bin_counter + 2, partials);
    const int ncells = t.nbins * nmu;
    k_reduce_items<kMuVals><<<ncells, 256, 0, s>>>(partials, ng, ncells, sums, t.thresh, nmu);
    MuParams fp;
    fp.V = p.box_L * p.box_L * p.box_L;
    fp.kf = kTwoPi / p.box_L;
    fp.ts = p.theta_scale;
    fp.ncells = ncells;
    k_finalize_mu<<<(ncells + 127) / 128, 128, 0, s>>>(sums, moments_dev, fp, out);
    st.launches += 3;
    return cudaGetLastError();
}

size_t spectra_mu_partial_bytes(int ng, int nbins, int nmu)
{
    return static_cast<size_t>(ng) * nbins * nmu * kMuVals * sizeof(double);
}
size_t spectra_mu_sum_bytes(int nbins, int nmu) { return static_cast<size_t>(nbins) * nmu * kMuVals * sizeof(double); }

}  // namespace pkmom
