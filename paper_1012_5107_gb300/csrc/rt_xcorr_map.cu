// rt_xcorr_map.cu -- the cross-correlation function C(di, dj) of Eq. 15 over
// pixel shifts, its peak and its mean over several reference pairs (Sec. 5).
//
// Pass 1 forms, over the field-of-view window of columns j0..j1-1, the means
// of Eq. 14 and the denominator sum (f - <f>)^2 of Eq. 15 in FP64: blocks of
// 4 image rows per pair sum them (FP64 is slow on this GPU, so the work is
// spread over many SMs), then a block per pair and channel adds the chunks.
// Pass 2 is a direct correlation in tiles: a block owns 16 R x 16 R shifts
// (di, dj) and a chunk of 8 image rows x 128 columns of one pair and
// channel; it stages the chunk of f and the window of g its shifts need (zero
// outside the field-of-view window, where the finite photographs have no
// values) in shared memory, and each thread accumulates the products of its
// R x R shifts over the chunk with FP32 FMA (see xmap_tiles).
// Pass 3 adds, per shift, pair, channel and column chunk, the row chunks'
// sums with compensated (Kahan) FP32 summation, whose error is of the order
// of one FP32 rounding of the result, below the rounding already in each
// chunk's sum (FP64 adds are 64 times slower on this GPU).  Pass 4 adds the
// column chunks in FP64, divides by the denominators, stacks the channels
// (sum of numerators over sum of denominators) and averages the maps of the
// pairs; pass 5 finds the peak of the stacked mean map and its shift.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rt_internal.h"

namespace grt {

constexpr int kMapT = 16;         // threads along di and along dj
constexpr int kMapRows = 8;       // image rows per chunk
constexpr int kMapCols = 128;     // image columns per chunk
constexpr int kMapBlock = kMapT * kMapT;
constexpr int kMapMaxShift = 64;

// Staged g window of a block with R x R shifts per thread: rows x padded
// columns (one column past the window is read, never used, by the sliding
// loads of the last column).
template <int R> struct MapTile {
    static constexpr int TD = kMapT * R;                  // shifts per block along di and dj
    static constexpr int GR = kMapRows + TD - 1;
    static constexpr int GC = kMapCols + TD;
    static constexpr size_t smem = sizeof(float) * ((size_t)GR * GC + (size_t)kMapRows * kMapCols);
};
constexpr int kMapMaxPairs = 64;

struct MapImages {
    const float* f[kMapMaxPairs];
    const float* g[kMapMaxPairs];
};

constexpr int kMomRows = 4;       // image rows per block of pass 1
constexpr int kMomBlock = 256;

// A window row's values, (i W + j0) C ... (i W + j1) C, are contiguous, and
// the stride T is a multiple of C, so thread t meets only channel t mod C;
// the block's per-channel sums go to part[((pair nchunks + chunk) C + c) 3 + q]
// (q: sum f, sum g, sum f^2).
__global__ void __launch_bounds__(kMomBlock) xmap_moment_rows(MapImages im, int H, int W, int C, int j0, int j1,
                                                              int nchunks, double* __restrict__ part)
{
    __shared__ double red[3][kMomBlock];
    const int chunk = blockIdx.x, pair = blockIdx.y;
    const float* f = im.f[pair];
    const float* g = im.g[pair];
    const int T = (kMomBlock / C) * C;
    const int len = (j1 - j0) * C;
    const int t = threadIdx.x;
    const int i0 = chunk * kMomRows, i1 = min(H, i0 + kMomRows);
    double sf = 0.0, sg = 0.0, sff = 0.0;
    if (t < T) {
        for (int i = i0; i < i1; ++i) {
            const int64_t base = ((int64_t)i * W + j0) * C;
#pragma unroll 4
            for (int e = t; e < len; e += T) {
                const double a = __ldg(f + base + e), b = __ldg(g + base + e);
                sf += a;
                sg += b;
                sff += a * a;
            }
        }
    }
    red[0][t] = sf;
    red[1][t] = sg;
    red[2][t] = sff;
    __syncthreads();
    if (t < 3 * C) {
        const int q = t / C, c = t - q * C;
        double acc = 0.0;
        for (int k = c; k < T; k += C) acc += red[q][k];
        part[(((int64_t)pair * nchunks + chunk) * C + c) * 3 + q] = acc;
    }
}

// Block per (pair, channel): the chunks' sums, then the statistics.
__global__ void __launch_bounds__(128) xmap_moment_stats(const double* __restrict__ part, int H, int C, int j0,
                                                         int j1, int nchunks, double* __restrict__ stats)
{
    const int pc = blockIdx.x, pair = pc / C, c = pc % C;
    double v[3] = {0.0, 0.0, 0.0};
    for (int k = threadIdx.x; k < nchunks; k += blockDim.x) {
        const double* p = part + (((int64_t)pair * nchunks + k) * C + c) * 3;
        v[0] += p[0];
        v[1] += p[1];
        v[2] += p[2];
    }
    __shared__ double red[3][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < 3; ++q) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[q][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[3];
        for (int q = 0; q < 3; ++q) t[q] = red[q][0] + red[q][1] + red[q][2] + red[q][3];
        const double N = (double)H * (double)(j1 - j0);
        const double mf = t[0] / N, mg = t[1] / N;          // Eq. 14
        stats[3 * pc + 0] = mf;
        stats[3 * pc + 1] = mg;
        stats[3 * pc + 2] = t[2] - t[0] * mf;               // sum (f - <f>)^2, Eq. 15 denominator
    }
}

// Thread (ty, tx) owns the shifts di = di_lo + ty R + a, dj = dj_lo + tx R + b
// (a, b < R).  The product f(i, j) g(i + di, j + dj) of chunk row r and column
// q reads g_s[r + ty R + a][q + tx R + b]; along q each of the R g rows a
// thread reads slides by one column, so a column costs one broadcast f load
// and R g loads for R^2 FMAs.  The chunk's sum per shift is FP32 (8 x 128
// products); part[((pc nchunks + chunk) nshift + s)], chunk = rc ncc + cc.
template <int R>
__global__ void __launch_bounds__(kMapBlock) xmap_tiles(MapImages im, const double* __restrict__ stats, int H, int W,
                                                        int C, int j0, int j1, int max_di, int max_dj, int ncc,
                                                        int nchunks, float* __restrict__ part)
{
    using Tl = MapTile<R>;
    extern __shared__ float map_smem[];
    float* g_s = map_smem;                                   // [GR][GC]
    float* f_s = map_smem + (size_t)Tl::GR * Tl::GC;         // [kMapRows][kMapCols]
    const int ndi = 2 * max_di + 1, ndj = 2 * max_dj + 1;
    const int tiles_dj = (ndj + Tl::TD - 1) / Tl::TD;
    const int tdi = blockIdx.x / tiles_dj, tdj = blockIdx.x % tiles_dj;
    const int chunk = blockIdx.y;
    const int rc = chunk / ncc, cc = chunk % ncc;
    const int pc = blockIdx.z;
    const int pair = pc / C, c = pc % C;
    const float* f = im.f[pair];
    const float* g = im.g[pair];
    const float mf = (float)stats[3 * pc + 0], mg = (float)stats[3 * pc + 1];
    const int di_lo = -max_di + tdi * Tl::TD, dj_lo = -max_dj + tdj * Tl::TD;
    const int i0 = rc * kMapRows, jc = j0 + cc * kMapCols;
    for (int k = threadIdx.x; k < kMapRows * kMapCols; k += kMapBlock) {
        const int r = k / kMapCols, q = k % kMapCols;
        const int i = i0 + r, j = jc + q;
        f_s[k] = (i < H && j < j1) ? __ldg(f + ((int64_t)i * W + j) * C + c) - mf : 0.0f;
    }
    for (int k = threadIdx.x; k < Tl::GR * Tl::GC; k += kMapBlock) {
        const int r = k / Tl::GC, q = k % Tl::GC;
        const int i = i0 + di_lo + r, j = jc + dj_lo + q;
        g_s[k] = (i >= 0 && i < H && j >= j0 && j < j1) ? __ldg(g + ((int64_t)i * W + j) * C + c) - mg : 0.0f;
    }
    __syncthreads();
    const int ty = threadIdx.x / kMapT, tx = threadIdx.x % kMapT;
    float acc[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) acc[a][b] = 0.0f;
    for (int r = 0; r < kMapRows; ++r) {
        const float* fr = f_s + r * kMapCols;
        const float* gr = g_s + (size_t)(r + ty * R) * Tl::GC + tx * R;
        float win[R][R];
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) win[a][b] = gr[a * Tl::GC + b];
#pragma unroll 16
        for (int q = 0; q < kMapCols; ++q) {
            const float fv = fr[q];
#pragma unroll
            for (int a = 0; a < R; ++a) {
#pragma unroll
                for (int b = 0; b < R; ++b) acc[a][b] = fmaf(fv, win[a][b], acc[a][b]);
#pragma unroll
                for (int b = 0; b + 1 < R; ++b) win[a][b] = win[a][b + 1];
                win[a][R - 1] = gr[a * Tl::GC + q + R];
            }
        }
    }
    const int64_t nshift = (int64_t)ndi * ndj;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const int di = di_lo + ty * R + a;
#pragma unroll
        for (int b = 0; b < R; ++b) {
            const int dj = dj_lo + tx * R + b;
            if (di <= max_di && dj <= max_dj) {
                const int64_t sh = (int64_t)(di + max_di) * ndj + (dj + max_dj);
                part[((int64_t)pc * nchunks + chunk) * nshift + sh] = acc[a][b];
            }
        }
    }
}

// Thread per (pair and channel pc, column chunk cc, shift s): the row chunks'
// sums, compensated; colsum[(pc ncc + cc) nshift + s] = sum - compensation.
__global__ void __launch_bounds__(256) xmap_sum(const float* __restrict__ part, int nrc, int ncc, int64_t n,
                                                int nshift, double* __restrict__ colsum)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int s = (int)(t % nshift);
    const int64_t pq = t / nshift;
    const int64_t pc = pq / ncc, cc = pq % ncc;
    const float* p = part + ((pc * nrc * ncc) + cc) * nshift + s;
    const int64_t stride = (int64_t)ncc * nshift;
    float sum = 0.0f, comp = 0.0f;
#pragma unroll 8
    for (int k = 0; k < nrc; ++k) {
        const float y = p[k * stride] - comp;
        const float u = sum + y;
        comp = (u - sum) - y;
        sum = u;
    }
    colsum[t] = (double)sum - (double)comp;
}

__global__ void __launch_bounds__(256) xmap_finish(const double* __restrict__ colsum,
                                                   const double* __restrict__ stats, int n_pairs, int C, int ncc,
                                                   int nshift, double* __restrict__ out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nshift) return;
    double mean[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int p = 0; p < n_pairs; ++p) {
        double num_all = 0.0, den_all = 0.0;
        for (int c = 0; c < C; ++c) {
            const int pc = p * C + c;
            double num = 0.0;
            for (int q = 0; q < ncc; ++q) num += colsum[((int64_t)pc * ncc + q) * nshift + s];
            const double den = stats[3 * pc + 2];
            mean[c] += num / den;
            num_all += num;
            den_all += den;
        }
        mean[C] += num_all / den_all;
    }
    for (int c = 0; c <= C; ++c) out[(int64_t)s * (C + 1) + c] = mean[c] / (double)n_pairs;
}

// Peak of the stacked-channel map: largest value, the first in row-major
// order (di, then dj ascending) among equal ones.
__global__ void __launch_bounds__(1024) xmap_peak(const double* __restrict__ map, int C, int max_di, int max_dj,
                                                  double* __restrict__ peak)
{
    const int ndj = 2 * max_dj + 1, nshift = (2 * max_di + 1) * ndj;
    double best = -INFINITY;
    int bi = nshift;
    for (int s = threadIdx.x; s < nshift; s += blockDim.x) {
        const double v = map[(int64_t)s * (C + 1) + C];
        if (v > best || (v == best && s < bi)) { best = v; bi = s; }
    }
    __shared__ double sv[32];
    __shared__ int si[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sv[warp] = best; si[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (sv[w] > best || (sv[w] == best && si[w] < bi)) { best = sv[w]; bi = si[w]; }
        peak[0] = best;
        peak[1] = (double)(bi / ndj - max_di);
        peak[2] = (double)(bi % ndj - max_dj);
    }
}

template <int R>
static cudaError_t launch_tiles(dim3 grid, cudaStream_t st, const MapImages& im, const double* stats, int H, int W,
                               int C, int j0, int j1, int max_di, int max_dj, int ncc, int nchunks, float* part)
{
    const size_t smem = MapTile<R>::smem;
    cudaError_t e = cudaFuncSetAttribute(xmap_tiles<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    xmap_tiles<R><<<grid, kMapBlock, smem, st>>>(im, stats, H, W, C, j0, j1, max_di, max_dj, ncc, nchunks, part);
    return cudaGetLastError();
}

}  // namespace grt

using namespace grt;

extern "C" int rt_xcorr_map(const float* const* d_f, const float* const* d_g, int32_t n_pairs, int32_t height,
                            int32_t width, int32_t channels, double fov_deg, double hfov_deg, int32_t max_di,
                            int32_t max_dj, double* d_map, double* d_peak, void* stream)
{
    if (!d_f || !d_g || !d_map) { set_error("null pointer argument"); return RT_EINVAL; }
    if (n_pairs < 1 || n_pairs > kMapMaxPairs) { set_error("n_pairs must be 1..%d", kMapMaxPairs); return RT_EINVAL; }
    for (int p = 0; p < n_pairs; ++p)
        if (!d_f[p] || !d_g[p]) { set_error("image pointer of pair %d is NULL", p); return RT_EINVAL; }
    if (height < 1 || width < 1) { set_error("height and width must be >= 1"); return RT_EINVAL; }
    if (channels < 1 || channels > 4) { set_error("channels must be 1..4"); return RT_EINVAL; }
    if (max_di < 0 || max_di > kMapMaxShift || max_dj < 0 || max_dj > kMapMaxShift) {
        set_error("max_di and max_dj must be 0..%d", kMapMaxShift);
        return RT_EINVAL;
    }
    if (!(hfov_deg > 0.0 && hfov_deg < 180.0)) { set_error("hfov_deg must be in (0, 180)"); return RT_EINVAL; }
    if (!(fov_deg >= 0.0)) { set_error("fov_deg must be >= 0"); return RT_EINVAL; }
    Windows win;
    fov_windows(width, hfov_deg, &fov_deg, 1, &win);
    const int j0 = win.j0[0], j1 = win.j1[0];
    if (j1 <= j0) { set_error("the field of view holds no pixel column"); return RT_EINVAL; }
    MapImages im;
    for (int p = 0; p < n_pairs; ++p) { im.f[p] = d_f[p]; im.g[p] = d_g[p]; }
    const int ndi = 2 * max_di + 1, ndj = 2 * max_dj + 1, nshift = ndi * ndj;
    const int nrc = (height + kMapRows - 1) / kMapRows;
    const int ncc = (j1 - j0 + kMapCols - 1) / kMapCols;
    if ((int64_t)nrc * ncc > 65535) {
        set_error("rt_xcorr_map: %d x %d window chunks of %d x %d pixels exceed 65535", nrc, ncc, kMapRows, kMapCols);
        return RT_EINVAL;
    }
    const int nchunks = nrc * ncc;
    const int npc = n_pairs * channels;
    cudaStream_t st = (cudaStream_t)stream;
    const int mchunks = (height + kMomRows - 1) / kMomRows;
    double* stats = nullptr;
    double* partial = nullptr;
    // the moment sums of pass 1 (double) share the buffer of pass 2's chunk
    // sums (float), which they precede; the buffer holds the larger of the
    // two, then pass 3's column-chunk sums (double)
    const size_t chunk_bytes = (std::max(sizeof(float) * (size_t)npc * nchunks * nshift,
                                         sizeof(double) * (size_t)n_pairs * mchunks * channels * 3) + 255) &
                               ~(size_t)255;
    const size_t ncol = (size_t)npc * ncc * nshift;
    const size_t part_bytes = chunk_bytes + sizeof(double) * ncol;
    cudaError_t e = cudaMallocAsync((void**)&stats, sizeof(double) * 3 * npc, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&partial, part_bytes, st);
    if (e == cudaSuccess) {
        xmap_moment_rows<<<dim3(mchunks, n_pairs), kMomBlock, 0, st>>>(im, height, width, channels, j0, j1, mchunks,
                                                                        partial);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        xmap_moment_stats<<<npc, 128, 0, st>>>(partial, height, channels, j0, j1, mchunks, stats);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        // shifts per thread along each axis: the smallest odd R with
        // 16 R >= the larger shift range (1, 3 or 5; ranges past 80 take
        // more tiles of R = 5)
        const int nd = std::max(ndi, ndj);
        const int R = nd <= kMapT ? 1 : (nd <= 3 * kMapT ? 3 : 5);
        const int TD = kMapT * R;
        const dim3 grid(((ndi + TD - 1) / TD) * ((ndj + TD - 1) / TD), nchunks, npc);
        float* part = (float*)partial;
        if (R == 1)
            e = launch_tiles<1>(grid, st, im, stats, height, width, channels, j0, j1, max_di, max_dj, ncc, nchunks,
                                part);
        else if (R == 3)
            e = launch_tiles<3>(grid, st, im, stats, height, width, channels, j0, j1, max_di, max_dj, ncc, nchunks,
                                part);
        else
            e = launch_tiles<5>(grid, st, im, stats, height, width, channels, j0, j1, max_di, max_dj, ncc, nchunks,
                                part);
    }
    double* colsum = partial ? (double*)((char*)partial + chunk_bytes) : nullptr;
    if (e == cudaSuccess) {
        xmap_sum<<<(unsigned)((ncol + 255) / 256), 256, 0, st>>>((const float*)partial, nrc, ncc, (int64_t)ncol,
                                                                  nshift, colsum);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        xmap_finish<<<(nshift + 255) / 256, 256, 0, st>>>(colsum, stats, n_pairs, channels, ncc, nshift, d_map);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && d_peak) {
        xmap_peak<<<1, 1024, 0, st>>>(d_map, channels, max_di, max_dj, d_peak);
        e = cudaGetLastError();
    }
    if (partial) cudaFreeAsync(partial, st);
    if (stats) cudaFreeAsync(stats, st);
    if (e != cudaSuccess) {
        set_error("rt_xcorr_map: %s", cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? RT_ENOMEM : RT_ECUDA;
    }
    return RT_OK;
}
