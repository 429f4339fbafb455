// rt_xcorr_map.cu -- the cross-correlation function C(di, dj) of Eq. 15 over
// pixel shifts, its peak and its mean over several reference pairs (Sec. 5).
//
// Pass 1 forms, over the field-of-view window of columns j0..j1-1, the means
// of Eq. 14 and the denominator sum (f - <f>)^2 of Eq. 15 in FP64: blocks of
// 4 image rows per pair sum them (FP64 is slow on this GPU, so the work is
// spread over many SMs), then a block per pair and channel adds the chunks.
// Pass 2 is a direct correlation in tiles: a block owns 8 x 32 R shifts
// (di, dj) and a chunk of 32 image rows of one pair and channel; per row it
// stages the window's f row and the 8 g rows the shifts need (zero outside
// the window, where the finite photographs have no values) in shared memory,
// and every thread accumulates its R shifts' products over the chunk with
// FP32 FMA (see xmap_tiles).
// Pass 3 sums the chunks in FP64, divides by the denominators, stacks the
// channels (sum of numerators over sum of denominators) and averages the maps
// of the pairs; pass 4 finds the peak of the stacked mean map and its shift.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rt_internal.h"

namespace grt {

constexpr int kMapTDI = 8;        // shifts in di per block
constexpr int kMapTDJ = 32;       // shifts in dj per block (one warp)
constexpr int kMapTW = 128;       // columns staged per step
constexpr int kMapRows = 32;      // image rows per chunk
constexpr int kMapBlock = kMapTDI * kMapTDJ;
constexpr int kMapMaxShift = 64;
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

// One block: 8 row shifts (one per warp) x 32 R column shifts, lane l owning
// the R consecutive column shifts dj_lo + l R + k.  Along a staged row a lane
// keeps the R g values its shifts need in registers and slides them by one
// per column, so each step costs one broadcast f load and one g load for R
// FMAs; R is odd, so the lanes' g loads (stride R) hit distinct banks.
template <int R>
__global__ void __launch_bounds__(kMapBlock) xmap_tiles(MapImages im, const double* __restrict__ stats, int H, int W,
                                                        int C, int j0, int j1, int max_di, int max_dj, int nchunks,
                                                        double* __restrict__ partial)
{
    constexpr int TJ = kMapTDJ * R;              // column shifts per block
    constexpr int GW = kMapTW + TJ;              // staged g columns per row
    __shared__ float f_s[kMapTW];
    __shared__ float g_s[kMapTDI][GW];
    const int ndi = 2 * max_di + 1, ndj = 2 * max_dj + 1;
    const int tiles_dj = (ndj + TJ - 1) / TJ;
    const int tdi = blockIdx.x / tiles_dj, tdj = blockIdx.x % tiles_dj;
    const int chunk = blockIdx.y;
    const int pc = blockIdx.z;
    const int pair = pc / C, c = pc % C;
    const float* f = im.f[pair];
    const float* g = im.g[pair];
    const float mf = (float)stats[3 * pc + 0], mg = (float)stats[3 * pc + 1];
    const int di_lo = -max_di + tdi * kMapTDI, dj_lo = -max_dj + tdj * TJ;
    const int ty = threadIdx.x / kMapTDJ, tx = threadIdx.x % kMapTDJ;
    const int i0 = chunk * kMapRows, i1 = min(H, i0 + kMapRows);
    float acc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = 0.0f;
    const float* gr = &g_s[ty][tx * R];
    for (int i = i0; i < i1; ++i) {
        for (int jt = j0; jt < j1; jt += kMapTW) {
            for (int q = threadIdx.x; q < kMapTW; q += kMapBlock) {
                const int j = jt + q;
                f_s[q] = (j < j1) ? __ldg(f + ((int64_t)i * W + j) * C + c) - mf : 0.0f;
            }
            for (int q = threadIdx.x; q < kMapTDI * GW; q += kMapBlock) {
                const int r = q / GW, col = q % GW;
                const int ig = i + di_lo + r, jg = jt + dj_lo + col;
                g_s[r][col] = (ig >= 0 && ig < H && jg >= j0 && jg < j1)
                                  ? __ldg(g + ((int64_t)ig * W + jg) * C + c) - mg
                                  : 0.0f;
            }
            __syncthreads();
            float win[R];
#pragma unroll
            for (int k = 0; k < R; ++k) win[k] = gr[k];
#pragma unroll 32
            for (int q = 0; q < kMapTW; ++q) {
                const float fv = f_s[q];
#pragma unroll
                for (int k = 0; k < R; ++k) acc[k] = fmaf(fv, win[k], acc[k]);
#pragma unroll
                for (int k = 0; k + 1 < R; ++k) win[k] = win[k + 1];
                win[R - 1] = gr[q + R];
            }
            __syncthreads();
        }
    }
    const int di = di_lo + ty;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int dj = dj_lo + tx * R + k;
        if (di <= max_di && dj <= max_dj) {
            const int s = (di + max_di) * ndj + (dj + max_dj);
            partial[((int64_t)pc * nchunks + chunk) * ((int64_t)ndi * ndj) + s] = (double)acc[k];
        }
    }
}

__global__ void __launch_bounds__(256) xmap_finish(const double* __restrict__ partial,
                                                   const double* __restrict__ stats, int n_pairs, int C, int nchunks,
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
            for (int k = 0; k < nchunks; ++k) num += partial[((int64_t)pc * nchunks + k) * nshift + s];
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
    const int nchunks = (height + kMapRows - 1) / kMapRows;
    const int npc = n_pairs * channels;
    cudaStream_t st = (cudaStream_t)stream;
    const int mchunks = (height + kMomRows - 1) / kMomRows;
    double* stats = nullptr;
    double* partial = nullptr;
    // the moment sums of pass 1 share the buffer of pass 2's partial sums,
    // which they precede; the buffer holds the larger of the two
    const size_t part_doubles = std::max((size_t)npc * nchunks * nshift, (size_t)n_pairs * mchunks * channels * 3);
    cudaError_t e = cudaMallocAsync((void**)&stats, sizeof(double) * 3 * npc, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&partial, sizeof(double) * part_doubles, st);
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
        // column shifts per lane: the smallest odd R with 32 R >= ndj (1, 3 or 5)
        const int R = ndj <= kMapTDJ ? 1 : (ndj <= 3 * kMapTDJ ? 3 : 5);
        const dim3 grid(((ndi + kMapTDI - 1) / kMapTDI) * ((ndj + kMapTDJ * R - 1) / (kMapTDJ * R)), nchunks, npc);
        if (R == 1)
            xmap_tiles<1><<<grid, kMapBlock, 0, st>>>(im, stats, height, width, channels, j0, j1, max_di, max_dj,
                                                      nchunks, partial);
        else if (R == 3)
            xmap_tiles<3><<<grid, kMapBlock, 0, st>>>(im, stats, height, width, channels, j0, j1, max_di, max_dj,
                                                      nchunks, partial);
        else
            xmap_tiles<5><<<grid, kMapBlock, 0, st>>>(im, stats, height, width, channels, j0, j1, max_di, max_dj,
                                                      nchunks, partial);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        xmap_finish<<<(nshift + 255) / 256, 256, 0, st>>>(partial, stats, n_pairs, channels, nchunks, nshift, d_map);
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
