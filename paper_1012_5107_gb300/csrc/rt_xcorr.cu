// rt_xcorr.cu -- image cross-correlation C(0,0) of Eqs. 14-15 (Sec. 5).
//
// The window sums are FP64 moments (sum f, sum g, sum f^2, sum f g) per
// channel, and FP64 arithmetic is slow on this GPU (two fused multiply-adds
// per SM and cycle), so every pass spreads its FP64 work over many SMs:
//   1. column moments per row chunk (64 rows; at most 64 chunks, so taller
//      images have longer chunks): a block takes 32 columns of
//      the flattened row (one per lane, so loads are coalesced) and splits
//      the chunk's rows over its 8 warps, then adds the warps' sums;
//   2. window slices: a block per (window, slice) adds the chunks' moments
//      of 1/64 of the window's columns;
//   3. a block adds each window's slices, and one thread per window forms
//        C_c = (S_fg - S_f S_g / N) / (S_ff - S_f^2 / N)
//      per channel (the numerator and denominator of Eq. 15 after the mean
//      subtraction of Eq. 14) and the same ratio over the stacked channels.
// Images of at most 4096 values and 64 values per row (a centre line) take
// one block instead: a launch costs more than their arithmetic.
// The order of the additions is fixed, so results repeat bit for bit.
#include <cmath>

#include "rt_internal.h"

namespace grt {

struct alignas(32) Moments { double sf, sg, sff, sfg; };

constexpr int kXcorrBlock = 256;
constexpr int kXcorrWarps = kXcorrBlock / 32;
constexpr int kXcorrRows = 64;         // rows per chunk of pass 1
constexpr int kXcorrMaxChunks = 64;
constexpr int kXcorrSlices = 64;       // column slices per window in pass 2
constexpr int kXcorrSmallRow = 64;     // one-block path: values per row (W C) at most
constexpr int kXcorrSmallAll = 4096;   // and values (H W C) at most
static_assert(kXcorrTailBytes >= (size_t)kMaxWindows * kXcorrSlices * 16 * sizeof(double) + 256,
              "window-slice scratch too small");

int xcorr_chunks(int H)
{
    const int c = (H + kXcorrRows - 1) / kXcorrRows;
    return c < kXcorrMaxChunks ? c : kXcorrMaxChunks;
}

static size_t xcorr_chunk_bytes(int H, int W, int C)
{
    const size_t b = (size_t)xcorr_chunks(H) * (size_t)W * (size_t)C * sizeof(Moments);
    return (b + 255) & ~(size_t)255;
}

static bool xcorr_one_block(int H, int W, int C)
{
    const int WC = W * C;
    return WC <= kXcorrSmallRow && (int64_t)H * WC <= kXcorrSmallAll;
}

size_t xcorr_scratch_bytes(int H, int W, int C)
{
    return xcorr_one_block(H, W, C) ? 0 : xcorr_chunk_bytes(H, W, C) + kXcorrTailBytes;
}

__global__ void __launch_bounds__(kXcorrBlock) xcorr_columns(const float* __restrict__ f, const float* __restrict__ g,
                                                           int H, int WC, int rows_per_chunk,
                                                           Moments* __restrict__ partial)
{
    __shared__ double red[4][kXcorrWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = blockIdx.x * 32 + lane;
    const int chunk = blockIdx.y;
    const int i0 = chunk * rows_per_chunk;
    const int i1 = min(H, i0 + rows_per_chunk);
    double sf = 0.0, sg = 0.0, sff = 0.0, sfg = 0.0;
    if (q < WC) {
#pragma unroll 4
        for (int i = i0 + warp; i < i1; i += kXcorrWarps) {
            const double a = __ldg(f + (size_t)i * WC + q), b = __ldg(g + (size_t)i * WC + q);
            sf += a;
            sg += b;
            sff += a * a;
            sfg += a * b;
        }
    }
    red[0][warp][lane] = sf;
    red[1][warp][lane] = sg;
    red[2][warp][lane] = sff;
    red[3][warp][lane] = sfg;
    __syncthreads();
    if (threadIdx.x < 4 * 32) {
        const int m = threadIdx.x >> 5, l = threadIdx.x & 31;     // moment, column of the block
        const int qq = blockIdx.x * 32 + l;
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kXcorrWarps; ++w) s += red[m][w][l];
        if (qq < WC) reinterpret_cast<double*>(partial + (size_t)chunk * WC + qq)[m] = s;
    }
}

// Pass 2.  A chunk's moments of the slice's columns are contiguous doubles,
// V = 4 C per column (channel-major moments), so a block reads them
// coalesced with T = a multiple of V threads: every thread then meets only
// one of the V values and adds it with one FP64 add per double (a shuffle
// tree over 16 accumulators spent most of the slow FP64 issue on idle lanes).
__global__ void __launch_bounds__(kXcorrBlock) xcorr_slices(const Moments* __restrict__ partial, int nchunks, int W,
                                                          int C, Windows win, double* __restrict__ slices)
{
    __shared__ double red[kXcorrBlock];
    const int w = blockIdx.x, s = blockIdx.y;
    const int j0 = win.j0[w];
    const int ncols = max(0, win.j1[w] - j0);
    const int c0 = j0 + (int)((int64_t)ncols * s / kXcorrSlices);
    const int n = j0 + (int)((int64_t)ncols * (s + 1) / kXcorrSlices) - c0;
    const int V = 4 * C;
    const int T = (kXcorrBlock / V) * V;
    const int t = threadIdx.x;
    double acc = 0.0;
    if (t < T) {
        // k runs over (chunk, offset) pairs; k = t mod T keeps the value
        // index k mod V = t mod V, since the row length and T are multiples of V
        const int len = n * V;
        const double* base = reinterpret_cast<const double*>(partial) + (size_t)c0 * V;
        const size_t row = (size_t)W * V;
#pragma unroll 4
        for (int k = t; k < nchunks * len; k += T) {
            const int ch = k / len, o = k - ch * len;
            acc += __ldg(base + ch * row + o);
        }
    }
    red[t] = acc;
    __syncthreads();
    if (t < V) {
        double tot = 0.0;
        for (int k = t; k < T; k += V) tot += red[k];
        slices[((size_t)w * kXcorrSlices + s) * 16 + t] = tot;
    }
}

// Pass 3: thread (window, value) adds the window's slices; then one thread
// per window forms C.
static_assert(kMaxWindows * 16 == kXcorrBlock, "one finishing thread per window and value");
__global__ void __launch_bounds__(kXcorrBlock) xcorr_finish(const double* __restrict__ slices, int H, int C,
                                                          Windows win, double* __restrict__ out)
{
    __shared__ double tot[kMaxWindows][16];
    const int t = threadIdx.x;
    const int w = t >> 4, q = t & 15;
    if (w < win.n && q < 4 * C) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < kXcorrSlices; ++k) s += slices[((size_t)w * kXcorrSlices + k) * 16 + q];
        tot[w][q] = s;
    }
    __syncthreads();
    if (t >= win.n) return;
    const double N = (double)H * (double)max(0, win.j1[t] - win.j0[t]);
    double num_all = 0.0, den_all = 0.0;
    for (int c = 0; c < C; ++c) {
        const double sf = tot[t][4 * c], sg = tot[t][4 * c + 1], sff = tot[t][4 * c + 2], sfg = tot[t][4 * c + 3];
        const double num = sfg - sf * sg / N;
        const double den = sff - sf * sf / N;
        out[t * (C + 1) + c] = num / den;
        num_all += num;
        den_all += den;
    }
    out[t * (C + 1) + C] = num_all / den_all;
}

// The one-block path.  Threads stride over the image's values with a
// stride T that is a multiple of W C, so each meets one column and channel
// (q = t mod W C); the column moments are the sums over the threads of each
// q, and one thread per window adds its columns and forms C as in pass 3.
__global__ void __launch_bounds__(kXcorrBlock) xcorr_small(const float* __restrict__ f, const float* __restrict__ g,
                                                         int H, int W, int C, Windows win, double* __restrict__ out)
{
    __shared__ double red[4][kXcorrBlock];
    __shared__ double col[4][kXcorrSmallRow];
    const int WC = W * C;
    const int T = (kXcorrBlock / WC) * WC;
    const int n = H * WC;
    const int t = threadIdx.x;
    double sf = 0.0, sg = 0.0, sff = 0.0, sfg = 0.0;
    if (t < T) {
#pragma unroll 4
        for (int e = t; e < n; e += T) {
            const double a = __ldg(f + e), b = __ldg(g + e);
            sf += a;
            sg += b;
            sff += a * a;
            sfg += a * b;
        }
    }
    red[0][t] = sf;
    red[1][t] = sg;
    red[2][t] = sff;
    red[3][t] = sfg;
    __syncthreads();
    if (t < 4 * WC) {
        const int m = t / WC, q = t - m * WC;
        double acc = 0.0;
        for (int k = q; k < T; k += WC) acc += red[m][k];
        col[m][q] = acc;
    }
    __syncthreads();
    if (t >= win.n) return;
    const int j0 = win.j0[t], j1 = win.j1[t];
    const double N = (double)H * (double)max(0, j1 - j0);
    double num_all = 0.0, den_all = 0.0;
    for (int c = 0; c < C; ++c) {
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = j0; j < j1; ++j)
            for (int m = 0; m < 4; ++m) v[m] += col[m][j * C + c];
        const double num = v[3] - v[0] * v[1] / N;
        const double den = v[2] - v[0] * v[0] / N;
        out[t * (C + 1) + c] = num / den;
        num_all += num;
        den_all += den;
    }
    out[t * (C + 1) + C] = num_all / den_all;
}

cudaError_t launch_xcorr(const float* f, const float* g, int H, int W, int C, const Windows& win, void* scratch,
                         double* out, cudaStream_t stream)
{
    const int WC = W * C;
    if (xcorr_one_block(H, W, C)) {
        xcorr_small<<<1, kXcorrBlock, 0, stream>>>(f, g, H, W, C, win, out);
        return cudaGetLastError();
    }
    const int nchunks = xcorr_chunks(H);
    const int rpc = (H + nchunks - 1) / nchunks;
    Moments* partial = (Moments*)scratch;
    double* slices = (double*)((char*)scratch + xcorr_chunk_bytes(H, W, C));
    dim3 grid1((WC + 31) / 32, nchunks);
    xcorr_columns<<<grid1, kXcorrBlock, 0, stream>>>(f, g, H, WC, rpc, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    xcorr_slices<<<dim3(win.n, kXcorrSlices), kXcorrBlock, 0, stream>>>(partial, nchunks, W, C, win, slices);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    xcorr_finish<<<1, kXcorrBlock, 0, stream>>>(slices, H, C, win, out);
    return cudaGetLastError();
}

void fov_windows(int W, double hfov_deg, const double* fov_deg, int n_fov, Windows* win)
{
    const double tx = tan(0.5 * hfov_deg * kPi / 180.0);
    win->n = n_fov;
    for (int q = 0; q < n_fov; ++q) {
        int lo = W, hi = -1;
        for (int j = 0; j < W; ++j) {
            const double px = 2.0 * (j + 0.5) / W - 1.0;
            const double alpha = atan(fabs(px) * tx) * 180.0 / kPi;
            if (alpha <= 0.5 * fov_deg[q] + 1e-9) {
                if (j < lo) lo = j;
                if (j > hi) hi = j;
            }
        }
        if (hi < lo) { lo = 0; hi = -1; }
        win->j0[q] = lo;
        win->j1[q] = hi + 1;
    }
}

}  // namespace grt
