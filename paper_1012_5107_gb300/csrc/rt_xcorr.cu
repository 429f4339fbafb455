// rt_xcorr.cu -- image cross-correlation C(0,0) of Eqs. 14-15 (Sec. 5).
//
// Pass 1 sums, per row chunk (64 rows) and per (column, channel), the FP64
// moments (sum f, sum g, sum f^2, sum f g); consecutive threads read
// consecutive floats of a row, so the loads are coalesced.  Pass 2 reduces,
// one block per field-of-view window, the chunks and the window's columns:
// with 64-row chunks it reads 8 records per column of a 512-row image (it
// read 64 with 8-row chunks, and one block per window made that the call's
// latency).  It forms
//   C_c = (S_fg - S_f S_g / N) / (S_ff - S_f^2 / N)
// per channel (the numerator and denominator of Eq. 15 after the mean
// subtraction of Eq. 14) and the same ratio over the stacked channels.
#include <cmath>

#include "rt_internal.h"

namespace grt {

struct alignas(32) Moments { double sf, sg, sff, sfg; };

constexpr int kXcorrBlock = 256;
constexpr int kXcorrRows = 64;         // rows per chunk of pass 1
constexpr int kXcorrMaxChunks = 64;

int xcorr_chunks(int H)
{
    const int c = (H + kXcorrRows - 1) / kXcorrRows;
    return c < kXcorrMaxChunks ? c : kXcorrMaxChunks;
}

__global__ void __launch_bounds__(kXcorrBlock) xcorr_columns(const float* __restrict__ f, const float* __restrict__ g,
                                                           int H, int WC, int rows_per_chunk,
                                                           Moments* __restrict__ partial)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (q >= WC) return;
    const int i0 = chunk * rows_per_chunk;
    const int i1 = min(H, i0 + rows_per_chunk);
    double sf = 0.0, sg = 0.0, sff = 0.0, sfg = 0.0;
    for (int i = i0; i < i1; ++i) {
        const double a = __ldg(f + (size_t)i * WC + q), b = __ldg(g + (size_t)i * WC + q);
        sf += a;
        sg += b;
        sff += a * a;
        sfg += a * b;
    }
    partial[(size_t)chunk * WC + q] = Moments{sf, sg, sff, sfg};
}

__global__ void __launch_bounds__(kXcorrBlock) xcorr_windows(const Moments* __restrict__ partial, int nchunks, int H,
                                                           int W, int C, Windows win, double* __restrict__ out)
{
    __shared__ double red[kXcorrBlock / 32][16];
    const int w = blockIdx.x;
    const int j0 = win.j0[w], j1 = win.j1[w];
    const int ncols = j1 - j0;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int t = threadIdx.x; t < nchunks * ncols; t += blockDim.x) {
        const int chunk = t / ncols, j = j0 + t % ncols;
        const Moments* p = partial + (size_t)chunk * W * C + (size_t)j * C;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c < C) {
                const Moments v = p[c];
                acc[4 * c + 0] += v.sf;
                acc[4 * c + 1] += v.sg;
                acc[4 * c + 2] += v.sff;
                acc[4 * c + 3] += v.sfg;
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        double x = acc[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp][q] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[16];
        for (int q = 0; q < 16; ++q) {
            tot[q] = 0.0;
            for (int k = 0; k < kXcorrBlock / 32; ++k) tot[q] += red[k][q];
        }
        const double N = (double)H * (double)ncols;
        double num_all = 0.0, den_all = 0.0;
        for (int c = 0; c < C; ++c) {
            const double sf = tot[4 * c], sg = tot[4 * c + 1], sff = tot[4 * c + 2], sfg = tot[4 * c + 3];
            const double num = sfg - sf * sg / N;
            const double den = sff - sf * sf / N;
            out[w * (C + 1) + c] = num / den;
            num_all += num;
            den_all += den;
        }
        out[w * (C + 1) + C] = num_all / den_all;
    }
}

cudaError_t launch_xcorr(const float* f, const float* g, int H, int W, int C, const Windows& win, void* partial,
                         double* out, cudaStream_t stream)
{
    const int WC = W * C;
    const int nchunks = xcorr_chunks(H);
    const int rpc = (H + nchunks - 1) / nchunks;
    dim3 grid1((WC + kXcorrBlock - 1) / kXcorrBlock, nchunks);
    xcorr_columns<<<grid1, kXcorrBlock, 0, stream>>>(f, g, H, WC, rpc, (Moments*)partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    xcorr_windows<<<win.n, kXcorrBlock, 0, stream>>>((const Moments*)partial, nchunks, H, W, C, win, out);
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
