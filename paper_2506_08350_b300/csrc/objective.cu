// The paper's training objective on sm_103a: L = L_recon + L_SSIM on the
// focal stack (the loss paragraph of Sec. 4.1), and the Adan optimiser step
// (Sec. 5, implementation).
//
//   L_recon = mean over (view, plane, channel, pixel) of d^2 (1 + M + I_gt^2),
//             d = I - I_gt, M the binary plane mask (|I M - I_gt M|^2 and
//             |I I_gt - I_gt I_gt|^2 are d^2 M and d^2 I_gt^2);
//   L_SSIM  = lambda_1 mean over (view, plane, channel) of (1 - SSIM).
// SSIM is the structural similarity of Wang et al.: local means, variances
// and covariance under an 11 x 11 Gaussian window (standard deviation 1.5,
// the image continued by zeros), constants C1 = 0.01^2, C2 = 0.03^2.  With
// n the number of intensity values, L = (1/n) sum (d^2 w + lambda_1 (1 - S))
// and dL/dI = (2 d w - lambda_1 (G(dS/dmx) + 2 I G(dS/dm2) + I_gt G(dS/dmxy)))
// / n, G the (self-adjoint) window average, m2 = G(x^2 + y^2) and mxy =
// G(x y): the variances enter SSIM only through their sum, so pass 1 needs
// four window averages (x, y, x^2 + y^2, x y) and pass 2 three.
//
// Both passes take a 32 x 32 output tile per 128-thread block.  The window is
// separable: a horizontal pass over the 42 halo rows (each thread slides over
// four neighbouring columns, so an input is read 3.5 times, not 11) writes the
// row sums to shared memory, and a vertical pass in registers (each thread
// owns a column and eight output rows and scatters every row sum into the
// outputs it touches) finishes the window.  Quantities travel in pairs through
// packed FP32x2 FMAs.  A shared input row holds 48 columns starting 16-byte
// aligned three columns left of the halo, so the halo arrives by 16-byte
// asynchronous copies when rows are 16-byte aligned in memory (W a multiple
// of 4) and the horizontal pass reads it with 16-byte loads (eight lanes of a
// row cover all banks).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>

#include "common.cuh"

namespace hcgs {

constexpr int SS_R = 5;                  // window radius
constexpr int SS_TAPS = 2 * SS_R + 1;    // 11
constexpr int SS_TW = 32, SS_TH = 32;    // output tile
constexpr int SS_EW = SS_TW + 2 * SS_R;  // halo tile width (42)
constexpr int SS_EH = SS_TH + 2 * SS_R;  // halo tile height (42)
constexpr int SS_XW = 48;                // shared row of an input plane: columns x0 - 3 .. x0 + 44
constexpr int SS_XO = 3;                 // shared column of the halo's first column x0 = tile x - 5
constexpr int SS_K = 4;                  // columns per thread in the horizontal pass
constexpr int SS_ROWS = 8;               // output rows per thread in the vertical pass
constexpr int SS_NT = SS_TH / SS_ROWS * 32;  // 128 threads
constexpr float SS_C1 = 0.01f * 0.01f, SS_C2 = 0.03f * 0.03f;
static_assert(SS_XW % 4 == 0 && SS_XO + SS_EW <= SS_XW && (SS_XO + SS_R) % 4 == 0, "row layout");

// the normalised 1D factor of the window, formed on the host in double, and
// the same taps paired for the packed FP32x2 FMAs
__constant__ float c_ssim_g[SS_TAPS];
__constant__ float2 c_ssim_g2[SS_TAPS];

static cudaError_t ssim_window_upload() {
    static bool done[256] = {};  // per device (the table never changes)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 256 && done[dev]) return cudaSuccess;
    double g[SS_TAPS], s = 0.0;
    for (int k = 0; k < SS_TAPS; k++) {
        const double x = k - SS_R;
        g[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    float gf[SS_TAPS];
    for (int k = 0; k < SS_TAPS; k++) gf[k] = (float)(g[k] / s);
    float2 gf2[SS_TAPS];
    for (int k = 0; k < SS_TAPS; k++) gf2[k] = make_float2(gf[k], gf[k]);
    e = cudaMemcpyToSymbol(c_ssim_g, gf, sizeof(gf));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ssim_g2, gf2, sizeof(gf2));
    if (e == cudaSuccess && dev >= 0 && dev < 256) done[dev] = true;
    return e;
}

__device__ __forceinline__ float2 gtap(int t) { return c_ssim_g2[t]; }

// Horizontal window sums of NP quantity pairs and NS single quantities
// derived from NIN input planes: inp[NIN][SS_EH][SS_XW] -> h2[NP][SS_EH][SS_TW]
// (float2) and h1[NS][SS_EH][SS_TW].  quant(in, pairs, singles) forms the
// quantities of one input column.
template <int NIN, int NP, int NS, class Quant>
__device__ __forceinline__ void ssim_rows(const float (*inp)[SS_EH][SS_XW], float2 (*h2)[SS_EH][SS_TW],
                                          float (*h1)[SS_EH][SS_TW], Quant quant) {
    constexpr int NS1 = NS > 0 ? NS : 1;
    constexpr int NV = (SS_XO + SS_K + 2 * SS_R + 3) / 4;  // 16-byte loads per row segment (5)
    for (int it = threadIdx.x; it < SS_EH * (SS_TW / SS_K); it += SS_NT) {
        const int r = it / (SS_TW / SS_K), c0 = (it % (SS_TW / SS_K)) * SS_K;
        float2 a2[NP][SS_K];
        float a1[NS1][SS_K];
#pragma unroll
        for (int k = 0; k < SS_K; k++) {
#pragma unroll
            for (int q = 0; q < NP; q++) a2[q][k] = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < NS1; q++) a1[q][k] = 0.f;
        }
        // the row segment of the outputs c0 .. c0 + 3: halo columns c0 .. c0 + 13
        float seg[NIN][4 * NV];
#pragma unroll
        for (int a = 0; a < NIN; a++) {
            const float4* src = reinterpret_cast<const float4*>(&inp[a][r][c0]);
#pragma unroll
            for (int u = 0; u < NV; u++) {
                const float4 v = src[u];
                seg[a][4 * u] = v.x;
                seg[a][4 * u + 1] = v.y;
                seg[a][4 * u + 2] = v.z;
                seg[a][4 * u + 3] = v.w;
            }
        }
#pragma unroll
        for (int i = 0; i < SS_K + 2 * SS_R; i++) {
            float in[NIN];
            float2 v2[NP];
            float v1[NS1];
#pragma unroll
            for (int a = 0; a < NIN; a++) in[a] = seg[a][SS_XO + i];
            quant(in, v2, v1);
#pragma unroll
            for (int k = 0; k < SS_K; k++) {
                const int t = i - k;
                if (t >= 0 && t < SS_TAPS) {
#pragma unroll
                    for (int q = 0; q < NP; q++) a2[q][k] = __ffma2_rn(gtap(t), v2[q], a2[q][k]);
#pragma unroll
                    for (int q = 0; q < NS; q++) a1[q][k] = fmaf(c_ssim_g[t], v1[q], a1[q][k]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NP; q++) {
            float4* d = reinterpret_cast<float4*>(&h2[q][r][c0]);
            d[0] = make_float4(a2[q][0].x, a2[q][0].y, a2[q][1].x, a2[q][1].y);
            d[1] = make_float4(a2[q][2].x, a2[q][2].y, a2[q][3].x, a2[q][3].y);
        }
#pragma unroll
        for (int q = 0; q < NS; q++)
            *reinterpret_cast<float4*>(&h1[q][r][c0]) = make_float4(a1[q][0], a1[q][1], a1[q][2], a1[q][3]);
    }
}

// Vertical window sums for the thread's column and SS_ROWS output rows.
template <int NP, int NS>
__device__ __forceinline__ void ssim_cols(const float2 (*h2)[SS_EH][SS_TW], const float (*h1)[SS_EH][SS_TW],
                                          int col, int row0, float2 (&o2)[NP][SS_ROWS],
                                          float (&o1)[NS > 0 ? NS : 1][SS_ROWS]) {
#pragma unroll
    for (int k = 0; k < SS_ROWS; k++) {
#pragma unroll
        for (int q = 0; q < NP; q++) o2[q][k] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < NS; q++) o1[q][k] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < SS_ROWS + 2 * SS_R; i++) {
        float2 v2[NP];
        float v1[NS > 0 ? NS : 1];
#pragma unroll
        for (int q = 0; q < NP; q++) v2[q] = h2[q][row0 + i][col];
#pragma unroll
        for (int q = 0; q < NS; q++) v1[q] = h1[q][row0 + i][col];
#pragma unroll
        for (int k = 0; k < SS_ROWS; k++) {
            const int t = i - k;
            if (t >= 0 && t < SS_TAPS) {
#pragma unroll
                for (int q = 0; q < NP; q++) o2[q][k] = __ffma2_rn(gtap(t), v2[q], o2[q][k]);
#pragma unroll
                for (int q = 0; q < NS; q++) o1[q][k] = fmaf(c_ssim_g[t], v1[q], o1[q][k]);
            }
        }
    }
}

__device__ __forceinline__ float block_sum(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < SS_NT / 32; i++) s += red[i];  // fixed order: deterministic
    return s;
}

// Asynchronous 4- / 8-byte copies global -> shared; a copy with valid = false
// reads nothing and writes zeros (the window's zero continuation).
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}

// Copies of the halo rows y0 .. y0 + SS_EH - 1 of one image into shared rows
// of SS_XW columns starting at column xs of the image (elements of ES bytes).
// VEC: 16-byte chunks (xs and the image's row pitch 16-byte aligned: a chunk
// lies wholly inside or wholly outside the row); otherwise one element per
// copy, the halo columns only.  put(dst_row, dst_col, off, ok, bytes) issues
// one copy of `bytes` at element offset `off` of the image (0 where ok is false).
template <bool VEC, int ES, class Put>
__device__ __forceinline__ void halo_copy(int xs, int y0, int H, int W, Put put) {
    if constexpr (VEC) {
        constexpr int PER = 16 / ES, NCH = SS_XW / PER, TOT = SS_EH * NCH;
#pragma unroll
        for (int k = 0; k < (TOT + SS_NT - 1) / SS_NT; k++) {
            const int e = threadIdx.x + k * SS_NT;
            const int r = e / NCH, ch = e % NCH, gy = y0 + r, gx = xs + ch * PER;
            const bool ok = gy >= 0 && gy < H && gx >= 0 && gx < W;
            if (e < TOT) put(r, ch * PER, ok ? (unsigned)gy * (unsigned)W + gx : 0u, ok, 16);
        }
    } else {
        const int lane = threadIdx.x & 31;
        const int gx0 = xs + SS_XO + lane, gx1 = gx0 + 32;
        const bool c0ok = gx0 >= 0 && gx0 < W, c1ok = lane < SS_EW - 32 && gx1 >= 0 && gx1 < W;
        for (int r = threadIdx.x >> 5; r < SS_EH; r += SS_NT / 32) {
            const int gy = y0 + r;
            const bool rok = gy >= 0 && gy < H;
            const unsigned row = rok ? (unsigned)gy * (unsigned)W : 0u;
            put(r, SS_XO + lane, rok && c0ok ? row + gx0 : 0u, rok && c0ok, ES);
            if (lane < SS_EW - 32) put(r, SS_XO + 32 + lane, rok && c1ok ? row + gx1 : 0u, rok && c1ok, ES);
        }
    }
}

__device__ __forceinline__ void cp_async_n(void* dst, const void* src, bool ok, int bytes) {
    if (bytes == 16)
        cp_async16(dst, src, ok);
    else if (bytes == 8)
        cp_async8(dst, src, ok);
    else
        cp_async4(dst, src, ok);
}

// ---- tensor-memory-access (TMA) halo tiles (16-byte aligned rows) ----
// A box of SS_XW x SS_EH elements at (x, y) of image z lands in a dense
// shared tile [SS_EH][SS_XW] (the layout of the copies above); elements
// outside the image arrive as zeros (the window's zero continuation).
struct SsimMaps {
    CUtensorMap a, b;  // pass 1: intensities (or field) and targets; pass 2: the three maps (a)
};

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* m, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* m, int x, int y, int z, int w,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
        : "memory");
}

// Waits (bounded) for the tile copies (the barrier initialised and the copies
// issued before a block barrier); on a timeout waits once more for the copies
// in flight, records it in the status word and tells the CTA to leave.
__device__ __forceinline__ bool tma_tiles_ready(uint64_t* bar, int* status) {
    const bool ok = __syncthreads_and(mbar_wait(bar, 0));
    if (!ok && threadIdx.x == 0) {
        mbar_wait(bar, 0);
        atomicOr(status, STATUS_WAIT_TIMEOUT);
    }
    return ok;
}

// Pass 1 over each (view, plane, channel) image: the partial derivatives of
// the SSIM map dS/dmx, dS/dm2, dS/dmxy (to dmap[3][n]) and the block's part of
// sum (d^2 w + lambda (1 - S)).  The intensities come either from I or, when
// V is given, as |V|^2 of the propagated field (then also written to I for
// pass 2).  grid (tiles x, tiles y, B L C), SS_NT threads.
template <bool FROM_FIELD, bool VEC>
__global__ void __launch_bounds__(SS_NT)
    k_ssim_partials(const float2* __restrict__ V, float* __restrict__ I, const float* __restrict__ Igt,
                    const float* __restrict__ M, int C, int H, int W, float lam, int plain, float* __restrict__ dmap,
                    float* __restrict__ partials, const __grid_constant__ SsimMaps maps, int* status) {
    __shared__ __align__(128) float inp[2][SS_EH][SS_XW];
    __shared__ __align__(128) float2 h[2][SS_EH][SS_TW];
    __shared__ float red[SS_NT / 32];
    __shared__ __align__(8) uint64_t bar;
    const int img = blockIdx.z;
    const size_t HW = (size_t)H * W, n = (size_t)gridDim.z * HW;
    const int xs = blockIdx.x * SS_TW - SS_R - SS_XO, y0 = blockIdx.y * SS_TH - SS_R;
    const float* ysrc = Igt + (size_t)img * HW;
    const float* xsrc = I + (size_t)img * HW;
    const float2* vsrc = FROM_FIELD ? V + (size_t)img * HW : nullptr;
    // the field's halo is staged in the row-sum buffer (idle until the row pass)
    float2 (*stage)[SS_XW] = reinterpret_cast<float2 (*)[SS_XW]>(&h[0][0][0]);
    static_assert(sizeof(float2) * SS_EH * SS_XW <= sizeof(h), "staging fits");
    if constexpr (VEC) {
        // two tensor copies by one thread, completed on the barrier
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            mbar_init_fence();
            constexpr unsigned bytes = SS_EH * SS_XW * (sizeof(float) + (FROM_FIELD ? sizeof(float2) : sizeof(float)));
            mbar_expect_tx(&bar, bytes);
            tma_load_3d(&inp[1][0][0], &maps.b, xs, y0, img, &bar);
            tma_load_3d(FROM_FIELD ? (void*)&stage[0][0] : (void*)&inp[0][0][0], &maps.a, xs, y0, img, &bar);
        }
        __syncthreads();  // the barrier is initialised before anyone waits on it
    } else {
        halo_copy<VEC, 4>(xs, y0, H, W, [&](int r, int c, unsigned off, bool ok, int bytes) {
            cp_async_n(&inp[1][r][c], ysrc + off, ok, bytes);
            if constexpr (!FROM_FIELD) cp_async_n(&inp[0][r][c], xsrc + off, ok, bytes);
        });
        if constexpr (FROM_FIELD)
            halo_copy<VEC, 8>(xs, y0, H, W, [&](int r, int c, unsigned off, bool ok, int bytes) {
                cp_async_n(&stage[r][c], vsrc + off, ok, bytes);
            });
    }
    // the mask values of the thread's outputs, needed in the epilogue
    const int col = threadIdx.x & 31, row0 = (threadIdx.x >> 5) * SS_ROWS;
    const float* m = M ? M + (size_t)(img / C) * HW : nullptr;  // masks per (view, plane)
    const int gx = blockIdx.x * SS_TW + col;
    float mv[SS_ROWS];
#pragma unroll
    for (int k = 0; k < SS_ROWS; k++) {
        const int gy = blockIdx.y * SS_TH + row0 + k;
        mv[k] = (m && gx < W && gy < H) ? m[(size_t)gy * W + gx] : 0.f;
    }
    if constexpr (VEC) {
        if (!tma_tiles_ready(&bar, status)) return;
    } else {
        cp_async_wait_all();
        __syncthreads();
    }
    if constexpr (FROM_FIELD) {
        const int lane = threadIdx.x & 31;
        for (int r = threadIdx.x >> 5; r < SS_EH; r += SS_NT / 32) {
            const float2 v = stage[r][SS_XO + lane];
            inp[0][r][SS_XO + lane] = fmaf(v.x, v.x, v.y * v.y);
            if (lane < SS_EW - 32) {
                const float2 u = stage[r][SS_XO + 32 + lane];
                inp[0][r][SS_XO + 32 + lane] = fmaf(u.x, u.x, u.y * u.y);
            }
        }
        __syncthreads();
    }
    // row sums of the pairs (x, y) and (x^2 + y^2, x y)
    ssim_rows<2, 2, 0>(inp, h, nullptr, [](const float (&a)[2], float2 (&v2)[2], float (&)[1]) {
        v2[0] = make_float2(a[0], a[1]);
        v2[1] = make_float2(fmaf(a[0], a[0], a[1] * a[1]), a[0] * a[1]);
    });
    __syncthreads();
    float2 mu[2][SS_ROWS];
    float unused[1][SS_ROWS];
    ssim_cols<2, 0>(h, nullptr, col, row0, mu, unused);
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < SS_ROWS; k++) {
        const int gy = blockIdx.y * SS_TH + row0 + k;
        if (gx >= W || gy >= H) continue;
        const float mx = mu[0][k].x, my = mu[0][k].y, m2 = mu[1][k].x, mxy = mu[1][k].y;
        const float c = fmaf(mx, mx, fmaf(my, my, SS_C1));
        const float a = fmaf(2.f * mx, my, SS_C1);
        const float b = 2.f * (mxy - mx * my) + SS_C2;
        const float d = m2 - mx * mx - my * my + SS_C2;
        const float icd = __frcp_rn(c * d);
        const float S = a * b * icd;
        const float Sc = S * d * icd, Sd = S * c * icd;  // S / c, S / d
        const size_t p = (size_t)img * HW + (size_t)gy * W + gx;
        dmap[p] = 2.f * my * (b - a) * icd + 2.f * mx * (Sd - Sc);
        dmap[n + p] = -Sd;
        dmap[2 * n + p] = 2.f * a * icd;
        const float xv = inp[0][row0 + k + SS_R][SS_XO + SS_R + col];
        const float yv = inp[1][row0 + k + SS_R][SS_XO + SS_R + col];
        if constexpr (FROM_FIELD) I[p] = xv;
        const float dl = xv - yv;
        const float w = plain ? 1.f : 1.f + mv[k] + yv * yv;
        acc += dl * dl * w + lam * (1.f - S);
    }
    const float s = block_sum(acc, red);
    if (threadIdx.x == 0) partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

// Pass 2: g = dL/dI = (2 d w - lambda (G dmap0 + 2 I G dmap1 + I_gt G dmap2)) / n,
// written to gI, or (TO_FIELD) turned into dL/dV = 2 g V in place over V.
template <bool TO_FIELD, bool VEC>
__global__ void __launch_bounds__(SS_NT)
    k_ssim_grad(const float* __restrict__ I, const float* __restrict__ Igt, const float* __restrict__ M, int C,
                int H, int W, float lam, int plain, float inv_n, const float* __restrict__ dmap,
                float* __restrict__ gI, float2* __restrict__ V, const __grid_constant__ SsimMaps maps, int* status) {
    __shared__ __align__(128) float inp[3][SS_EH][SS_XW];
    __shared__ __align__(16) float2 h2[1][SS_EH][SS_TW];
    __shared__ __align__(16) float h1[1][SS_EH][SS_TW];
    __shared__ __align__(8) uint64_t bar;
    const int img = blockIdx.z;
    const size_t HW = (size_t)H * W, n = (size_t)gridDim.z * HW;
    const int xs = blockIdx.x * SS_TW - SS_R - SS_XO, y0 = blockIdx.y * SS_TH - SS_R;
    const float* d0 = dmap + (size_t)img * HW;
    const float* d1 = d0 + n;
    const float* d2 = d1 + n;
    if constexpr (VEC) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            mbar_init_fence();
            mbar_expect_tx(&bar, 3 * SS_EH * SS_XW * sizeof(float));
#pragma unroll
            for (int q = 0; q < 3; q++) tma_load_4d(&inp[q][0][0], &maps.a, xs, y0, img, q, &bar);
        }
        __syncthreads();  // the barrier is initialised before anyone waits on it
    } else {
        halo_copy<VEC, 4>(xs, y0, H, W, [&](int r, int c, unsigned off, bool ok, int bytes) {
            cp_async_n(&inp[0][r][c], d0 + off, ok, bytes);
            cp_async_n(&inp[1][r][c], d1 + off, ok, bytes);
            cp_async_n(&inp[2][r][c], d2 + off, ok, bytes);
        });
    }
    // the thread's own I, I_gt, M for the epilogue, loaded meanwhile
    const int col = threadIdx.x & 31, row0 = (threadIdx.x >> 5) * SS_ROWS;
    const float* m = M ? M + (size_t)(img / C) * HW : nullptr;
    const int gx = blockIdx.x * SS_TW + col;
    float xo[SS_ROWS], yo[SS_ROWS], mv[SS_ROWS];
    float2 vo[TO_FIELD ? SS_ROWS : 1];
#pragma unroll
    for (int k = 0; k < SS_ROWS; k++) {
        const int gy = blockIdx.y * SS_TH + row0 + k;
        const bool in = gx < W && gy < H;
        const size_t p = (size_t)img * HW + (size_t)gy * W + gx;
        xo[k] = in ? I[p] : 0.f;
        yo[k] = in ? Igt[p] : 0.f;
        mv[k] = (m && in) ? m[(size_t)gy * W + gx] : 0.f;
        if constexpr (TO_FIELD) vo[k] = in ? V[p] : make_float2(0.f, 0.f);
    }
    if constexpr (VEC) {
        if (!tma_tiles_ready(&bar, status)) return;
    } else {
        cp_async_wait_all();
        __syncthreads();
    }
    ssim_rows<3, 1, 1>(inp, h2, h1, [](const float (&a)[3], float2 (&v2)[1], float (&v1)[1]) {
        v2[0] = make_float2(a[0], a[1]);
        v1[0] = a[2];
    });
    __syncthreads();
    float2 g01[1][SS_ROWS];
    float g2[1][SS_ROWS];
    ssim_cols<1, 1>(h2, h1, col, row0, g01, g2);
#pragma unroll
    for (int k = 0; k < SS_ROWS; k++) {
        const int gy = blockIdx.y * SS_TH + row0 + k;
        if (gx >= W || gy >= H) continue;
        const size_t p = (size_t)img * HW + (size_t)gy * W + gx;
        const float xv = xo[k], yv = yo[k];
        const float w = plain ? 1.f : 1.f + mv[k] + yv * yv;
        const float g = inv_n * (2.f * (xv - yv) * w - lam * (g01[0][k].x + 2.f * xv * g01[0][k].y + yv * g2[0][k]));
        if constexpr (TO_FIELD) {
            const float2 v = vo[TO_FIELD ? k : 0];
            V[p] = make_float2(2.f * g * v.x, 2.f * g * v.y);
        } else {
            gI[p] = g;
        }
    }
}

// Tensor map of `planes` stacked images of H x W elements (es = 4 or 8 bytes)
// at `base`: dims (W, H, nimg[, planes]), box SS_XW x SS_EH, zeros outside.
// Rows must be 16-byte aligned (W es a multiple of 16).  The driver's encoder
// is looked up once through the runtime.
static bool encode_halo_map(CUtensorMap* m, const void* base, int es, int W, int H, uint64_t nimg, int planes) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    if (!encode) return false;
    const int rank = planes > 1 ? 4 : 3;
    const cuuint64_t dims[4] = {(cuuint64_t)W, (cuuint64_t)H, nimg, (cuuint64_t)planes};
    const cuuint64_t strides[3] = {(cuuint64_t)W * es, (cuuint64_t)H * W * es, nimg * H * W * es};
    const cuuint32_t box[4] = {SS_XW, SS_EH, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return encode(m, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Loss partials and gradient of L_recon + L_SSIM for B L C images of H x W.
// V != nullptr: intensities |V|^2 (written to I), gradient dL/dV over V;
// otherwise intensities read from I and dL/dI written to gI.  plain = 1: the
// squared error carries weight 1 (no mask or target weighting).  dmap holds
// 3 B L C H W floats; partials one float per block (query with partials = NULL).
hcgs_status ssim_recon_loss(hcgs_ctx* ctx, float2* V, float* I, const float* Igt, const float* M, int B, int L,
                            int C, int H, int W, float lam, float* dmap, float* partials, int* nblocks_out,
                            float* gI, cudaStream_t st, int plain) {
    const dim3 grid((W + SS_TW - 1) / SS_TW, (H + SS_TH - 1) / SS_TH, B * L * C);
    *nblocks_out = (int)(grid.x * grid.y * grid.z);
    if (!partials) return HCGS_OK;  // size query
    HCGS_CUDA(ctx, ssim_window_upload());
    const int blk = SS_NT;
    const float inv_n = (float)(1.0 / ((double)B * L * C * H * W));
    // tensor copies need 16-byte aligned rows: W a multiple of 4 and aligned bases
    auto al = [](const void* q) { return q == nullptr || ((uintptr_t)q & 15) == 0; };
    bool vec = W % 4 == 0 && al(V) && al(I) && al(Igt) && al(dmap);
    SsimMaps m1{}, m2{};
    if (vec) {
        const uint64_t nimg = (uint64_t)B * L * C;
        const bool ok = encode_halo_map(&m1.a, V ? (const void*)V : (const void*)I, V ? 8 : 4, W, H, nimg, 1) &&
                        encode_halo_map(&m1.b, Igt, 4, W, H, nimg, 1) && encode_halo_map(&m2.a, dmap, 4, W, H, nimg, 3);
        if (!ok) vec = false;  // driver without the entry point: element copies
    }
#define HCGS_SSIM_LAUNCH(F, VEC)                                                                              \
    do {                                                                                                      \
        HCGS_KERNEL(ctx, "k_ssim_partials", st,                                                               \
                    (k_ssim_partials<F, VEC><<<grid, blk, 0, st>>>(V, I, Igt, M, C, H, W, lam, plain, dmap, partials, \
                                                                   m1, ctx->d_status)));                      \
        HCGS_KERNEL(ctx, "k_ssim_grad", st,                                                                   \
                    (k_ssim_grad<F, VEC><<<grid, blk, 0, st>>>(I, Igt, M, C, H, W, lam, plain, inv_n, dmap,     \
                                                               F ? nullptr : gI, F ? V : nullptr, m2,         \
                                                               ctx->d_status)));                              \
    } while (0)
    if (V && vec)
        HCGS_SSIM_LAUNCH(true, true);
    else if (V)
        HCGS_SSIM_LAUNCH(true, false);
    else if (vec)
        HCGS_SSIM_LAUNCH(false, true);
    else
        HCGS_SSIM_LAUNCH(false, false);
#undef HCGS_SSIM_LAUNCH
    return HCGS_OK;
}

// The plain focal-stack loss on a propagated field (the zero-padded route,
// where the inverse propagation is not fused with the loss): I = |V|^2,
// block partials of sum (I - I_gt)^2, and dL/dV = (4/n)(I - I_gt) V in place.
__global__ void k_focal_field(float2* __restrict__ V, const float* __restrict__ Igt, float* __restrict__ Iout,
                              int64_t n, float g4n, float* __restrict__ partials) {
    __shared__ float red[8];
    float acc = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = V[i];
        const float I = fmaf(v.x, v.x, v.y * v.y);
        const float d = I - Igt[i];
        if (Iout) Iout[i] = I;
        acc = fmaf(d, d, acc);
        V[i] = make_float2(g4n * d * v.x, g4n * d * v.y);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        partials[blockIdx.x] = t;
    }
}

int focal_field_blocks(int64_t n) { return (int)std::min<int64_t>(148 * 8, (n + 255) / 256); }

hcgs_status focal_field(hcgs_ctx* ctx, float2* V, const float* Igt, float* Iout, int64_t n, float* partials,
                        cudaStream_t st) {
    const float g4n = (float)(4.0 / (double)n);
    HCGS_KERNEL(ctx, "k_focal_field", st,
                k_focal_field<<<focal_field_blocks(n), 256, 0, st>>>(V, Igt, Iout, n, g4n, partials));
    return HCGS_OK;
}

// Phase-only conversion pieces: e^{j phi}; the real and imaginary parts of a
// field as two planes (part-major) and back; dL/dphi = Im(conj(e^{j phi}) g)
// for g = dL/dRe + j dL/dIm of e^{j phi}; the phase of a complex hologram.
__global__ void k_phasor(const float* __restrict__ phi, float2* __restrict__ P, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float s, c;
        sincosf(phi[i], &s, &c);
        P[i] = make_float2(c, s);
    }
}

__global__ void k_split_parts(const float2* __restrict__ U, float* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 u = U[i];
        out[i] = u.x;
        out[n + i] = u.y;
    }
}

__global__ void k_merge_parts(const float* __restrict__ g, float2* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = make_float2(g[i], g[n + i]);
}

__global__ void k_phase_grad(const float* __restrict__ phi, const float2* __restrict__ gP, float* __restrict__ gphi,
                             int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float s, c;
        sincosf(phi[i], &s, &c);
        const float2 g = gP[i];
        gphi[i] = c * g.y - s * g.x;
    }
}

__global__ void k_scale(const float* __restrict__ x, float s, float* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = s * x[i];
}

__global__ void k_phase_of(const float2* __restrict__ P, float* __restrict__ phi, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 p = P[i];
        phi[i] = atan2f(p.y, p.x);
    }
}

static int ew_blocks(int64_t n) { return (int)std::min<int64_t>(148 * 16, (n + 255) / 256); }

hcgs_status phasor(hcgs_ctx* ctx, const float* phi, float2* P, int64_t n, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_phasor", st, k_phasor<<<ew_blocks(n), 256, 0, st>>>(phi, P, n));
    return HCGS_OK;
}
hcgs_status split_parts(hcgs_ctx* ctx, const float2* U, float* out, int64_t n, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_split_parts", st, k_split_parts<<<ew_blocks(n), 256, 0, st>>>(U, out, n));
    return HCGS_OK;
}
hcgs_status merge_parts(hcgs_ctx* ctx, const float* g, float2* out, int64_t n, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_merge_parts", st, k_merge_parts<<<ew_blocks(n), 256, 0, st>>>(g, out, n));
    return HCGS_OK;
}
hcgs_status phase_grad(hcgs_ctx* ctx, const float* phi, const float2* gP, float* gphi, int64_t n, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_phase_grad", st, k_phase_grad<<<ew_blocks(n), 256, 0, st>>>(phi, gP, gphi, n));
    return HCGS_OK;
}
hcgs_status scale(hcgs_ctx* ctx, const float* x, float s, float* out, int64_t n, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_scale", st, k_scale<<<ew_blocks(n), 256, 0, st>>>(x, s, out, n));
    return HCGS_OK;
}
hcgs_status phase_of(hcgs_ctx* ctx, const float2* P, float* phi, int64_t n, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_phase_of", st, k_phase_of<<<ew_blocks(n), 256, 0, st>>>(P, phi, n));
    return HCGS_OK;
}

// ---------------------------------------------------------------------------
// Adan (Xie et al., Algorithm 1), decay-factor form: first step m = g, v = 0,
// n = g^2; second step v = g - g_prev; then the moving averages
//   m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2)(g - g_prev),
//   n <- b3 n + (1 - b3)(g + b2 (g - g_prev))^2;
// p <- (p - lr (m + b2 v) / (sqrt(n) + eps)) / (1 + wd lr); g_prev <- g.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void adan_elem(float* __restrict__ p, const float* __restrict__ g,
                                          float* __restrict__ gp, float* __restrict__ m, float* __restrict__ v,
                                          float* __restrict__ nn, int64_t i, int step, float lr, float b1,
                                          float b2, float b3, float eps, float shrink) {
    const float gi = g[i];
    float mi, vi, ni;
    if (step == 1) {
        mi = gi;
        vi = 0.f;
        ni = gi * gi;
    } else {
        const float dg = gi - gp[i];
        mi = fmaf(b1, m[i], (1.f - b1) * gi);
        vi = step == 2 ? dg : fmaf(b2, v[i], (1.f - b2) * dg);
        const float u = fmaf(b2, dg, gi);
        ni = fmaf(b3, nn[i], (1.f - b3) * u * u);
    }
    m[i] = mi;
    v[i] = vi;
    nn[i] = ni;
    gp[i] = gi;
    p[i] = (p[i] - lr * fmaf(b2, vi, mi) / (sqrtf(ni) + eps)) * shrink;
}

__global__ void k_adan(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ gp,
                       float* __restrict__ m, float* __restrict__ v, float* __restrict__ nn, int64_t count,
                       int step, float lr, float b1, float b2, float b3, float eps, float wd) {
    const float shrink = 1.f / (1.f + wd * lr);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        adan_elem(p, g, gp, m, v, nn, i, step, lr, b1, b2, b3, eps, shrink);
}

// Several parameter arrays in one launch (block layout as k_adam_multi; the
// arithmetic is adan_elem's, so the result equals one k_adan per array).
__global__ void __launch_bounds__(OPT_THREADS) k_adan_multi(OptArrays A, int step, float b1, float b2, float b3,
                                                            float eps, float wd) {
    int a = 0;
    while (a + 1 < A.k && (int64_t)blockIdx.x >= A.first[a + 1]) a++;
    const float lr = A.lr[a];
    const float shrink = 1.f / (1.f + wd * lr);
    const int64_t base = ((int64_t)blockIdx.x - A.first[a]) * OPT_EPB;
    for (int e = threadIdx.x; e < OPT_EPB; e += OPT_THREADS) {
        const int64_t i = base + e;
        if (i < A.count[a])
            adan_elem(A.p[a], A.g[a], A.gp[a], A.m[a], A.v[a], A.n[a], i, step, lr, b1, b2, b3, eps, shrink);
    }
}

hcgs_status adan_multi(hcgs_ctx* ctx, OptArrays& A, int step, float b1, float b2, float b3, float eps, float wd,
                       cudaStream_t st) {
    const int64_t blocks = opt_blocks(A);
    if (blocks == 0) return HCGS_OK;
    HCGS_KERNEL(ctx, "k_adan", st,
                k_adan_multi<<<(unsigned)blocks, OPT_THREADS, 0, st>>>(A, step, b1, b2, b3, eps, wd));
    return HCGS_OK;
}

hcgs_status adan(hcgs_ctx* ctx, float* p, const float* g, float* gp, float* m, float* v, float* n, int64_t count,
                 int step, float lr, float b1, float b2, float b3, float eps, float wd, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>(148 * 16, (count + 255) / 256);
    HCGS_KERNEL(ctx, "k_adan", st, k_adan<<<blocks, 256, 0, st>>>(p, g, gp, m, v, n, count, step, lr, b1, b2, b3, eps, wd));
    return HCGS_OK;
}

}  // namespace hcgs
