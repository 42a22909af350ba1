// Learned-initialisation network (no counterpart in the paper): a 4-layer
// ReLU MLP 16 -> 128 -> 128 -> 128 -> 16 with BF16 operands and FP32
// accumulation on the tensor cores (mma.m16n8k16), forward and reverse mode.
//
// Forward: each warp owns 16 rows; activations stay in shared memory as BF16;
// weights are read as B fragments through L1.  Reverse mode: a CTA owns 128
// rows, recomputes the forward into shared memory, then per layer computes
// the bias and weight gradients over its 128 rows (weight gradient = a
// tensor-core product with k = 128 rows, added once per CTA) and the input
// gradient of the next layer down.
#include "common.cuh"

namespace hcgs {

constexpr int MLP_IN = 16, MLP_HID = 128, MLP_OUT = 16;
constexpr int LDI = MLP_IN + 8;    // padded row strides (bf16 elements) against bank conflicts
constexpr int LDH = MLP_HID + 8;

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint16_t f2bf(float x) {
    // round to nearest even
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);  // NaN stays NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }
__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

// A fragment of a row-major 16 x 16 block at X (leading dimension ld).
__device__ __forceinline__ void frag_a(uint32_t* a, const uint16_t* X, int ld, int k0, int gid, int tig) {
    a[0] = ld32(X + gid * ld + k0 + 2 * tig);
    a[1] = ld32(X + (gid + 8) * ld + k0 + 2 * tig);
    a[2] = ld32(X + gid * ld + k0 + 8 + 2 * tig);
    a[3] = ld32(X + (gid + 8) * ld + k0 + 8 + 2 * tig);
}
// B fragment for y = x W^T with W row-major [nout][K]: B(k, n) = W[n0 + n][k0 + k].
__device__ __forceinline__ void frag_b(uint32_t* b, const uint16_t* W, int K, int n0, int k0, int gid, int tig) {
    b[0] = __ldg(reinterpret_cast<const unsigned int*>(W + (size_t)(n0 + gid) * K + k0 + 2 * tig));
    b[1] = __ldg(reinterpret_cast<const unsigned int*>(W + (size_t)(n0 + gid) * K + k0 + 8 + 2 * tig));
}

// One layer for the warp's 16 rows: Y = act(X W^T + b), Y as BF16 in smem.
template <int K, int NOUT, bool RELU>
__device__ __forceinline__ void layer_smem(const uint16_t* X, int ldx, const uint16_t* W, const float* bias,
                                           uint16_t* Y, int ldy, int gid, int tig) {
#pragma unroll 2
    for (int nt = 0; nt < NOUT / 8; nt++) {
        const int n0 = nt * 8;
        const float b0 = bias[n0 + 2 * tig], b1 = bias[n0 + 2 * tig + 1];
        float d[4] = {b0, b1, b0, b1};
#pragma unroll
        for (int kt = 0; kt < K / 16; kt++) {
            uint32_t a[4], b[2];
            frag_a(a, X, ldx, kt * 16, gid, tig);
            frag_b(b, W, K, n0, kt * 16, gid, tig);
            mma16816(d, a, b);
        }
        if (RELU)
            for (int e = 0; e < 4; e++) d[e] = fmaxf(d[e], 0.f);
        *reinterpret_cast<uint32_t*>(Y + gid * ldy + n0 + 2 * tig) = pack2(f2bf(d[0]), f2bf(d[1]));
        *reinterpret_cast<uint32_t*>(Y + (gid + 8) * ldy + n0 + 2 * tig) = pack2(f2bf(d[2]), f2bf(d[3]));
    }
}

__device__ __forceinline__ void load_x(uint16_t* xs, const uint16_t* x, int row0, int N, int lane) {
    for (int e = lane; e < 16 * MLP_IN; e += 32) {
        const int r = e / MLP_IN, c = e % MLP_IN;
        xs[r * LDI + c] = row0 + r < N ? x[(size_t)(row0 + r) * MLP_IN + c] : (uint16_t)0;
    }
    __syncwarp();
}

struct MlpW {
    const uint16_t *W1, *W2, *W3, *W4;
    const float *b1, *b2, *b3, *b4;
};

constexpr size_t MLP_FWD_SMEM = (size_t)8 * 16 * (LDI + 2 * LDH) * sizeof(uint16_t);

__global__ void __launch_bounds__(256) k_mlp_fwd(MlpW w, const uint16_t* __restrict__ x, int N,
                                                 float* __restrict__ y) {
    extern __shared__ __align__(16) uint16_t fsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    uint16_t* sx = fsm + warp * 16 * (LDI + 2 * LDH);
    uint16_t* sa = sx + 16 * LDI;
    uint16_t* sb = sa + 16 * LDH;
    const int row0 = (blockIdx.x * 8 + warp) * 16;
    if (row0 >= N) return;
    load_x(sx, x, row0, N, lane);
    layer_smem<MLP_IN, MLP_HID, true>(sx, LDI, w.W1, w.b1, sa, LDH, gid, tig);
    __syncwarp();
    layer_smem<MLP_HID, MLP_HID, true>(sa, LDH, w.W2, w.b2, sb, LDH, gid, tig);
    __syncwarp();
    layer_smem<MLP_HID, MLP_HID, true>(sb, LDH, w.W3, w.b3, sa, LDH, gid, tig);
    __syncwarp();
    // output layer, FP32
    for (int nt = 0; nt < MLP_OUT / 8; nt++) {
        const int n0 = nt * 8;
        const float b0 = w.b4[n0 + 2 * tig], b1 = w.b4[n0 + 2 * tig + 1];
        float d[4] = {b0, b1, b0, b1};
#pragma unroll
        for (int kt = 0; kt < MLP_HID / 16; kt++) {
            uint32_t a[4], b[2];
            frag_a(a, sa, LDH, kt * 16, gid, tig);
            frag_b(b, w.W4, MLP_HID, n0, kt * 16, gid, tig);
            mma16816(d, a, b);
        }
        const int r0 = row0 + gid, r1 = row0 + gid + 8;
        if (r0 < N) { y[(size_t)r0 * MLP_OUT + n0 + 2 * tig] = d[0]; y[(size_t)r0 * MLP_OUT + n0 + 2 * tig + 1] = d[1]; }
        if (r1 < N) { y[(size_t)r1 * MLP_OUT + n0 + 2 * tig] = d[2]; y[(size_t)r1 * MLP_OUT + n0 + 2 * tig + 1] = d[3]; }
    }
}

// W [rows][cols] -> Wt [cols][rows] (bf16)
__global__ void k_transpose_bf16(const uint16_t* __restrict__ W, uint16_t* __restrict__ Wt, int rows, int cols) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int r = i / cols, c = i % cols;
    Wt[(size_t)c * rows + r] = W[i];
}

// CTA-level weight gradient over 128 rows: gW[o][i] += sum_r gZ[r][o] X[r][i].
// gZ: smem [128][ldz] bf16, X: smem [128][ldx] bf16.
template <int NOUT, int K>
__device__ void weight_grad(const uint16_t* gZ, int ldz, const uint16_t* X, int ldx, float* gW, int warp, int gid,
                            int tig) {
    constexpr int MT = NOUT / 16, NT = K / 8;
    for (int p = warp; p < MT * NT; p += 8) {
        const int m0 = (p / NT) * 16, n0 = (p % NT) * 8;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
        for (int k0 = 0; k0 < 128; k0 += 16) {
            uint32_t a[4], b[2];
            // A(m, k) = gZ[k0 + k][m0 + m]
            a[0] = pack2(gZ[(k0 + 2 * tig) * ldz + m0 + gid], gZ[(k0 + 2 * tig + 1) * ldz + m0 + gid]);
            a[1] = pack2(gZ[(k0 + 2 * tig) * ldz + m0 + gid + 8], gZ[(k0 + 2 * tig + 1) * ldz + m0 + gid + 8]);
            a[2] = pack2(gZ[(k0 + 2 * tig + 8) * ldz + m0 + gid], gZ[(k0 + 2 * tig + 9) * ldz + m0 + gid]);
            a[3] = pack2(gZ[(k0 + 2 * tig + 8) * ldz + m0 + gid + 8], gZ[(k0 + 2 * tig + 9) * ldz + m0 + gid + 8]);
            // B(k, n) = X[k0 + k][n0 + n]
            b[0] = pack2(X[(k0 + 2 * tig) * ldx + n0 + gid], X[(k0 + 2 * tig + 1) * ldx + n0 + gid]);
            b[1] = pack2(X[(k0 + 2 * tig + 8) * ldx + n0 + gid], X[(k0 + 2 * tig + 9) * ldx + n0 + gid]);
            mma16816(d, a, b);
        }
        atomicAdd(gW + (m0 + gid) * K + n0 + 2 * tig, d[0]);
        atomicAdd(gW + (m0 + gid) * K + n0 + 2 * tig + 1, d[1]);
        atomicAdd(gW + (m0 + gid + 8) * K + n0 + 2 * tig, d[2]);
        atomicAdd(gW + (m0 + gid + 8) * K + n0 + 2 * tig + 1, d[3]);
    }
}

// Column sums of gZ[128][ldz] (first NOUT columns) into gb.
template <int NOUT>
__device__ void bias_grad(const uint16_t* gZ, int ldz, float* gb, int rows) {
    for (int c = threadIdx.x; c < NOUT; c += blockDim.x) {
        float s = 0.f;
        for (int r = 0; r < rows; r++) s += bf2f(gZ[r * ldz + c]);
        atomicAdd(gb + c, s);
    }
}

// Input gradient for the warp's 16 rows: gX = (gZ W) masked by (H > 0),
// written as BF16.  Wt is W transposed: [K][NOUT] row-major.
template <int NOUT, int K>
__device__ __forceinline__ void input_grad(const uint16_t* gZ, int ldz, const uint16_t* Wt, const uint16_t* Hm,
                                           int ldh, uint16_t* gX, int ldg, int gid, int tig) {
    for (int nt = 0; nt < K / 8; nt++) {
        const int n0 = nt * 8;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < NOUT / 16; kt++) {
            uint32_t a[4], b[2];
            frag_a(a, gZ, ldz, kt * 16, gid, tig);
            frag_b(b, Wt, NOUT, n0, kt * 16, gid, tig);
            mma16816(d, a, b);
        }
        const int c = n0 + 2 * tig;
        const float m0 = bf2f(Hm[gid * ldh + c]) > 0.f ? 1.f : 0.f, m1 = bf2f(Hm[gid * ldh + c + 1]) > 0.f ? 1.f : 0.f;
        const float m2 = bf2f(Hm[(gid + 8) * ldh + c]) > 0.f ? 1.f : 0.f, m3 = bf2f(Hm[(gid + 8) * ldh + c + 1]) > 0.f ? 1.f : 0.f;
        *reinterpret_cast<uint32_t*>(gX + gid * ldg + c) = pack2(f2bf(d[0] * m0), f2bf(d[1] * m1));
        *reinterpret_cast<uint32_t*>(gX + (gid + 8) * ldg + c) = pack2(f2bf(d[2] * m2), f2bf(d[3] * m3));
    }
}

struct MlpG {
    float *gW1, *gW2, *gW3, *gW4, *gb1, *gb2, *gb3, *gb4;
    const uint16_t *W2t, *W3t, *W4t;
};

constexpr size_t MLP_BWD_SMEM = (size_t)128 * (LDI + 3 * LDH + LDH + LDI) * sizeof(uint16_t);

__global__ void __launch_bounds__(256) k_mlp_bwd(MlpW w, MlpG g, const uint16_t* __restrict__ x, int N,
                                                 const float* __restrict__ gy) {
    extern __shared__ __align__(16) uint16_t smem[];
    uint16_t* sx = smem;                    // [128][LDI]
    uint16_t* h1 = sx + 128 * LDI;          // [128][LDH]
    uint16_t* h2 = h1 + 128 * LDH;
    uint16_t* h3 = h2 + 128 * LDH;
    uint16_t* gz = h3 + 128 * LDH;          // [128][LDH] current layer's dL/dZ
    uint16_t* gz4 = gz + 128 * LDH;         // [128][LDI] output layer's dL/dZ
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int row0 = blockIdx.x * 128 + warp * 16;
    const int rows = min(128, N - (int)blockIdx.x * 128);
    // forward recompute for this warp's rows
    load_x(sx + warp * 16 * LDI, x, row0, N, lane);
    layer_smem<MLP_IN, MLP_HID, true>(sx + warp * 16 * LDI, LDI, w.W1, w.b1, h1 + warp * 16 * LDH, LDH, gid, tig);
    __syncwarp();
    layer_smem<MLP_HID, MLP_HID, true>(h1 + warp * 16 * LDH, LDH, w.W2, w.b2, h2 + warp * 16 * LDH, LDH, gid, tig);
    __syncwarp();
    layer_smem<MLP_HID, MLP_HID, true>(h2 + warp * 16 * LDH, LDH, w.W3, w.b3, h3 + warp * 16 * LDH, LDH, gid, tig);
    // output-layer gradient (rows past N are zero)
    for (int e = lane; e < 16 * MLP_OUT; e += 32) {
        const int r = e / MLP_OUT, c = e % MLP_OUT;
        gz4[(warp * 16 + r) * LDI + c] = row0 + r < N ? f2bf(gy[(size_t)(row0 + r) * MLP_OUT + c]) : (uint16_t)0;
    }
    __syncthreads();
    // layer 4
    bias_grad<MLP_OUT>(gz4, LDI, g.gb4, rows);
    weight_grad<MLP_OUT, MLP_HID>(gz4, LDI, h3, LDH, g.gW4, warp, gid, tig);
    input_grad<MLP_OUT, MLP_HID>(gz4 + warp * 16 * LDI, LDI, g.W4t, h3 + warp * 16 * LDH, LDH, gz + warp * 16 * LDH,
                                 LDH, gid, tig);
    __syncthreads();
    // layer 3
    bias_grad<MLP_HID>(gz, LDH, g.gb3, rows);
    weight_grad<MLP_HID, MLP_HID>(gz, LDH, h2, LDH, g.gW3, warp, gid, tig);
    __syncthreads();
    // gz (layer 3) -> gz (layer 2): compute into h3's space, which is no longer needed
    input_grad<MLP_HID, MLP_HID>(gz + warp * 16 * LDH, LDH, g.W3t, h2 + warp * 16 * LDH, LDH, h3 + warp * 16 * LDH,
                                 LDH, gid, tig);
    __syncthreads();
    uint16_t* gz2 = h3;
    bias_grad<MLP_HID>(gz2, LDH, g.gb2, rows);
    weight_grad<MLP_HID, MLP_HID>(gz2, LDH, h1, LDH, g.gW2, warp, gid, tig);
    __syncthreads();
    input_grad<MLP_HID, MLP_HID>(gz2 + warp * 16 * LDH, LDH, g.W2t, h1 + warp * 16 * LDH, LDH, gz + warp * 16 * LDH,
                                 LDH, gid, tig);
    __syncthreads();
    bias_grad<MLP_HID>(gz, LDH, g.gb1, rows);
    weight_grad<MLP_HID, MLP_IN>(gz, LDH, sx, LDI, g.gW1, warp, gid, tig);
}

// Mean squared error of the first K of the 16 output columns against
// target[N][16]; gy = dL/dy (zero in the unused columns).  Per-block partial
// sums, reduced in a fixed order by k_reduce_sum.
__global__ void k_mlp_mse(const float* __restrict__ y, const float* __restrict__ tgt, int N, int K, float scale,
                          float* __restrict__ gy, float* __restrict__ partials) {
    __shared__ float red[32];
    float part = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * MLP_OUT; i += gridDim.x * blockDim.x) {
        const int c = i % MLP_OUT;
        float g = 0.f;
        if (c < K) {
            const float d = y[i] - tgt[i];
            part += d * d;
            g = 2.f * scale * d;
        }
        gy[i] = g;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// round-to-nearest-even float32 -> bfloat16
__global__ void k_cast_bf16(const float* __restrict__ src, uint16_t* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = f2bf(src[i]);
}

hcgs_status mlp_mse(hcgs_ctx* ctx, const float* y, const float* tgt, int N, int K, float* loss, float* gy,
                    cudaStream_t st) {
    const int blocks = 296;
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[5], blocks * sizeof(float), &ctx->bytes));
    const float scale = 1.f / ((float)N * (float)K);
    HCGS_KERNEL(ctx, "k_mlp_mse", st, k_mlp_mse<<<blocks, 256, 0, st>>>(y, tgt, N, K, scale, gy, (float*)ctx->ws[5].p));
    return reduce_sum(ctx, (const float*)ctx->ws[5].p, blocks, scale, loss, st);
}

hcgs_status cast_bf16(hcgs_ctx* ctx, const float* src, uint16_t* dst, int64_t n, cudaStream_t st) {
    if (n <= 0) return HCGS_OK;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 8) blocks = 148 * 8;
    HCGS_KERNEL(ctx, "k_cast_bf16", st, k_cast_bf16<<<(unsigned)blocks, 256, 0, st>>>(src, dst, n));
    return HCGS_OK;
}

static MlpW make_w(const uint16_t* const* W, const float* const* b) {
    MlpW w;
    w.W1 = W[0]; w.W2 = W[1]; w.W3 = W[2]; w.W4 = W[3];
    w.b1 = b[0]; w.b2 = b[1]; w.b3 = b[2]; w.b4 = b[3];
    return w;
}

hcgs_status mlp_fwd(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* const* W, const float* const* b,
                    float* y, cudaStream_t st) {
    const int rows_per_cta = 128;
    HCGS_CUDA(ctx, cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_FWD_SMEM));
    HCGS_KERNEL(ctx, "k_mlp_fwd", st, k_mlp_fwd<<<(N + rows_per_cta - 1) / rows_per_cta, 256, MLP_FWD_SMEM, st>>>(make_w(W, b), x, N, y));
    HCGS_LAUNCH(ctx, "k_mlp_fwd");
    return HCGS_OK;
}

hcgs_status mlp_bwd(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* const* W, const float* const* b,
                    const float* gy, float* const* gW, float* const* gb, cudaStream_t st) {
    const size_t nW[4] = {(size_t)MLP_HID * MLP_IN, (size_t)MLP_HID * MLP_HID, (size_t)MLP_HID * MLP_HID,
                          (size_t)MLP_OUT * MLP_HID};
    const size_t nb[4] = {MLP_HID, MLP_HID, MLP_HID, MLP_OUT};
    for (int k = 0; k < 4; k++) {
        HCGS_CUDA(ctx, cudaMemsetAsync(gW[k], 0, nW[k] * sizeof(float), st));
        HCGS_CUDA(ctx, cudaMemsetAsync(gb[k], 0, nb[k] * sizeof(float), st));
    }
    if (N == 0) return HCGS_OK;
    // transposed W2, W3, W4 for the input gradients
    const size_t nt = nW[1] + nW[2] + nW[3];
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[4], nt * sizeof(uint16_t), &ctx->bytes));
    uint16_t* W2t = (uint16_t*)ctx->ws[4].p;
    uint16_t* W3t = W2t + nW[1];
    uint16_t* W4t = W3t + nW[2];
    HCGS_KERNEL(ctx, "k_transpose_bf16", st, k_transpose_bf16<<<(int)((nW[1] + 255) / 256), 256, 0, st>>>(W[1], W2t, MLP_HID, MLP_HID));
    HCGS_KERNEL(ctx, "k_transpose_bf16", st, k_transpose_bf16<<<(int)((nW[2] + 255) / 256), 256, 0, st>>>(W[2], W3t, MLP_HID, MLP_HID));
    HCGS_KERNEL(ctx, "k_transpose_bf16", st, k_transpose_bf16<<<(int)((nW[3] + 255) / 256), 256, 0, st>>>(W[3], W4t, MLP_OUT, MLP_HID));
    HCGS_LAUNCH(ctx, "k_transpose_bf16");
    MlpG g;
    g.gW1 = gW[0]; g.gW2 = gW[1]; g.gW3 = gW[2]; g.gW4 = gW[3];
    g.gb1 = gb[0]; g.gb2 = gb[1]; g.gb3 = gb[2]; g.gb4 = gb[3];
    g.W2t = W2t; g.W3t = W3t; g.W4t = W4t;
    HCGS_CUDA(ctx, cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_BWD_SMEM));
    HCGS_KERNEL(ctx, "k_mlp_bwd", st, k_mlp_bwd<<<(N + 127) / 128, 256, MLP_BWD_SMEM, st>>>(make_w(W, b), g, x, N, gy));
    HCGS_LAUNCH(ctx, "k_mlp_bwd");
    return HCGS_OK;
}

}  // namespace hcgs
