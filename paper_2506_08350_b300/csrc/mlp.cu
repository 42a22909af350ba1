// Learned-initialisation network (no counterpart in the paper): a 4-layer
// ReLU MLP 16 -> 128 -> 128 -> 128 -> 16 with BF16 operands and FP32
// accumulation on the fifth-generation tensor cores (tcgen05.mma, kind::f16,
// accumulators in tensor memory), forward and reverse mode.
//
// Persistent CTAs over tiles of 128 rows, one per SM: the forward runs four
// warpgroups per CTA, each on its own tiles, the reverse mode one warpgroup;
// thread t of a warpgroup owns row t of its tile in every epilogue (TMEM lane
// t holds row t of an M = 128 accumulator).  The weights stay in shared memory
// for the CTA's lifetime, in core-matrix form: 8 x 8 blocks of BF16 (8 rows,
// 16 contiguous bytes each) that serve as K-major operands (features along K)
// and, read through the other descriptor mode, as MN-major operands (features
// along M or N), so one copy of W is both W^T in the forward and W in the
// input gradients.  One elected thread issues the MMAs and commits them to an
// mbarrier; every thread waits on it (bounded), reads its accumulator row
// with tcgen05.ld, applies bias / ReLU / the ReLU mask in FP32, rounds to
// BF16 and writes the next operand back to shared memory.
//
// Reverse mode recomputes the forward of the tile (the activations H1..H3
// stay in shared memory), then per layer l: the weight gradient
// dW_l += dZ_l^T H_{l-1} accumulates in TMEM over all tiles of the CTA (the
// bias gradient rides along as one extra column: H_{l-1} carries a block of
// ones, so that column is sum_rows dZ_l), and the input gradient dZ_l W_l,
// masked by the ReLU decisions kept from the forward, gives dZ_{l-1}.  At the
// end each CTA adds its accumulators to the outputs once.
#include <cuda_bf16.h>

#include "common.cuh"

namespace hcgs {

constexpr int MLP_IN = 16, MLP_HID = 128, MLP_OUT = 16;

__device__ __forceinline__ uint16_t f2bf(float x) {
    // round to nearest even
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);  // NaN stays NaN
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
// (lo, hi) -> packed bf16x2, round to nearest even
__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// ---- tcgen05 (inline PTX) ----
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {  // whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {  // whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// D[tmem] (+)= A B^T, A from descriptor a (M x 16), B from descriptor b (N x 16)
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// the mbarrier's phase completes once every MMA issued so far by this thread is done
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 (16) consecutive FP32 columns of this thread's TMEM lane from taddr
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    tc_wait_ld();
#pragma unroll
    for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
}
// 64 consecutive FP32 columns of this thread's TMEM lane from taddr (one
// round trip instead of two 32-column loads)
__device__ __forceinline__ void tc_ld64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
    tc_wait_ld();
#pragma unroll
    for (int j = 0; j < 64; j++) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    tc_wait_ld();
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// Core-matrix layout of an R x F BF16 matrix (F features per row, both
// multiples of 8): element (r, f) at byte ((r / 8) (F / 8) + f / 8) 128 +
// (r % 8) 16 + (f % 8) 2, i.e. 8-row groups, each a run of F / 8 blocks of
// 8 x 8 elements.
__host__ __device__ constexpr uint32_t cm_off(int r, int f, int F) {
    return (uint32_t)((((r >> 3) * (F >> 3) + (f >> 3)) << 7) + ((r & 7) << 4) + ((f & 7) << 1));
}
// Shared-memory matrix descriptor without swizzling: start address, the
// stride between core matrices along K (lbo) and along M / N (sbo), in bytes.
__device__ __forceinline__ uint64_t sm_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Operand views of a core-matrix buffer at saddr with F features, for the
// MMA's K-step s (16 elements of K):
//  K-major: rows along M / N, features along K (features 16 s .. 16 s + 15);
//  MN-major: features along M / N, rows along K (rows 16 s .. 16 s + 15).
__device__ __forceinline__ uint64_t op_k(uint32_t saddr, int F, int s) {
    return sm_desc(saddr + (uint32_t)s * 256u, 128u, (uint32_t)F * 16u);
}
__device__ __forceinline__ uint64_t op_mn(uint32_t saddr, int F, int s) {
    return sm_desc(saddr + (uint32_t)s * (uint32_t)F * 32u, (uint32_t)F * 16u, 128u);
}
// Instruction descriptor of kind::f16: BF16 A and B, FP32 D, M x N, each
// operand K-major (0) or MN-major (1).
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Copy an R x F row-major BF16 matrix (16-byte aligned rows) into core-matrix form.
__device__ __forceinline__ void load_cm(uint8_t* dst, const uint16_t* __restrict__ src, int R, int F) {
    const int chunks = R * (F >> 3);
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
        const int r = i / (F >> 3), j = i % (F >> 3);
        *reinterpret_cast<uint4*>(dst + cm_off(r, 8 * j, F)) =
            __ldg(reinterpret_cast<const uint4*>(src + (size_t)r * F + 8 * j));
    }
}

// Make the threads' shared-memory writes visible to the tensor cores and
// order everything before the next MMA issue.
__device__ __forceinline__ void sync_for_mma() {
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Bounded wait of every thread for the MMA phase; all threads agree on the
// outcome.  On a timeout the status word records it.
__device__ __forceinline__ bool wait_mma(uint64_t* bar, uint32_t& phase, int* status) {
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    const int bad = __syncthreads_or(!ok);
    if (bad && threadIdx.x == 0) atomicOr(status, STATUS_WAIT_TIMEOUT);
    tc_fence_after();
    return !bad;
}

// CH consecutive FP32 columns (32 or 64) of this thread's TMEM lane
template <int CH>
__device__ __forceinline__ void tc_ldn(uint32_t taddr, float (&v)[CH]) {
    if constexpr (CH == 64) tc_ld64(taddr, v);
    else tc_ld32(taddr, v);
}

// Hidden-layer epilogue of this thread's row: h = bf16(relu(z + b)) for the
// 128 accumulator columns at taddr, read CH at a time, written to the
// core-matrix buffer H (F features per row) at row r.  The bias is added in
// packed FP32, the ReLU taken on the rounded pair (rounding keeps the sign,
// so relu and rounding commute).
template <int CH = 64>
__device__ __forceinline__ void epi_hidden(uint32_t taddr, const float* b, uint8_t* H, int F, int r) {
    const __nv_bfloat162 zero = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll 1
    for (int c = 0; c < 128 / CH; c++) {
        float v[CH];
        tc_ldn<CH>(taddr + CH * c, v);
        const float2* bb = reinterpret_cast<const float2*>(b + CH * c);
        uint32_t p[CH / 2];
#pragma unroll
        for (int j = 0; j < CH / 2; j++) {
            const float2 z = __fadd2_rn(make_float2(v[2 * j], v[2 * j + 1]), bb[j]);
            __nv_bfloat162 h = __floats2bfloat162_rn(z.x, z.y);
            h = __hmax2(h, zero);
            p[j] = *reinterpret_cast<const uint32_t*>(&h);
        }
#pragma unroll
        for (int q = 0; q < CH / 8; q++)
            *reinterpret_cast<uint4*>(H + cm_off(r, CH * c + 8 * q, F)) =
                make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
    }
}

// Gradient epilogue: dZ = bf16(dH) where the layer's activation h (row r of
// Hl, F features) is positive, else 0, into G (128 features).
__device__ __forceinline__ void epi_grad(uint32_t taddr, const uint8_t* Hl, int F, uint8_t* G, int r) {
    const __nv_bfloat162 zero = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll 1
    for (int c = 0; c < 2; c++) {
        float v[64];
        tc_ld64(taddr + 64 * c, v);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint4 hw = *reinterpret_cast<const uint4*>(Hl + cm_off(r, 64 * c + 8 * q, F));
            const uint32_t hv[4] = {hw.x, hw.y, hw.z, hw.w};
            uint32_t p[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int j = 4 * q + k;
                const __nv_bfloat162 d = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                const uint32_t m = __hgt2_mask(*reinterpret_cast<const __nv_bfloat162*>(&hv[k]), zero);
                p[k] = *reinterpret_cast<const uint32_t*>(&d) & m;
            }
            *reinterpret_cast<uint4*>(G + cm_off(r, 64 * c + 8 * q, MLP_HID)) = make_uint4(p[0], p[1], p[2], p[3]);
        }
    }
}

struct MlpW {
    const uint16_t *W1, *W2, *W3, *W4;
    const float *b1, *b2, *b3, *b4;
};

// ---------------------------------------------------------------------------
// forward: y = W4 relu(W3 relu(W2 relu(W1 x + b1) + b2) + b3) + b4
// ---------------------------------------------------------------------------
// One CTA of F_WG warpgroups per SM.  The weights and biases are staged once
// per CTA and shared; each warpgroup runs its own stream of 128-row tiles
// with its own X and H tiles in shared memory, its own 128 TMEM columns
// (hidden accumulator; the 16 output columns reuse the first 16 of them once
// the last hidden epilogue has read them), its own mbarrier and its own named
// barrier.  While one warpgroup reads back and rounds an accumulator, the
// tensor cores run the MMAs the other warpgroups have issued, so the MMAs of
// a tile no longer wait for their own epilogues alone.
//
// shared memory (bytes): W1 [128][16], W2, W3 [128][128], W4 [16][128],
// biases, then per warpgroup the X tile [128][16] and the hidden tile
// [128][128] (reused by every layer), then the mbarriers and the TMEM slot.
constexpr int F_WG = 4;
constexpr int F_EPI = 32;  // accumulator columns per tcgen05.ld in the forward's epilogues
constexpr uint32_t FS_W1 = 0, FS_W2 = FS_W1 + 128 * 16 * 2, FS_W3 = FS_W2 + 128 * 128 * 2,
                   FS_W4 = FS_W3 + 128 * 128 * 2, FS_B = FS_W4 + 16 * 128 * 2,
                   FS_TILES = (FS_B + (3 * 128 + 16) * 4 + 1023) & ~1023u, FS_X = 0, FS_H = 128 * 16 * 2,
                   FS_WG = FS_H + 128 * 128 * 2, FS_BAR = FS_TILES + F_WG * FS_WG, FS_END = FS_BAR + 8 * F_WG + 16;
static_assert(FS_END <= 232448, "forward shared memory above the per-CTA limit");
constexpr uint32_t F_TMEM_COLS = 512;  // all of the SM's TMEM (one CTA per SM), 128 columns per warpgroup
static_assert(128 * F_WG <= F_TMEM_COLS, "forward TMEM above the per-SM 512 columns");

// Named barrier of one warpgroup (id 1 + warpgroup; 0 is the CTA barrier).
__device__ __forceinline__ void wg_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
// Named-barrier OR over the warpgroup's 128 threads.
__device__ __forceinline__ bool wg_bar_or(int id, bool p) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.or.pred b, %2, 128, a;\n selp.u32 %0, 1, 0, b;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(id)
        : "memory");
    return r != 0;
}
// sync_for_mma / wait_mma for one warpgroup
__device__ __forceinline__ void wg_sync_for_mma(int id) {
    fence_proxy_async_smem();
    tc_fence_before();
    wg_bar(id);
    tc_fence_after();
}
__device__ __forceinline__ bool wg_wait_mma(uint64_t* bar, uint32_t& phase, int* status, int id) {
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    const bool bad = wg_bar_or(id, !ok);
    if (bad && (threadIdx.x & 127) == 0) atomicOr(status, STATUS_WAIT_TIMEOUT);
    tc_fence_after();
    return !bad;
}

__global__ void __launch_bounds__(128 * F_WG, 1) k_mlp_fwd(MlpW w, const uint16_t* __restrict__ x, int N,
                                                         float* __restrict__ y, int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int wg = threadIdx.x >> 7, t = threadIdx.x & 127, warp = threadIdx.x >> 5;
    const int bid = 1 + wg;  // this warpgroup's named barrier
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + FS_BAR) + wg;
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + FS_BAR + 8 * F_WG);
    float* sb = reinterpret_cast<float*>(sm + FS_B);
    uint8_t* sx = sm + FS_TILES + wg * FS_WG + FS_X;
    uint8_t* sh = sm + FS_TILES + wg * FS_WG + FS_H;
    if (warp == 0) tc_alloc(slot, F_TMEM_COLS);
    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    load_cm(sm + FS_W1, w.W1, MLP_HID, MLP_IN);
    load_cm(sm + FS_W2, w.W2, MLP_HID, MLP_HID);
    load_cm(sm + FS_W3, w.W3, MLP_HID, MLP_HID);
    load_cm(sm + FS_W4, w.W4, MLP_OUT, MLP_HID);
    for (int i = threadIdx.x; i < 3 * MLP_HID + MLP_OUT; i += blockDim.x)
        sb[i] = i < 128 ? w.b1[i] : i < 256 ? w.b2[i - 128] : i < 384 ? w.b3[i - 256] : w.b4[i - 384];
    sync_for_mma();
    const uint32_t tm = *slot + 128u * (uint32_t)wg;                 // this warpgroup's columns
    const uint32_t tl = tm + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's TMEM lanes
    const uint32_t sa = smem_addr(sm), sxa = smem_addr(sx), sha = smem_addr(sh);
    constexpr uint32_t ID_H = tc_idesc(128, 128, 0, 0), ID_O = tc_idesc(128, 16, 0, 0);
    uint32_t phase = 0;
    const int ntiles = (N + 127) / 128;
    const int first = blockIdx.x * F_WG + wg, stride = gridDim.x * F_WG;
    // this thread's input row of tile i (zeros past N)
    auto load_x = [&](int i, uint4& x0, uint4& x1) {
        const int rr = i * 128 + t;
        x0 = make_uint4(0, 0, 0, 0);
        x1 = x0;
        if (i < ntiles && rr < N) {
            const uint4* xr = reinterpret_cast<const uint4*>(x + (size_t)rr * MLP_IN);
            x0 = __ldg(xr);
            x1 = __ldg(xr + 1);
        }
    };
    uint4 nx0, nx1;  // the next tile's row, loaded one tile ahead
    load_x(first, nx0, nx1);
    for (int i = first; i < ntiles; i += stride) {
        const int row = i * 128 + t;
        *reinterpret_cast<uint4*>(sx + cm_off(t, 0, MLP_IN)) = nx0;
        *reinterpret_cast<uint4*>(sx + cm_off(t, 8, MLP_IN)) = nx1;
        load_x(i + stride, nx0, nx1);
        wg_sync_for_mma(bid);
        if (t == 0) {
            tc_mma(tm, op_k(sxa, MLP_IN, 0), op_k(sa + FS_W1, MLP_IN, 0), ID_H, 0);
            tc_commit(bar);
        }
        if (!wg_wait_mma(bar, phase, status, bid)) break;
        epi_hidden<F_EPI>(tl, sb, sh, MLP_HID, t);
        bool ok = true;
#pragma unroll 1
        for (int layer = 0; layer < 2 && ok; layer++) {
            const uint32_t Wl = layer == 0 ? FS_W2 : FS_W3;
            wg_sync_for_mma(bid);
            if (t == 0) {
#pragma unroll
                for (int s = 0; s < 8; s++) tc_mma(tm, op_k(sha, MLP_HID, s), op_k(sa + Wl, MLP_HID, s), ID_H, s);
                tc_commit(bar);
            }
            ok = wg_wait_mma(bar, phase, status, bid);
            if (ok) epi_hidden<F_EPI>(tl, sb + 128 * (layer + 1), sh, MLP_HID, t);
        }
        if (!ok) break;
        // output layer into the first 16 columns (the last epilogue has read them)
        wg_sync_for_mma(bid);
        if (t == 0) {
#pragma unroll
            for (int s = 0; s < 8; s++) tc_mma(tm, op_k(sha, MLP_HID, s), op_k(sa + FS_W4, MLP_HID, s), ID_O, s);
            tc_commit(bar);
        }
        if (!wg_wait_mma(bar, phase, status, bid)) break;
        float o[16];
        tc_ld16(tl, o);
        if (row < N) {
            float4* yr = reinterpret_cast<float4*>(y + (size_t)row * MLP_OUT);
#pragma unroll
            for (int q = 0; q < 4; q++)
                yr[q] = make_float4(o[4 * q] + sb[384 + 4 * q], o[4 * q + 1] + sb[385 + 4 * q],
                                    o[4 * q + 2] + sb[386 + 4 * q], o[4 * q + 3] + sb[387 + 4 * q]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(*slot, F_TMEM_COLS);
}

// ---------------------------------------------------------------------------
// reverse mode
// ---------------------------------------------------------------------------
// shared memory (bytes): the weights as in the forward; X extended to 32
// features (x | 1 0 ... 0); H1, H2 extended to 144 (h | 1 0 ... 0); H3; the
// output gradient tile dZ4 [128][16]; one gradient tile dZ [128][128]; biases
constexpr int FX = 32, FHE = 144;
constexpr uint32_t BS_W1 = 0, BS_W2 = BS_W1 + 128 * 16 * 2, BS_W3 = BS_W2 + 128 * 128 * 2,
                   BS_W4 = BS_W3 + 128 * 128 * 2, BS_X = BS_W4 + 16 * 128 * 2, BS_H1 = BS_X + 128 * FX * 2,
                   BS_H2 = BS_H1 + 128 * FHE * 2, BS_H3 = BS_H2 + 128 * FHE * 2, BS_G4 = BS_H3 + 128 * 128 * 2,
                   BS_GZ = BS_G4 + 128 * 16 * 2, BS_B = BS_GZ + 128 * 128 * 2, BS_BAR = BS_B + 3 * 128 * 4,
                   BS_END = BS_BAR + 16;
// TMEM columns: per-tile accumulator, then the gradients kept over all tiles
constexpr uint32_t BT_Z = 0, BT_GW3 = 128, BT_GW2 = 288, BT_GW1 = 448, BT_GW4 = 480, B_TMEM_COLS = 512;

struct MlpG {
    float *gW1, *gW2, *gW3, *gW4, *gb1, *gb2, *gb3, *gb4;
};

// the ones block of an extended buffer: feature F0 = 1, F0 + 1 .. F0 + 15 = 0
__device__ __forceinline__ void ones_block(uint8_t* buf, int F, int F0, int r) {
    const uint32_t one = 0x3F80u;  // bf16 1.0
    *reinterpret_cast<uint4*>(buf + cm_off(r, F0, F)) = make_uint4(one, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(buf + cm_off(r, F0 + 8, F)) = make_uint4(0u, 0u, 0u, 0u);
}

// 32 FP32 values of a TMEM row added to global memory (16-byte aligned)
__device__ __forceinline__ void red_add32(float* dst, const float (&v)[32]) {
#pragma unroll
    for (int q = 0; q < 8; q++)
        atomicAdd(reinterpret_cast<float4*>(dst) + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
}

__global__ void __launch_bounds__(128, 1) k_mlp_bwd(MlpW w, MlpG g, const uint16_t* __restrict__ x, int N,
                                                    const float* __restrict__ gy, int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + BS_BAR);
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + BS_BAR + 8);
    float* sb = reinterpret_cast<float*>(sm + BS_B);
    if (warp == 0) tc_alloc(slot, B_TMEM_COLS);
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    load_cm(sm + BS_W1, w.W1, MLP_HID, MLP_IN);
    load_cm(sm + BS_W2, w.W2, MLP_HID, MLP_HID);
    load_cm(sm + BS_W3, w.W3, MLP_HID, MLP_HID);
    load_cm(sm + BS_W4, w.W4, MLP_OUT, MLP_HID);
    sb[tid] = w.b1[tid];
    sb[128 + tid] = w.b2[tid];
    sb[256 + tid] = w.b3[tid];
    ones_block(sm + BS_X, FX, MLP_IN, tid);
    ones_block(sm + BS_H1, FHE, MLP_HID, tid);
    ones_block(sm + BS_H2, FHE, MLP_HID, tid);
    sync_for_mma();
    const uint32_t tm = *slot;
    const uint32_t tl = tm + ((uint32_t)(warp * 32) << 16);
    const uint32_t sa = smem_addr(sm);
    constexpr uint32_t ID_FWD = tc_idesc(128, 128, 0, 0);   // Z = H W^T
    constexpr uint32_t ID_IN = tc_idesc(128, 128, 0, 1);    // dH = dZ W
    constexpr uint32_t ID_W4 = tc_idesc(128, 16, 1, 1);     // dW4^T = H3^T dZ4
    constexpr uint32_t ID_WH = tc_idesc(128, FHE, 1, 1);    // [dW | db] = dZ^T [H | 1]
    constexpr uint32_t ID_W1 = tc_idesc(128, FX, 1, 1);     // [dW1 | db1] = dZ1^T [X | 1]
    uint32_t phase = 0;
    float gb4[16];
#pragma unroll
    for (int j = 0; j < 16; j++) gb4[j] = 0.f;
    bool ok = true;
    int ntile_cta = 0;
    const int ntiles = (N + 127) / 128;
    // this thread's rows of x and gy in tile t (zeros past N), loaded one tile ahead
    auto load_rows = [&](int t, uint4& x0, uint4& x1, float4 (&g4)[4]) {
        const int rr = t * 128 + tid;
        x0 = make_uint4(0, 0, 0, 0);
        x1 = x0;
#pragma unroll
        for (int q = 0; q < 4; q++) g4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < ntiles && rr < N) {
            const uint4* xr = reinterpret_cast<const uint4*>(x + (size_t)rr * MLP_IN);
            x0 = __ldg(xr);
            x1 = __ldg(xr + 1);
            const float4* gq = reinterpret_cast<const float4*>(gy + (size_t)rr * MLP_OUT);
#pragma unroll
            for (int q = 0; q < 4; q++) g4[q] = __ldg(gq + q);
        }
    };
    uint4 nx0, nx1;
    float4 ng[4];
    load_rows(blockIdx.x, nx0, nx1, ng);
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int acc = ntile_cta > 0;  // accumulate onto the earlier tiles' weight gradients
        float gr[16];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            gr[4 * q] = ng[q].x; gr[4 * q + 1] = ng[q].y; gr[4 * q + 2] = ng[q].z; gr[4 * q + 3] = ng[q].w;
        }
        *reinterpret_cast<uint4*>(sm + BS_X + cm_off(tid, 0, FX)) = nx0;
        *reinterpret_cast<uint4*>(sm + BS_X + cm_off(tid, 8, FX)) = nx1;
        load_rows(t + gridDim.x, nx0, nx1, ng);
        // dZ4 = gy as BF16 (the tensor-core operand); the bias gradient of the
        // output layer sums the same rounded values
        uint32_t p[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            p[j] = pack_bf2(gr[2 * j], gr[2 * j + 1]);
            gb4[2 * j] += __uint_as_float(p[j] << 16);
            gb4[2 * j + 1] += __uint_as_float(p[j] & 0xFFFF0000u);
        }
        *reinterpret_cast<uint4*>(sm + BS_G4 + cm_off(tid, 0, 16)) = make_uint4(p[0], p[1], p[2], p[3]);
        *reinterpret_cast<uint4*>(sm + BS_G4 + cm_off(tid, 8, 16)) = make_uint4(p[4], p[5], p[6], p[7]);
        // forward recompute: H1, H2 (extended), H3 and the ReLU masks
        sync_for_mma();
        if (tid == 0) {
            tc_mma(tm + BT_Z, op_k(sa + BS_X, FX, 0), op_k(sa + BS_W1, MLP_IN, 0), ID_FWD, 0);
            tc_commit(bar);
        }
        if (!(ok = wait_mma(bar, phase, status))) break;
        epi_hidden(tl + BT_Z, sb, sm + BS_H1, FHE, tid);
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 8; s++)
                tc_mma(tm + BT_Z, op_k(sa + BS_H1, FHE, s), op_k(sa + BS_W2, MLP_HID, s), ID_FWD, s);
            tc_commit(bar);
        }
        if (!(ok = wait_mma(bar, phase, status))) break;
        epi_hidden(tl + BT_Z, sb + 128, sm + BS_H2, FHE, tid);
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 8; s++)
                tc_mma(tm + BT_Z, op_k(sa + BS_H2, FHE, s), op_k(sa + BS_W3, MLP_HID, s), ID_FWD, s);
            tc_commit(bar);
        }
        if (!(ok = wait_mma(bar, phase, status))) break;
        epi_hidden(tl + BT_Z, sb + 256, sm + BS_H3, MLP_HID, tid);
        // layer 4: dW4^T += H3^T dZ4; dH3 = dZ4 W4
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 8; s++)
                tc_mma(tm + BT_GW4, op_mn(sa + BS_H3, MLP_HID, s), op_mn(sa + BS_G4, 16, s), ID_W4, acc | s);
            tc_mma(tm + BT_Z, op_k(sa + BS_G4, 16, 0), op_mn(sa + BS_W4, MLP_HID, 0), ID_IN, 0);
            tc_commit(bar);
        }
        if (!(ok = wait_mma(bar, phase, status))) break;
        epi_grad(tl + BT_Z, sm + BS_H3, MLP_HID, sm + BS_GZ, tid);
        // layers 3, 2: [dW | db] += dZ^T [H | 1]; dH = dZ W
#pragma unroll 1
        for (int layer = 3; layer >= 2 && ok; layer--) {
            const uint32_t Hprev = layer == 3 ? BS_H2 : BS_H1;
            const uint32_t Wl = layer == 3 ? BS_W3 : BS_W2;
            const uint32_t Dw = layer == 3 ? BT_GW3 : BT_GW2;
            sync_for_mma();
            if (tid == 0) {
#pragma unroll
                for (int s = 0; s < 8; s++)
                    tc_mma(tm + Dw, op_mn(sa + BS_GZ, MLP_HID, s), op_mn(sa + Hprev, FHE, s), ID_WH, acc | s);
#pragma unroll
                for (int s = 0; s < 8; s++)
                    tc_mma(tm + BT_Z, op_k(sa + BS_GZ, MLP_HID, s), op_mn(sa + Wl, MLP_HID, s), ID_IN, s);
                tc_commit(bar);
            }
            if ((ok = wait_mma(bar, phase, status))) epi_grad(tl + BT_Z, sm + Hprev, FHE, sm + BS_GZ, tid);
        }
        if (!ok) break;
        // layer 1: [dW1 | db1] += dZ1^T [X | 1]
        sync_for_mma();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 8; s++)
                tc_mma(tm + BT_GW1, op_mn(sa + BS_GZ, MLP_HID, s), op_mn(sa + BS_X, FX, s), ID_W1, acc | s);
            tc_commit(bar);
        }
        if (!(ok = wait_mma(bar, phase, status))) break;
        ntile_cta++;
    }
    if (ok && ntile_cta > 0) {
        // this CTA's sums, added once: thread t holds row t of every accumulator
        float v[32];
        const int o = tid;
#pragma unroll 1
        for (int c = 0; c < 4; c++) {
            tc_ld32(tl + BT_GW3 + 32 * c, v);
            red_add32(g.gW3 + (size_t)o * MLP_HID + 32 * c, v);
            tc_ld32(tl + BT_GW2 + 32 * c, v);
            red_add32(g.gW2 + (size_t)o * MLP_HID + 32 * c, v);
        }
        float u[16];
        tc_ld16(tl + BT_GW3 + 128, u);
        atomicAdd(g.gb3 + o, u[0]);
        tc_ld16(tl + BT_GW2 + 128, u);
        atomicAdd(g.gb2 + o, u[0]);
        tc_ld32(tl + BT_GW1, v);  // columns 0..15: dW1[o][:], column 16: db1[o]
#pragma unroll
        for (int q = 0; q < 4; q++)
            atomicAdd(reinterpret_cast<float4*>(g.gW1 + (size_t)o * MLP_IN) + q,
                      make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
        atomicAdd(g.gb1 + o, v[16]);
        tc_ld16(tl + BT_GW4, u);  // row i = tid of dW4^T: dW4[k][i] for k = 0..15
#pragma unroll
        for (int k = 0; k < 16; k++) atomicAdd(g.gW4 + (size_t)k * MLP_HID + tid, u[k]);
    }
    // the output layer's bias gradient: the threads' sums, reduced through shared memory
    tc_fence_before();
    __syncthreads();
    float* red = reinterpret_cast<float*>(sm + BS_GZ);
#pragma unroll
    for (int j = 0; j < 16; j++) red[j * 128 + tid] = gb4[j];
    __syncthreads();
    if (tid < 16) {
        float s = 0.f;
        for (int k = 0; k < 128; k++) s += red[tid * 128 + k];
        if (ntile_cta > 0) atomicAdd(g.gb4 + tid, s);
    }
    __syncthreads();
    if (warp == 0) tc_dealloc(tm, B_TMEM_COLS);
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

static int sm_count(hcgs_ctx* ctx) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || n < 1) n = 148;
    return n;
}

hcgs_status mlp_fwd(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* const* W, const float* const* b,
                    float* y, cudaStream_t st) {
    const int tiles = (N + 127) / 128;
    const int wgs = (tiles + F_WG - 1) / F_WG;  // CTAs that have a tile for every warpgroup
    const int grid = wgs < sm_count(ctx) ? wgs : sm_count(ctx);  // one CTA per SM
    HCGS_CUDA(ctx, cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FS_END));
    HCGS_KERNEL(ctx, "k_mlp_fwd", st,
                k_mlp_fwd<<<grid, 128 * F_WG, FS_END, st>>>(make_w(W, b), x, N, y, ctx->d_status));
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
    MlpG g;
    g.gW1 = gW[0]; g.gW2 = gW[1]; g.gW3 = gW[2]; g.gW4 = gW[3];
    g.gb1 = gb[0]; g.gb2 = gb[1]; g.gb3 = gb[2]; g.gb4 = gb[3];
    const int tiles = (N + 127) / 128;
    const int grid = tiles < sm_count(ctx) ? tiles : sm_count(ctx);  // one CTA per SM (all of TMEM)
    HCGS_CUDA(ctx, cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BS_END));
    HCGS_KERNEL(ctx, "k_mlp_bwd", st, k_mlp_bwd<<<grid, 128, BS_END, st>>>(make_w(W, b), g, x, N, gy, ctx->d_status));
    return HCGS_OK;
}

}  // namespace hcgs
