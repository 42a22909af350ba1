// Band-limited angular spectrum method on sm_103a.
//
// Forward recording (Eq. layer2plane_asm + Eq. sum_planes) for a batch of
// views is run as three HBM passes, with the plane sum taken in the frequency
// domain (equal to the per-plane sum by linearity):
//   1. column DFT of every plane field           (fft_cols, batched)
//   2. per (view, channel, row): row DFT of each plane, multiply by the
//      transfer function H_{Z_l} (Eq. band_limited_asm_transfer_function),
//      accumulate over planes in shared memory, inverse row DFT  (rows_sum)
//   3. inverse column DFT of the sum, scaled by 1/(H W)     (fft_cols)
// The adjoint and the inverse propagation (Eq. plane2layer_asm) use the
// mirror image: column DFT of one field, then per row one forward row DFT
// and L (multiply by conj H, inverse row DFT) outputs (rows_spread), then
// inverse column DFTs.
//
// Transforms are mixed-radix (2, 3, 4, 5, 8) Stockham autosort transforms in
// shared memory; 1080 = 8*5*3*3*3 and 1920 = 8*8*2*3*5 are not powers of two.
// The transfer-function phase 2 pi z sqrt(1/lambda^2 - f^2) is formed in FP64
// and reduced mod 2 pi before it is rounded to an FP32 complex factor; the
// table holds one quadrant because H depends on f_x^2 and f_y^2 only.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "fft.cuh"

namespace hcgs {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward transform) or +i (inverse transform)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Small DFTs, y_k = sum_m v_m exp(-+ 2 pi i k m / R).
template <int R, bool INV>
__device__ __forceinline__ void dft(float2* v);

template <>
__device__ __forceinline__ void dft<2, false>(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void dft<2, true>(float2* v) { dft<2, false>(v); }

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
    const float s = 0.86602540378443865f;  // sin(2 pi / 3)
    float2 t = cadd(v[1], v[2]);
    float2 d = csub(v[1], v[2]);
    float2 a = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    float2 b = cscale(mul_mi<INV>(d), s);
    v[0] = cadd(v[0], t);
    v[1] = cadd(a, b);
    v[2] = csub(a, b);
}
template <>
__device__ __forceinline__ void dft<3, false>(float2* v) { dft3<false>(v); }
template <>
__device__ __forceinline__ void dft<3, true>(float2* v) { dft3<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft4(float2* v) {
    float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    float2 s13 = cadd(v[1], v[3]), d13 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
}
template <>
__device__ __forceinline__ void dft<4, false>(float2* v) { dft4<false>(v); }
template <>
__device__ __forceinline__ void dft<4, true>(float2* v) { dft4<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft5(float2* v) {
    const float c1 = 0.30901699437494742f;   // cos(2 pi / 5)
    const float c2 = -0.80901699437494742f;  // cos(4 pi / 5)
    const float s1 = 0.95105651629515357f;   // sin(2 pi / 5)
    const float s2 = 0.58778525229247313f;   // sin(4 pi / 5)
    float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    float2 a1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
    float2 a2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
    float2 b1 = mul_mi<INV>(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
    float2 b2 = mul_mi<INV>(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}
template <>
__device__ __forceinline__ void dft<5, false>(float2* v) { dft5<false>(v); }
template <>
__device__ __forceinline__ void dft<5, true>(float2* v) { dft5<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
    const float r = 0.70710678118654752f;
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV>(e);
    dft4<INV>(o);
    // o_k *= w^k, w = exp(-+ i pi / 4)
    o[1] = cmul(o[1], make_float2(r, INV ? r : -r));
    o[2] = mul_mi<INV>(o[2]);
    o[3] = cmul(o[3], make_float2(-r, INV ? r : -r));
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = cadd(e[k], o[k]);
        v[k + 4] = csub(e[k], o[k]);
    }
}
template <>
__device__ __forceinline__ void dft<8, false>(float2* v) { dft8<false>(v); }
template <>
__device__ __forceinline__ void dft<8, true>(float2* v) { dft8<true>(v); }

// One Stockham stage on `ntrans` transforms of length n; element i of
// transform t lives at buf[t * ts + i * es].  Ns = product of earlier radices.
template <int R, bool INV>
__device__ __forceinline__ void stage(const float2* __restrict__ src, float2* __restrict__ dst, int n, int Ns,
                                      int ntrans, int es, int ts, const float2* __restrict__ tw, int tid,
                                      int nthr) {
    const int m = n / R;
    const int total = m * ntrans;
    const int twstep = n / (Ns * R);
    for (int w = tid; w < total; w += nthr) {
        const int t = w % ntrans;
        const int j = w / ntrans;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = src[t * ts + (j + r * m) * es];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                float2 w_ = tw[r * k * twstep];
                if (INV) w_.y = -w_.y;
                v[r] = cmul(v[r], w_);
            }
        }
        dft<R, INV>(v);
        const int idxD = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) dst[t * ts + (idxD + r * Ns) * es] = v[r];
    }
}

// Runs all stages, ping-ponging between a and b; returns the buffer that
// holds the result.  Ends with a barrier.
template <bool INV>
__device__ float2* run_fft(float2* a, float2* b, const FftPlanArg& p, int ntrans, int es, int ts,
                           const float2* tw) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    int Ns = 1;
    for (int s = 0; s < p.nst; s++) {
        const int R = p.radix[s];
        switch (R) {
            case 2: stage<2, INV>(a, b, p.n, Ns, ntrans, es, ts, tw, tid, nthr); break;
            case 3: stage<3, INV>(a, b, p.n, Ns, ntrans, es, ts, tw, tid, nthr); break;
            case 4: stage<4, INV>(a, b, p.n, Ns, ntrans, es, ts, tw, tid, nthr); break;
            case 5: stage<5, INV>(a, b, p.n, Ns, ntrans, es, ts, tw, tid, nthr); break;
            default: stage<8, INV>(a, b, p.n, Ns, ntrans, es, ts, tw, tid, nthr); break;
        }
        __syncthreads();
        Ns *= R;
        float2* t = a; a = b; b = t;
    }
    return a;
}

__device__ __forceinline__ int mirror(int k, int n) { return k <= n / 2 ? k : n - k; }

// ---------------------------------------------------------------------------
// Compile-time plans for the lengths of the paper-shaped workloads (1080,
// 1920, 256, 512): constant divisors, unrolled radix sequence, and a padded
// shared-memory layout (one extra slot every 32 complex values) that spreads
// the strided Stockham stores over the banks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pad32(int e) { return e + (e >> 5); }
__host__ __device__ constexpr int padded_len(int e) { return e + e / 32 + 1; }

template <int N, int NS, int R, bool INV, int NTRANS, int ES, int TS>
__device__ __forceinline__ void stage_ct(const float2* __restrict__ src, float2* __restrict__ dst,
                                         const float2* __restrict__ tw) {
    constexpr int M = N / R, TOTAL = M * NTRANS, TWSTEP = N / (NS * R);
    for (int w = threadIdx.x; w < TOTAL; w += blockDim.x) {
        const int t = w % NTRANS, j = w / NTRANS, k = j % NS;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = src[pad32(t * TS + (j + r * M) * ES)];
        if (NS > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                float2 w_ = tw[r * k * TWSTEP];
                if (INV) w_.y = -w_.y;
                v[r] = cmul(v[r], w_);
            }
        }
        dft<R, INV>(v);
        const int idxD = (j / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; r++) dst[pad32(t * TS + (idxD + r * NS) * ES)] = v[r];
    }
}

template <bool INV, int N, int NTRANS, int ES, int TS, int NS, int R, int... RS>
struct CtStages {
    static __device__ __forceinline__ float2* run(float2* a, float2* b, const float2* tw) {
        stage_ct<N, NS, R, INV, NTRANS, ES, TS>(a, b, tw);
        __syncthreads();
        if constexpr (sizeof...(RS) == 0) {
            return b;
        } else {
            return CtStages<INV, N, NTRANS, ES, TS, NS * R, RS...>::run(b, a, tw);
        }
    }
};

template <int N, int... RS>
struct CtPlan {
    static constexpr int n = N;
    template <bool INV, int NTRANS, int ES, int TS>
    static __device__ __forceinline__ float2* run(float2* a, float2* b, const float2* tw) {
        return CtStages<INV, N, NTRANS, ES, TS, 1, RS...>::run(a, b, tw);
    }
};
using Plan1080 = CtPlan<1080, 8, 5, 3, 3, 3>;
using Plan1920 = CtPlan<1920, 8, 8, 2, 5, 3>;
using Plan512 = CtPlan<512, 8, 8, 8>;
using Plan256 = CtPlan<256, 8, 8, 4>;

// columns: grid (ceil(W/CW), nplanes), CW adjacent columns per CTA
template <bool INV, class PL, int CW>
__global__ void __launch_bounds__(256) k_fft_cols_ct(const float2* __restrict__ in, float2* __restrict__ out, int W,
                                                     const float2* __restrict__ tw_g, float scale) {
    constexpr int N = PL::n, E = N * CW, EP = padded_len(E);
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* Bb = sm + EP;
    float2* tw = sm + 2 * EP;
    const int col0 = blockIdx.x * CW;
    const size_t base = (size_t)blockIdx.y * N * W;
    for (int e = threadIdx.x; e < N; e += blockDim.x) tw[e] = tw_g[e];
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int i = e / CW, cc = e % CW, col = col0 + cc;
        A[pad32(e)] = col < W ? in[base + (size_t)i * W + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float2* res = PL::template run<INV, CW, CW, 1>(A, Bb, tw);
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int i = e / CW, cc = e % CW, col = col0 + cc;
        if (col < W) out[base + (size_t)i * W + col] = cscale(res[pad32(e)], scale);
    }
}

template <bool CONJ, class PL>
__global__ void __launch_bounds__(512) k_rows_sum_ct(const float2* __restrict__ in, float2* __restrict__ out, int L,
                                                     int C, int H, const float2* __restrict__ hq,
                                                     const float2* __restrict__ tw_g) {
    constexpr int W = PL::n, EP = padded_len(W);
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* Bb = sm + EP;
    float2* acc = sm + 2 * EP;
    float2* tw = sm + 3 * EP;
    const int b = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
    const int ky = mirror(i, H);
    constexpr int hw2 = W / 2 + 1;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        tw[j] = tw_g[j];
        acc[pad32(j)] = make_float2(0.f, 0.f);
    }
    for (int l = 0; l < L; l++) {
        const float2* src = in + ((((size_t)b * L + l) * C + c) * H + i) * W;
        for (int j = threadIdx.x; j < W; j += blockDim.x) A[pad32(j)] = src[j];
        __syncthreads();
        const float2* res = PL::template run<false, 1, 1, 0>(A, Bb, tw);
        const float2* hrow = hq + (((size_t)c * L + l) * (H / 2 + 1) + ky) * hw2;
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            float2 h = hrow[mirror(j, W)];
            if (CONJ) h.y = -h.y;
            acc[pad32(j)] = cadd(acc[pad32(j)], cmul(res[pad32(j)], h));
        }
        __syncthreads();
    }
    const float2* res = PL::template run<true, 1, 1, 0>(acc, A, tw);
    float2* dst = out + (((size_t)b * C + c) * H + i) * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) dst[j] = res[pad32(j)];
}

template <bool CONJ, class PL>
__global__ void __launch_bounds__(512) k_rows_spread_ct(const float2* __restrict__ in, float2* __restrict__ out,
                                                        int L, int C, int H, const float2* __restrict__ hq,
                                                        const float2* __restrict__ tw_g) {
    constexpr int W = PL::n, EP = padded_len(W);
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* Bb = sm + EP;
    float2* S = sm + 2 * EP;
    float2* tw = sm + 3 * EP;
    const int b = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
    const int ky = mirror(i, H);
    constexpr int hw2 = W / 2 + 1;
    const float2* src = in + (((size_t)b * C + c) * H + i) * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        tw[j] = tw_g[j];
        A[pad32(j)] = src[j];
    }
    __syncthreads();
    const float2* spec = PL::template run<false, 1, 1, 0>(A, Bb, tw);
    for (int j = threadIdx.x; j < W; j += blockDim.x) S[j] = spec[pad32(j)];
    __syncthreads();
    for (int l = 0; l < L; l++) {
        const float2* hrow = hq + (((size_t)c * L + l) * (H / 2 + 1) + ky) * hw2;
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            float2 h = hrow[mirror(j, W)];
            if (CONJ) h.y = -h.y;
            A[pad32(j)] = cmul(S[j], h);
        }
        __syncthreads();
        const float2* res = PL::template run<true, 1, 1, 0>(A, Bb, tw);
        float2* dst = out + ((((size_t)b * L + l) * C + c) * H + i) * W;
        for (int j = threadIdx.x; j < W; j += blockDim.x) dst[j] = res[pad32(j)];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// column transforms: grid (ceil(W/CW), nplanes); each CTA transforms CW
// adjacent columns of one plane, staged as smem[row][CW].
// ---------------------------------------------------------------------------
template <bool INV>
__global__ void k_fft_cols(const float2* __restrict__ in, float2* __restrict__ out, int H, int W, int CW,
                           FftPlanArg plan, const float2* __restrict__ tw_g, float scale) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* Bb = sm + (size_t)H * CW;
    float2* tw = Bb + (size_t)H * CW;
    const int col0 = blockIdx.x * CW;
    const size_t base = (size_t)blockIdx.y * H * W;
    for (int e = threadIdx.x; e < H; e += blockDim.x) tw[e] = tw_g[e];
    for (int e = threadIdx.x; e < H * CW; e += blockDim.x) {
        const int i = e / CW, cc = e - i * CW, col = col0 + cc;
        A[e] = col < W ? in[base + (size_t)i * W + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = run_fft<INV>(A, Bb, plan, CW, CW, 1, tw);
    for (int e = threadIdx.x; e < H * CW; e += blockDim.x) {
        const int i = e / CW, cc = e - i * CW, col = col0 + cc;
        if (col < W) out[base + (size_t)i * W + col] = cscale(res[e], scale);
    }
}

// Column pass of the focal-stack loss, in place on data[nplanes][H][W]:
//   V = scale * IDFT_cols(data);  I = |V|^2;  d = I - I_gt;
//   partial loss += d^2;  gV = 4 inv_count d V;  data = DFT_cols(gV).
__global__ void k_cols_focal_loss(float2* __restrict__ data, const float* __restrict__ Igt,
                                  float* __restrict__ Iout, float* __restrict__ partials, int H, int W, int CW,
                                  FftPlanArg plan, const float2* __restrict__ tw_g, float scale,
                                  float inv_count) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* Bb = sm + (size_t)H * CW;
    float2* tw = Bb + (size_t)H * CW;
    __shared__ float red[32];
    const int col0 = blockIdx.x * CW;
    const size_t base = (size_t)blockIdx.y * H * W;
    for (int e = threadIdx.x; e < H; e += blockDim.x) tw[e] = tw_g[e];
    for (int e = threadIdx.x; e < H * CW; e += blockDim.x) {
        const int i = e / CW, cc = e - i * CW, col = col0 + cc;
        A[e] = col < W ? data[base + (size_t)i * W + col] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = run_fft<true>(A, Bb, plan, CW, CW, 1, tw);
    float2* oth = res == A ? Bb : A;
    float part = 0.f;
    for (int e = threadIdx.x; e < H * CW; e += blockDim.x) {
        const int i = e / CW, cc = e - i * CW, col = col0 + cc;
        float2 g = make_float2(0.f, 0.f);
        if (col < W) {
            const float2 V = cscale(res[e], scale);
            const float I = V.x * V.x + V.y * V.y;
            const size_t o = base + (size_t)i * W + col;
            const float d = I - Igt[o];
            part += d * d;
            if (Iout) Iout[o] = I;
            g = cscale(V, 4.f * inv_count * d);
        }
        res[e] = g;
    }
    // block reduction of the loss partial (fixed order: deterministic)
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
    float2* r2 = run_fft<false>(res, oth, plan, CW, CW, 1, tw);
    for (int e = threadIdx.x; e < H * CW; e += blockDim.x) {
        const int i = e / CW, cc = e - i * CW, col = col0 + cc;
        if (col < W) data[base + (size_t)i * W + col] = r2[e];
    }
}

// ---------------------------------------------------------------------------
// row passes: grid (B, H, C) so that consecutive CTAs (views) share the
// transfer-function rows through L2.
// ---------------------------------------------------------------------------
template <bool CONJ>
__global__ void k_rows_sum(const float2* __restrict__ in, float2* __restrict__ out, int L, int C, int H, int W,
                           const float2* __restrict__ hq, FftPlanArg plan, const float2* __restrict__ tw_g) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* Bb = sm + W;
    float2* acc = sm + 2 * W;
    float2* tw = sm + 3 * W;
    const int b = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
    const int ky = mirror(i, H);
    const int hw2 = W / 2 + 1;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        tw[j] = tw_g[j];
        acc[j] = make_float2(0.f, 0.f);
    }
    for (int l = 0; l < L; l++) {
        const float2* src = in + ((((size_t)b * L + l) * C + c) * H + i) * W;
        for (int j = threadIdx.x; j < W; j += blockDim.x) A[j] = src[j];
        __syncthreads();
        float2* res = run_fft<false>(A, Bb, plan, 1, 1, 0, tw);
        const float2* hrow = hq + (((size_t)c * L + l) * (H / 2 + 1) + ky) * hw2;
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            float2 h = hrow[mirror(j, W)];
            if (CONJ) h.y = -h.y;
            acc[j] = cadd(acc[j], cmul(res[j], h));
        }
        __syncthreads();
    }
    float2* res = run_fft<true>(acc, A, plan, 1, 1, 0, tw);
    float2* dst = out + (((size_t)b * C + c) * H + i) * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) dst[j] = res[j];
}

template <bool CONJ>
__global__ void k_rows_spread(const float2* __restrict__ in, float2* __restrict__ out, int L, int C, int H,
                              int W, const float2* __restrict__ hq, FftPlanArg plan,
                              const float2* __restrict__ tw_g) {
    extern __shared__ float2 sm[];
    float2* A = sm;
    float2* Bb = sm + W;
    float2* S = sm + 2 * W;
    float2* tw = sm + 3 * W;
    const int b = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
    const int ky = mirror(i, H);
    const int hw2 = W / 2 + 1;
    const float2* src = in + (((size_t)b * C + c) * H + i) * W;
    for (int j = threadIdx.x; j < W; j += blockDim.x) {
        tw[j] = tw_g[j];
        A[j] = src[j];
    }
    __syncthreads();
    float2* spec = run_fft<false>(A, Bb, plan, 1, 1, 0, tw);
    for (int j = threadIdx.x; j < W; j += blockDim.x) S[j] = spec[j];
    __syncthreads();
    for (int l = 0; l < L; l++) {
        const float2* hrow = hq + (((size_t)c * L + l) * (H / 2 + 1) + ky) * hw2;
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            float2 h = hrow[mirror(j, W)];
            if (CONJ) h.y = -h.y;
            A[j] = cmul(S[j], h);
        }
        __syncthreads();
        float2* res = run_fft<true>(A, Bb, plan, 1, 1, 0, tw);
        float2* dst = out + ((((size_t)b * L + l) * C + c) * H + i) * W;
        for (int j = threadIdx.x; j < W; j += blockDim.x) dst[j] = res[j];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// transfer-function table, FP64
// ---------------------------------------------------------------------------
__global__ void k_build_hq(float2* __restrict__ hq, int H, int W, int C, int L, double px, double py, HArgs a) {
    const int hh = H / 2 + 1, wh = W / 2 + 1;
    const size_t total = (size_t)C * L * hh * wh;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e % wh);
        const int ky = (int)((e / wh) % hh);
        const int l = (int)((e / ((size_t)wh * hh)) % L);
        const int c = (int)(e / ((size_t)wh * hh * L));
        const double fx = kx / (W * px), fy = ky / (H * py);
        const double lam = a.lam[c];
        const double arg = 1.0 / (lam * lam) - (fx * fx + fy * fy);
        float2 h = make_float2(0.f, 0.f);
        if (arg >= 0.0) {
            const double twopi = 6.283185307179586476925286766559;
            double ph = twopi * a.z[l] * sqrt(arg);
            ph = ph - twopi * rint(ph / twopi);  // reduce to [-pi, pi] in FP64
            double s, co;
            sincos(ph, &s, &co);
            h = make_float2((float)co, (float)s);
        }
        hq[e] = h;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool fft_supported(int n) {
    if (n < 1 || n > MAX_FFT) return false;
    int m = n;
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

void factor_radices(int n, int* radix, int* nst) {
    int m = n;
    *nst = 0;
    while (m % 8 == 0) { radix[(*nst)++] = 8; m /= 8; }
    if (m % 4 == 0) { radix[(*nst)++] = 4; m /= 4; }
    if (m % 2 == 0) { radix[(*nst)++] = 2; m /= 2; }
    while (m % 5 == 0) { radix[(*nst)++] = 5; m /= 5; }
    while (m % 3 == 0) { radix[(*nst)++] = 3; m /= 3; }
}

static void factor(int n, FftPlan& p) { factor_radices(n, p.radix, &p.nst); }

static FftPlanArg plan_arg(const FftPlan* p) {
    FftPlanArg a;
    a.n = p->n;
    a.nst = p->nst;
    for (int s = 0; s < MAX_STAGES; s++) a.radix[s] = p->radix[s];
    return a;
}

hcgs_status get_plan(hcgs_ctx* ctx, int n, FftPlan** out) {
    auto it = ctx->plans.find(n);
    if (it != ctx->plans.end()) {
        *out = &it->second;
        return HCGS_OK;
    }
    if (!fft_supported(n)) {
        set_err(ctx, HCGS_ERR_UNSUPPORTED_SIZE, "FFT length " + std::to_string(n) + " is not 2^a 3^b 5^c <= 4096");
        return HCGS_ERR_UNSUPPORTED_SIZE;
    }
    FftPlan p;
    p.n = n;
    factor(n, p);
    std::vector<float2> tw(n);
    for (int m = 0; m < n; m++) {
        const double a = -2.0 * M_PI * (double)m / (double)n;
        tw[m] = make_float2((float)cos(a), (float)sin(a));
    }
    HCGS_CUDA(ctx, cudaMalloc(&p.tw, sizeof(float2) * n));
    ctx->bytes += sizeof(float2) * n;
    HCGS_CUDA(ctx, cudaMemcpy(p.tw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    auto ins = ctx->plans.emplace(n, p);
    *out = &ins.first->second;
    return HCGS_OK;
}

hcgs_status get_htab(hcgs_ctx* ctx, const hcgs_optics* o, const float2** out) {
    HKey k{o->H, o->W, o->C, o->L, o->pitch_x, o->pitch_y,
           std::vector<double>(o->wavelength, o->wavelength + o->C), std::vector<double>(o->plane_z, o->plane_z + o->L)};
    auto it = ctx->htab.find(k);
    if (it != ctx->htab.end()) {
        *out = (const float2*)it->second.p;
        return HCGS_OK;
    }
    DevBuf b;
    const size_t n = (size_t)o->C * o->L * (o->H / 2 + 1) * (o->W / 2 + 1);
    HCGS_CUDA(ctx, cudaMalloc(&b.p, n * sizeof(float2)));
    b.cap = n * sizeof(float2);
    ctx->bytes += b.cap;
    HArgs a{};
    for (int c = 0; c < o->C; c++) a.lam[c] = o->wavelength[c];
    for (int l = 0; l < o->L; l++) a.z[l] = o->plane_z[l];
    HCGS_KERNEL(ctx, "k_build_hq", 0, k_build_hq<<<1184, 256>>>((float2*)b.p, o->H, o->W, o->C, o->L, o->pitch_x, o->pitch_y, a));
    HCGS_LAUNCH(ctx, "k_build_hq");
    HCGS_CUDA(ctx, cudaDeviceSynchronize());
    ctx->htab.emplace(k, b);
    *out = (const float2*)b.p;
    return HCGS_OK;
}

static int col_width(int H) {
    // two slabs of H x CW complex plus the twiddles must fit in shared memory
    int cw = 8;
    while (cw > 1 && (size_t)(2 * cw + 1) * H * sizeof(float2) > 200 * 1024) cw /= 2;
    return cw;
}

template <typename K>
static cudaError_t allow_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class PL, int CW>
static hcgs_status fft_cols_ct(hcgs_ctx* ctx, const float2* in, float2* out, int nplanes, int W, bool inverse,
                               float scale, const float2* tw, cudaStream_t st) {
    constexpr int N = PL::n;
    const size_t smem = (2 * (size_t)padded_len(N * CW) + N) * sizeof(float2);
    dim3 grid((W + CW - 1) / CW, nplanes);
    if (inverse) {
        HCGS_CUDA(ctx, allow_smem(k_fft_cols_ct<true, PL, CW>, smem));
        HCGS_KERNEL(ctx, "k_fft_cols", st, k_fft_cols_ct<true, PL, CW><<<grid, 256, smem, st>>>(in, out, W, tw, scale));
    } else {
        HCGS_CUDA(ctx, allow_smem(k_fft_cols_ct<false, PL, CW>, smem));
        HCGS_KERNEL(ctx, "k_fft_cols", st, k_fft_cols_ct<false, PL, CW><<<grid, 256, smem, st>>>(in, out, W, tw, scale));
    }
    return HCGS_OK;
}

hcgs_status fft_cols(hcgs_ctx* ctx, const float2* in, float2* out, int nplanes, int H, int W, bool inverse,
                     float scale, cudaStream_t st) {
    if (nplanes <= 0) return HCGS_OK;
    FftPlan* p;
    hcgs_status s = get_plan(ctx, H, &p);
    if (s) return s;
    if (H == 1080) return fft_cols_ct<Plan1080, 4>(ctx, in, out, nplanes, W, inverse, scale, p->tw, st);
    if (H == 1920) return fft_cols_ct<Plan1920, 4>(ctx, in, out, nplanes, W, inverse, scale, p->tw, st);
    if (H == 512) return fft_cols_ct<Plan512, 8>(ctx, in, out, nplanes, W, inverse, scale, p->tw, st);
    if (H == 256) return fft_cols_ct<Plan256, 8>(ctx, in, out, nplanes, W, inverse, scale, p->tw, st);
    const int cw = col_width(H);
    const size_t smem = (size_t)(2 * cw + 1) * H * sizeof(float2);
    dim3 grid((W + cw - 1) / cw, nplanes);
    if (inverse) {
        HCGS_CUDA(ctx, allow_smem(k_fft_cols<true>, smem));
        HCGS_KERNEL(ctx, "k_fft_cols", st, k_fft_cols<true><<<grid, 512, smem, st>>>(in, out, H, W, cw, plan_arg(p), p->tw, scale));
    } else {
        HCGS_CUDA(ctx, allow_smem(k_fft_cols<false>, smem));
        HCGS_KERNEL(ctx, "k_fft_cols", st, k_fft_cols<false><<<grid, 512, smem, st>>>(in, out, H, W, cw, plan_arg(p), p->tw, scale));
    }
    HCGS_LAUNCH(ctx, "k_fft_cols");
    return HCGS_OK;
}

hcgs_status cols_focal_loss(hcgs_ctx* ctx, float2* data, const float* I_gt, float* I_out, float* partials,
                            int nplanes, int H, int W, float inv_count, float scale, int* nblocks_out,
                            cudaStream_t st) {
    FftPlan* p;
    hcgs_status s = get_plan(ctx, H, &p);
    if (s) return s;
    const int cw = col_width(H);
    const size_t smem = (size_t)(2 * cw + 1) * H * sizeof(float2);
    dim3 grid((W + cw - 1) / cw, nplanes);
    *nblocks_out = grid.x * grid.y;
    if (!partials) return HCGS_OK;  // size query
    HCGS_CUDA(ctx, allow_smem(k_cols_focal_loss, smem));
    HCGS_KERNEL(ctx, "k_cols_focal_loss", st, k_cols_focal_loss<<<grid, 512, smem, st>>>(data, I_gt, I_out, partials, H, W, cw, plan_arg(p), p->tw, scale,
                                               inv_count));
    HCGS_LAUNCH(ctx, "k_cols_focal_loss");
    return HCGS_OK;
}

static int row_threads(int W) {
    int t = ((W / 4 + 31) / 32) * 32;
    return t < 32 ? 32 : (t > 512 ? 512 : t);
}

template <class PL>
static hcgs_status rows_ct(hcgs_ctx* ctx, bool sum, const float2* in, float2* out, int B, int L, int C, int H,
                           const float2* hq, bool conjH, const float2* tw, cudaStream_t st) {
    constexpr int W = PL::n;
    const size_t smem = (3 * (size_t)padded_len(W) + W) * sizeof(float2);
    const int thr = row_threads(W);
    dim3 grid(B, H, C);
    if (sum) {
        if (conjH) {
            HCGS_CUDA(ctx, allow_smem(k_rows_sum_ct<true, PL>, smem));
            HCGS_KERNEL(ctx, "k_rows_sum", st, k_rows_sum_ct<true, PL><<<grid, thr, smem, st>>>(in, out, L, C, H, hq, tw));
        } else {
            HCGS_CUDA(ctx, allow_smem(k_rows_sum_ct<false, PL>, smem));
            HCGS_KERNEL(ctx, "k_rows_sum", st, k_rows_sum_ct<false, PL><<<grid, thr, smem, st>>>(in, out, L, C, H, hq, tw));
        }
    } else {
        if (conjH) {
            HCGS_CUDA(ctx, allow_smem(k_rows_spread_ct<true, PL>, smem));
            HCGS_KERNEL(ctx, "k_rows_spread", st, k_rows_spread_ct<true, PL><<<grid, thr, smem, st>>>(in, out, L, C, H, hq, tw));
        } else {
            HCGS_CUDA(ctx, allow_smem(k_rows_spread_ct<false, PL>, smem));
            HCGS_KERNEL(ctx, "k_rows_spread", st, k_rows_spread_ct<false, PL><<<grid, thr, smem, st>>>(in, out, L, C, H, hq, tw));
        }
    }
    return HCGS_OK;
}

static bool rows_ct_dispatch(hcgs_ctx* ctx, bool sum, const float2* in, float2* out, int B, int L, int C, int H,
                             int W, const float2* hq, bool conjH, const float2* tw, cudaStream_t st,
                             hcgs_status* res) {
    if (W == 1920) { *res = rows_ct<Plan1920>(ctx, sum, in, out, B, L, C, H, hq, conjH, tw, st); return true; }
    if (W == 1080) { *res = rows_ct<Plan1080>(ctx, sum, in, out, B, L, C, H, hq, conjH, tw, st); return true; }
    if (W == 512) { *res = rows_ct<Plan512>(ctx, sum, in, out, B, L, C, H, hq, conjH, tw, st); return true; }
    if (W == 256) { *res = rows_ct<Plan256>(ctx, sum, in, out, B, L, C, H, hq, conjH, tw, st); return true; }
    return false;
}

hcgs_status rows_sum(hcgs_ctx* ctx, const float2* in, float2* out, int B, int L, int C, int H, int W,
                     const float2* hq, bool conjH, cudaStream_t st) {
    FftPlan* p;
    hcgs_status s = get_plan(ctx, W, &p);
    if (s) return s;
    if (rows_ct_dispatch(ctx, true, in, out, B, L, C, H, W, hq, conjH, p->tw, st, &s)) return s;
    const size_t smem = 4 * (size_t)W * sizeof(float2);
    dim3 grid(B, H, C);
    if (conjH) {
        HCGS_CUDA(ctx, allow_smem(k_rows_sum<true>, smem));
        HCGS_KERNEL(ctx, "k_rows_sum", st, k_rows_sum<true><<<grid, row_threads(W), smem, st>>>(in, out, L, C, H, W, hq, plan_arg(p), p->tw));
    } else {
        HCGS_CUDA(ctx, allow_smem(k_rows_sum<false>, smem));
        HCGS_KERNEL(ctx, "k_rows_sum", st, k_rows_sum<false><<<grid, row_threads(W), smem, st>>>(in, out, L, C, H, W, hq, plan_arg(p), p->tw));
    }
    HCGS_LAUNCH(ctx, "k_rows_sum");
    return HCGS_OK;
}

hcgs_status rows_spread(hcgs_ctx* ctx, const float2* in, float2* out, int B, int L, int C, int H, int W,
                        const float2* hq, bool conjH, cudaStream_t st) {
    FftPlan* p;
    hcgs_status s = get_plan(ctx, W, &p);
    if (s) return s;
    if (rows_ct_dispatch(ctx, false, in, out, B, L, C, H, W, hq, conjH, p->tw, st, &s)) return s;
    const size_t smem = 4 * (size_t)W * sizeof(float2);
    dim3 grid(B, H, C);
    if (conjH) {
        HCGS_CUDA(ctx, allow_smem(k_rows_spread<true>, smem));
        HCGS_KERNEL(ctx, "k_rows_spread", st, k_rows_spread<true><<<grid, row_threads(W), smem, st>>>(in, out, L, C, H, W, hq, plan_arg(p), p->tw));
    } else {
        HCGS_CUDA(ctx, allow_smem(k_rows_spread<false>, smem));
        HCGS_KERNEL(ctx, "k_rows_spread", st, k_rows_spread<false><<<grid, row_threads(W), smem, st>>>(in, out, L, C, H, W, hq, plan_arg(p), p->tw));
    }
    HCGS_LAUNCH(ctx, "k_rows_spread");
    return HCGS_OK;
}

// out[b][c] = sum_l IDFT(Hsel DFT(in[b][l][c])), Hsel = H_{Z_l} or its conjugate.
hcgs_status asm_sum(hcgs_ctx* ctx, const float2* in, float2* out, int B, const hcgs_optics* o, bool conjH,
                    cudaStream_t st) {
    const float2* hq;
    hcgs_status s = get_htab(ctx, o, &hq);
    if (s) return s;
    const size_t planeN = (size_t)o->H * o->W;
    const size_t nS = (size_t)B * o->L * o->C * planeN;
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[0], nS * sizeof(float2), &ctx->bytes));
    float2* S = (float2*)ctx->ws[0].p;
    if ((s = fft_cols(ctx, in, S, B * o->L * o->C, o->H, o->W, false, 1.f, st))) return s;
    if ((s = rows_sum(ctx, S, out, B, o->L, o->C, o->H, o->W, hq, conjH, st))) return s;
    return fft_cols(ctx, out, out, B * o->C, o->H, o->W, true, 1.f / (float)planeN, st);
}

// out[b][l][c] = IDFT(Hsel DFT(in[b][c])).
hcgs_status asm_spread(hcgs_ctx* ctx, const float2* in, float2* out, int B, const hcgs_optics* o, bool conjH,
                       cudaStream_t st) {
    const float2* hq;
    hcgs_status s = get_htab(ctx, o, &hq);
    if (s) return s;
    const size_t planeN = (size_t)o->H * o->W;
    const size_t nS = (size_t)B * o->C * planeN;
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[1], nS * sizeof(float2), &ctx->bytes));
    float2* S = (float2*)ctx->ws[1].p;
    if ((s = fft_cols(ctx, in, S, B * o->C, o->H, o->W, false, 1.f, st))) return s;
    if ((s = rows_spread(ctx, S, out, B, o->L, o->C, o->H, o->W, hq, conjH, st))) return s;
    return fft_cols(ctx, out, out, B * o->L * o->C, o->H, o->W, true, 1.f / (float)planeN, st);
}

// ---------------------------------------------------------------------------
// raw launchers (explicit plans and tables, no context)
// ---------------------------------------------------------------------------
cudaError_t launch_fft_cols_raw(bool inverse, const float2* in, float2* out, int nplanes, int H, int W,
                                const FftPlanArg& plan, const float2* tw, float scale, cudaStream_t st) {
    const int cw = col_width(H);
    const size_t smem = (size_t)(2 * cw + 1) * H * sizeof(float2);
    const dim3 grid((W + cw - 1) / cw, nplanes);
    cudaError_t e;
    if (inverse) {
        if ((e = allow_smem(k_fft_cols<true>, smem)) != cudaSuccess) return e;
        k_fft_cols<true><<<grid, 512, smem, st>>>(in, out, H, W, cw, plan, tw, scale);
    } else {
        if ((e = allow_smem(k_fft_cols<false>, smem)) != cudaSuccess) return e;
        k_fft_cols<false><<<grid, 512, smem, st>>>(in, out, H, W, cw, plan, tw, scale);
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_spread_conj_raw(const float2* in, float2* out, int B, int L, int C, int H, int W,
                                        const float2* hq, const FftPlanArg& plan, const float2* tw,
                                        cudaStream_t st) {
    const size_t smem = 4 * (size_t)W * sizeof(float2);
    cudaError_t e = allow_smem(k_rows_spread<true>, smem);
    if (e != cudaSuccess) return e;
    k_rows_spread<true><<<dim3(B, H, C), row_threads(W), smem, st>>>(in, out, L, C, H, W, hq, plan, tw);
    return cudaGetLastError();
}

cudaError_t launch_build_hq_raw(float2* hq, int H, int W, int C, int L, double px, double py, const HArgs& a,
                                cudaStream_t st) {
    const size_t n = (size_t)C * L * (H / 2 + 1) * (W / 2 + 1);
    const int blocks = (int)std::min<size_t>(1184, (n + 255) / 256);
    k_build_hq<<<blocks, 256, 0, st>>>(hq, H, W, C, L, px, py, a);
    return cudaGetLastError();
}

}  // namespace hcgs
