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
#include <type_traits>
#include <utility>

#include "common.cuh"
#include "fft.cuh"

namespace hcgs {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// complex add, subtract and real scaling as packed FP32x2 operations
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
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
    float2 a = __ffma2_rn(make_float2(-0.5f, -0.5f), t, v[0]);
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
    const float2 C1 = make_float2(c1, c1), C2 = make_float2(c2, c2);
    const float2 S1 = make_float2(s1, s1), S2 = make_float2(s2, s2);
    float2 a1 = __ffma2_rn(C2, t2, __ffma2_rn(C1, t1, v[0]));
    float2 a2 = __ffma2_rn(C1, t2, __ffma2_rn(C2, t1, v[0]));
    float2 b1 = mul_mi<INV>(__ffma2_rn(S2, t4, __fmul2_rn(S1, t3)));
    float2 b2 = mul_mi<INV>(__ffma2_rn(make_float2(-s1, -s1), t4, __fmul2_rn(S2, t3)));
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
// Register-resident transforms for the lengths of the paper-shaped workloads
// (1080, 1920, 512, 256).
//
// A length-N transform is two or three Stockham stages of composite radix
// (9, 10, 12, 16, ... each an in-register DFT built from the small ones with
// compile-time twiddle constants).  A thread keeps its work items of a stage
// in registers: the first stage reads its inputs straight from global memory,
// the last stage hands its outputs to the caller in registers, and only the
// exchanges between stages go through shared memory (one in-place buffer, a
// write and a read per element each).  The padding of that buffer is chosen
// per exchange so that the strided stores and loads of the two stages it
// joins fall on distinct banks.  Because the last stage of one transform and
// the first stage of a transform with the reversed radix order own the same
// elements, a forward row transform can feed an inverse one, or an inverse
// column transform a forward one, without an exchange.
// ---------------------------------------------------------------------------
namespace rfft {

// compile-time loop over 0..n-1
template <class F, int... I>
__device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}
#define HCGS_CI(x) decltype(x)::value

// sin and cos on [0, pi/2] by their Taylor series, evaluated in double at
// compile time (the remainder after 12 terms is below 1e-20)
__host__ __device__ constexpr double ct_sin(double x) {
    double t = x, s = x;
    for (int n = 1; n <= 12; n++) {
        t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double ct_cos(double x) {
    double t = 1.0, s = 1.0;
    for (int n = 1; n <= 12; n++) {
        t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
        s += t;
    }
    return s;
}
// cos and sin of 2 pi m / n: quadrant q and remainder phi in [0, pi/2)
__host__ __device__ constexpr double ct_cos2pi(int m, int n) {
    const int a = ((m % n) + n) % n, q = (4 * a) / n;
    const double phi = 1.5707963267948966 * (double)(4 * a - q * n) / (double)n;
    return q == 0 ? ct_cos(phi) : q == 1 ? -ct_sin(phi) : q == 2 ? -ct_cos(phi) : ct_sin(phi);
}
__host__ __device__ constexpr double ct_sin2pi(int m, int n) {
    const int a = ((m % n) + n) % n, q = (4 * a) / n;
    const double phi = 1.5707963267948966 * (double)(4 * a - q * n) / (double)n;
    return q == 0 ? ct_sin(phi) : q == 1 ? ct_cos(phi) : q == 2 ? -ct_sin(phi) : -ct_cos(phi);
}

// a * exp(-+ 2 pi i m / r) (forward: -, inverse: +), exact for quarter turns
template <int M, int R, bool INV>
__device__ __forceinline__ float2 twc(float2 a) {
    constexpr int m = M % R;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (2 * m == R) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (4 * m == R) {
        return mul_mi<INV>(a);
    } else if constexpr (4 * m == 3 * R) {
        return mul_mi<!INV>(a);
    } else {
        constexpr float c = (float)ct_cos2pi(m, R);
        constexpr float s = INV ? (float)ct_sin2pi(m, R) : -(float)ct_sin2pi(m, R);
        return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

template <int R, bool INV>
struct Dft {
    static __device__ __forceinline__ void run(float2* v) { dft<R, INV>(v); }
};
// R = R1 R2: input n = R2 n1 + n2, output k = k1 + R1 k2;
// X[k1 + R1 k2] = sum_n2 W_R2^(n2 k2) W_R^(n2 k1) sum_n1 x[R2 n1 + n2] W_R1^(n1 k1)
template <int R1, int R2, bool INV>
struct DftSplit {
    static __device__ __forceinline__ void run(float2* v) {
        float2 y[R2][R1];
        sfor<R2>([&](auto a) {
            constexpr int n2 = HCGS_CI(a);
            sfor<R1>([&](auto b) { y[n2][HCGS_CI(b)] = v[R2 * HCGS_CI(b) + n2]; });
            Dft<R1, INV>::run(y[n2]);
            sfor<R1>([&](auto b) {
                constexpr int k1 = HCGS_CI(b);
                y[n2][k1] = twc<n2 * k1, R1 * R2, INV>(y[n2][k1]);
            });
        });
        sfor<R1>([&](auto b) {
            constexpr int k1 = HCGS_CI(b);
            float2 z[R2];
            sfor<R2>([&](auto a) { z[HCGS_CI(a)] = y[HCGS_CI(a)][k1]; });
            Dft<R2, INV>::run(z);
            sfor<R2>([&](auto a) { v[k1 + R1 * HCGS_CI(a)] = z[HCGS_CI(a)]; });
        });
    }
};
template <bool INV> struct Dft<6, INV> : DftSplit<2, 3, INV> {};
template <bool INV> struct Dft<9, INV> : DftSplit<3, 3, INV> {};
template <bool INV> struct Dft<10, INV> : DftSplit<2, 5, INV> {};
template <bool INV> struct Dft<12, INV> : DftSplit<4, 3, INV> {};
template <bool INV> struct Dft<15, INV> : DftSplit<3, 5, INV> {};
template <bool INV> struct Dft<16, INV> : DftSplit<4, 4, INV> {};

// Twiddles and DFT of one work item j of a stage (Ns = product of the earlier
// radices): v[r] *= w^r with w = W_{Ns R}^(j mod Ns) read from the length-N
// table.  The powers are a running product restarted from the table every
// four steps (w^4 read alongside w), so at most three products deep.
template <int N, int NS, int R, bool INV>
__device__ __forceinline__ void stage_math(float2 (&v)[R], int j, const float2* __restrict__ tw) {
    if constexpr (NS > 1) {
        constexpr int STEP = N / (NS * R);
        const int k = j % NS;
        float2 w = __ldg(tw + k * STEP);
        if (INV) w.y = -w.y;
        float2 w4 = make_float2(1.f, 0.f);
        if constexpr (R > 4) {
            w4 = __ldg(tw + 4 * k * STEP);
            if (INV) w4.y = -w4.y;
        }
        float2 base = w4, p = w;  // p = w^r, base = w^(4 floor(r / 4))
        sfor<R>([&](auto a) {
            constexpr int r = HCGS_CI(a);
            if constexpr (r >= 1) {
                if constexpr (r % 4 == 0) {
                    if constexpr (r > 4) base = cmul(base, w4);
                    p = base;
                } else if constexpr (r > 1) {
                    p = cmul(p, w);
                }
                v[r] = cmul(v[r], p);
            }
        });
    }
    Dft<R, INV>::run(v);
}

template <int... RS> struct Seq {};
// shared-memory slot of element e: one gap of Q slots after every P elements
template <int P, int Q>
struct Pad {
    static __device__ __forceinline__ int at(int e) { return Q == 0 ? e : e + Q * (e / P); }
    static constexpr int extent(int n) { return n + Q * ((n - 1) / P) + 1; }
};
template <class... Ls> struct Lays {};

// Work items of a stage: w = threadIdx.x + u T (u < U), transform t = w mod
// NTRANS, item j = w / NTRANS; element e of the buffer = position * NTRANS + t.
template <int M, int NTRANS, int T>
struct Items {
    static constexpr int TOTAL = M * NTRANS, U = (TOTAL + T - 1) / T;
    static __device__ __forceinline__ bool valid(int u) { return TOTAL % T == 0 || threadIdx.x + u * T < TOTAL; }
    static __device__ __forceinline__ int t(int u) { return (threadIdx.x + u * T) % NTRANS; }
    static __device__ __forceinline__ int j(int u) { return (threadIdx.x + u * T) / NTRANS; }
};

template <int N, bool INV, int NTRANS, int T, int NS, class RSeq, class LSeq>
struct Stages;

template <int N, bool INV, int NTRANS, int T, int NS, int R>
struct Stages<N, INV, NTRANS, T, NS, Seq<R>, Lays<>> {
    static constexpr int M = N / R;
    using It = Items<M, NTRANS, T>;
    static constexpr int U = It::U, RAD = R;
    static constexpr int smem(int) { return 0; }
    // v: this stage's inputs (element j + r M of item j); out(v) receives
    // the outputs (element j + r M of the transform again)
    template <class Out>
    static __device__ __forceinline__ void run(float2 (&v)[U][R], float2*, const float2* __restrict__ tw, Out&& out) {
        sfor<U>([&](auto a) { stage_math<N, NS, R, INV>(v[HCGS_CI(a)], It::j(HCGS_CI(a)), tw); });
        out(v);
    }
};

template <int N, bool INV, int NTRANS, int T, int NS, int R, int R2, int... RS, class L, class... LS>
struct Stages<N, INV, NTRANS, T, NS, Seq<R, R2, RS...>, Lays<L, LS...>> {
    static constexpr int M = N / R;
    using It = Items<M, NTRANS, T>;
    static constexpr int U = It::U, RAD = R;
    using Next = Stages<N, INV, NTRANS, T, NS * R, Seq<R2, RS...>, Lays<LS...>>;
    // complex slots of shared memory the exchanges use
    static constexpr int smem(int n) {
        return L::extent(n) > Next::smem(n) ? L::extent(n) : Next::smem(n);
    }
    template <class Out>
    static __device__ __forceinline__ void run(float2 (&v)[U][R], float2* sm, const float2* __restrict__ tw,
                                               Out&& out) {
        sfor<U>([&](auto a) { stage_math<N, NS, R, INV>(v[HCGS_CI(a)], It::j(HCGS_CI(a)), tw); });
        __syncthreads();  // earlier readers of the buffer are done
        sfor<U>([&](auto a) {
            constexpr int u = HCGS_CI(a);
            if (It::valid(u)) {
                const int j = It::j(u), t = It::t(u);
                const int base = (j / NS) * NS * R + j % NS;
                sfor<R>([&](auto b) {
                    constexpr int r = HCGS_CI(b);
                    sm[L::at((base + r * NS) * NTRANS + t)] = v[u][r];
                });
            }
        });
        __syncthreads();
        using Nt = typename Next::It;
        float2 v2[Next::U][R2];
        sfor<Next::U>([&](auto a) {
            constexpr int u = HCGS_CI(a);
            const bool ok = Nt::valid(u);
            const int j = Nt::j(u), t = Nt::t(u);
            sfor<R2>([&](auto b) {
                constexpr int r = HCGS_CI(b);
                v2[u][r] = ok ? sm[L::at((j + r * Next::M) * NTRANS + t)] : make_float2(0.f, 0.f);
            });
        });
        Next::run(v2, sm, tw, out);
    }
};

template <class V>
struct Shape {
    using A = std::remove_reference_t<V>;
    static constexpr int U = std::extent<A, 0>::value, R = std::extent<A, 1>::value;
};

// Column plan: N-point transforms of CW adjacent columns per CTA of T threads;
// radix order A with exchange layouts LA, and the reversed order B with LB.
template <int N_, int CW_, int T_, int MINB_, class A_, class LA_, class B_, class LB_>
struct ColPlan {
    static constexpr int N = N_, CW = CW_, T = T_, MINB = MINB_;
    using A = A_;
    using LA = LA_;
    using B = B_;
    using LB = LB_;
    template <bool INV> using SA = Stages<N, INV, CW, T, 1, A, LA>;
    template <bool INV> using SB = Stages<N, INV, CW, T, 1, B, LB>;
    static constexpr int smem_slots() {
        return SA<false>::smem(N * CW) > SB<false>::smem(N * CW) ? SA<false>::smem(N * CW) : SB<false>::smem(N * CW);
    }
};
// Row plan: one row per CTA of T threads.
// MINB_ / MINBS_: resident CTAs per SM the spread / sum pass's registers are capped for
template <int N_, int T_, int MINB_, class A_, class LA_, class B_, class LB_, int MINBS_ = MINB_>
struct RowPlan {
    static constexpr int N = N_, T = T_, MINB = MINB_, MINBS = MINBS_;
    template <bool INV> using SA = Stages<N, INV, 1, T, 1, A_, LA_>;
    template <bool INV> using SB = Stages<N, INV, 1, T, 1, B_, LB_>;
    static constexpr int smem_slots() {
        return SA<false>::smem(N) > SB<false>::smem(N) ? SA<false>::smem(N) : SB<false>::smem(N);
    }
};

using Cols1080 = ColPlan<1080, 8, 480, 2, Seq<12, 10, 9>, Lays<Pad<16, 4>, Pad<128, 1>>, Seq<9, 10, 12>,
                         Lays<Pad<1, 0>, Pad<512, 8>>>;
using Cols1920 = ColPlan<1920, 4, 384, 1, Seq<16, 12, 10>, Lays<Pad<16, 1>, Pad<160, 1>>, Seq<10, 12, 16>,
                         Lays<Pad<80, 4>, Pad<160, 8>>>;
using Cols512 = ColPlan<512, 16, 512, 2, Seq<8, 8, 8>, Lays<Pad<1, 0>, Pad<1, 0>>, Seq<8, 8, 8>,
                        Lays<Pad<1, 0>, Pad<1, 0>>>;
using Cols256 = ColPlan<256, 16, 256, 3, Seq<16, 16>, Lays<Pad<1, 0>>, Seq<16, 16>, Lays<Pad<1, 0>>>;

// 1920 = 8 x 15 x 16 on 128 threads: the stages have 240, 128 and 120 work
// items, so few threads idle at the exchange barriers (16 x 12 x 10 on 192
// threads left 37 % of them without a butterfly in the radix-16 stage)
using Rows1920 = RowPlan<1920, 128, 4, Seq<8, 15, 16>, Lays<Pad<16, 1>, Pad<128, 1>>, Seq<16, 15, 8>,
                         Lays<Pad<16, 1>, Pad<1, 0>>, 3>;
using Rows1080 = RowPlan<1080, 128, 4, Seq<12, 10, 9>, Lays<Pad<48, 1>, Pad<120, 4>>, Seq<9, 10, 12>,
                         Lays<Pad<1, 0>, Pad<1, 0>>>;
using Rows512 = RowPlan<512, 64, 8, Seq<8, 8, 8>, Lays<Pad<16, 1>, Pad<16, 2>>, Seq<8, 8, 8>,
                        Lays<Pad<16, 1>, Pad<16, 2>>>;
using Rows256 = RowPlan<256, 64, 8, Seq<4, 8, 8>, Lays<Pad<16, 1>, Pad<16, 2>>, Seq<8, 8, 4>,
                        Lays<Pad<16, 1>, Pad<16, 2>>>;

// Loads the first-stage inputs of a column slab (element row j + r M of
// column t) from global memory; columns at or beyond ncols read as zero.
template <class S, int CW>
__device__ __forceinline__ void load_cols(float2 (&v)[S::U][S::RAD], const float2* src, int W, int ncols) {
    using It = typename S::It;
    sfor<S::U>([&](auto a) {
        constexpr int u = HCGS_CI(a);
        const int t = It::t(u), j = It::j(u);
        const bool ok = It::valid(u) && t < ncols;
        sfor<S::RAD>([&](auto b) {
            constexpr int r = HCGS_CI(b);
            v[u][r] = ok ? src[(size_t)(j + r * S::M) * W + t] : make_float2(0.f, 0.f);
        });
    });
}

template <class S>
__device__ __forceinline__ void load_row(float2 (&v)[S::U][S::RAD], const float2* __restrict__ src) {
    using It = typename S::It;
    sfor<S::U>([&](auto a) {
        constexpr int u = HCGS_CI(a);
        const int j = It::j(u);
        const bool ok = It::valid(u);
        sfor<S::RAD>([&](auto b) {
            constexpr int r = HCGS_CI(b);
            v[u][r] = ok ? __ldg(src + j + r * S::M) : make_float2(0.f, 0.f);
        });
    });
}

// outputs of a last stage with U items of radix R: element j + r (N / R)
template <int N, int NTRANS, int T, class V, class F>
__device__ __forceinline__ void for_outputs(V& vo, F&& f) {
    using Sh = Shape<V>;
    using It = Items<N / Sh::R, NTRANS, T>;
    sfor<Sh::U>([&](auto a) {
        constexpr int u = HCGS_CI(a);
        if (It::valid(u)) {
            const int j = It::j(u), t = It::t(u);
            sfor<Sh::R>([&](auto b) {
                constexpr int r = HCGS_CI(b);
                f(vo[u][r], j + r * (N / Sh::R), t);
            });
        }
    });
}

}  // namespace rfft

// columns: grid (ceil(W / CW), nplanes); in == out allowed (each CTA reads its
// whole slab before it writes)
template <bool INV, class CP>
__global__ void __launch_bounds__(CP::T, CP::MINB) k_fft_cols_reg(const float2* in, float2* out, int W,
                                                                  const float2* __restrict__ tw, float scale) {
    using namespace rfft;
    using S = typename CP::template SA<INV>;
    extern __shared__ float2 sm[];
    const int col0 = blockIdx.x * CP::CW, ncols = W - col0;
    const size_t base = (size_t)blockIdx.y * CP::N * W + col0;
    float2 v[S::U][S::RAD];
    load_cols<S, CP::CW>(v, in + base, W, ncols);
    S::run(v, sm, tw, [&](auto& vo) {
        for_outputs<CP::N, CP::CW, CP::T>(vo, [&](float2 x, int pos, int t) {
            if (t < ncols) out[base + (size_t)pos * W + t] = cscale(x, scale);
        });
    });
}

// Column pass of the focal-stack loss, in place on data[nplanes][N][W]:
//   V = scale * IDFT_cols(data);  I = |V|^2;  d = I - I_gt;
//   partial loss += d^2;  gV = 4 inv_count d V;  data = DFT_cols(gV).
template <class CP>
__global__ void __launch_bounds__(CP::T, CP::MINB)
    k_cols_focal_loss_reg(float2* data, const float* __restrict__ Igt, float* __restrict__ Iout,
                          float* __restrict__ partials, int W, const float2* __restrict__ tw, float scale,
                          float inv_count) {
    using namespace rfft;
    using SI = typename CP::template SA<true>;
    using SF = typename CP::template SB<false>;
    extern __shared__ float2 sm[];
    __shared__ float red[32];
    const int col0 = blockIdx.x * CP::CW, ncols = W - col0;
    const size_t base = (size_t)blockIdx.y * CP::N * W + col0;
    float2 v[SI::U][SI::RAD];
    load_cols<SI, CP::CW>(v, data + base, W, ncols);
    SI::run(v, sm, tw, [&](auto& vo) {
        float part = 0.f;
        for_outputs<CP::N, CP::CW, CP::T>(vo, [&](float2& x, int pos, int t) {
            float2 g = make_float2(0.f, 0.f);
            if (t < ncols) {
                const float2 V = cscale(x, scale);
                const float I = V.x * V.x + V.y * V.y;
                const size_t o = base + (size_t)pos * W + t;
                const float d = I - Igt[o];
                part += d * d;
                if (Iout) Iout[o] = I;
                g = cscale(V, 4.f * inv_count * d);
            }
            x = g;
        });
        // items outside the transform hold zeros (never read back)
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            float s = 0.f;
            for (int w = 0; w < CP::T / 32; w++) s += red[w];
            partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
        }
        static_assert(Shape<decltype(vo)>::R == SF::RAD && Shape<decltype(vo)>::U == SF::U,
                      "the forward pass must start with the inverse pass's last radix");
        SF::run(vo, sm, tw, [&](auto& vf) {
            for_outputs<CP::N, CP::CW, CP::T>(vf, [&](float2 x, int pos, int t) {
                if (t < ncols) data[base + (size_t)pos * W + t] = x;
            });
        });
    });
}

// Row passes: grid (B, H, C) so that consecutive CTAs (views) share the
// transfer-function rows through L2.  The rows a CTA needs next (the next
// plane's input row and transfer-function row) are brought into a second
// shared-memory buffer by bulk copies while the current plane is transformed
// (two buffers, one mbarrier each).  Shared memory: the exchange buffer, then
// the row buffers, then the barriers.
template <class RP, bool WITH_INPUT>
struct RowSmem {
    static constexpr int W = RP::N, HS = hq_stride(RP::N);
    static constexpr int XS = (RP::smem_slots() + 1) & ~1;     // exchange (float2, even)
    static constexpr int IN = WITH_INPUT ? 2 * W : 0;          // input rows
    using SI = typename RP::template SB<true>;
    // the row's spectrum, held across the planes (spread pass), thread-major
    static constexpr int SP = WITH_INPUT ? 0 : ((SI::U * SI::RAD * RP::T + 1) & ~1);
    static constexpr size_t bytes = (size_t)(XS + IN + 2 * HS + SP) * sizeof(float2) + 2 * sizeof(uint64_t);
};

// If a bulk copy for plane l does not arrive within the bounded wait, the CTA
// waits once more (bounded) for it and for the next plane's copy if that was
// issued, records the timeout in the status word and leaves without writing.
__device__ __forceinline__ void rows_timeout(uint64_t* bar, int l, int L, int* status) {
    if (threadIdx.x == 0) {
        mbar_wait(&bar[l & 1], (l >> 1) & 1);
        if (l + 1 < L) mbar_wait(&bar[(l + 1) & 1], ((l + 1) >> 1) & 1);
        atomicOr(status, STATUS_WAIT_TIMEOUT);
    }
}

// A barrier that nothing completes (two arrivals expected, none made): the
// bounded wait runs out and the status word records it.
__global__ void k_wait_selftest(int* __restrict__ status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);
        mbar_init_fence();
    }
    __syncthreads();
    const bool ok = __syncthreads_and(mbar_wait(&bar, 0));
    if (!ok && threadIdx.x == 0) atomicOr(status, STATUS_WAIT_TIMEOUT);
}

// out[b][c][i] = IDFT( sum_l Hsel_l * DFT(in[b][l][c][i]) )
// (the row plan's MINB caps the registers; shared memory sets the CTAs per SM)
template <bool CONJ, class RP>
__global__ void __launch_bounds__(RP::T, RP::MINBS)
    k_rows_sum_reg(const float2* __restrict__ in, float2* __restrict__ out, int L, int C, int H,
                   const float2* __restrict__ hq, const float2* __restrict__ tw, int* __restrict__ status) {
    using namespace rfft;
    using SM = RowSmem<RP, true>;
    constexpr int W = RP::N, HS = SM::HS;
    using SF = typename RP::template SA<false>;
    using SI = typename RP::template SB<true>;
    extern __shared__ __align__(16) float2 sm[];
    float2* xb = sm;
    float2* rowb = sm + SM::XS;
    float2* hb = rowb + SM::IN;
    uint64_t* bar = reinterpret_cast<uint64_t*>(hb + 2 * HS);
    const int b = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
    const int ky = mirror(i, H);
    const float2* src0 = in + (((size_t)b * L * C + c) * H + i) * W;  // plane 0; planes are C*H*W apart
    const float2* h0 = hq + ((size_t)c * L * (H / 2 + 1) + ky) * HS;  // plane 0; planes are (H/2+1)*HS apart
    const size_t sstep = (size_t)C * H * W, hstep = (size_t)(H / 2 + 1) * HS;
    auto issue = [&](int l, int buf) {
        mbar_expect_tx(&bar[buf], (unsigned)((W + HS) * sizeof(float2)));
        bulk_load(rowb + buf * W, src0 + (size_t)l * sstep, W * sizeof(float2), &bar[buf]);
        bulk_load(hb + buf * HS, h0 + (size_t)l * hstep, HS * sizeof(float2), &bar[buf]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
        issue(0, 0);
        if (L > 1) issue(1, 1);
    }
    __syncthreads();
    float2 acc[SI::U][SI::RAD];
    sfor<SI::U>([&](auto a) { sfor<SI::RAD>([&](auto r) { acc[HCGS_CI(a)][HCGS_CI(r)] = make_float2(0.f, 0.f); }); });
    for (int l = 0; l < L; l++) {
        const int buf = l & 1;
        const bool ok = __syncthreads_and(mbar_wait(&bar[buf], (l >> 1) & 1));
        if (!ok) {
            rows_timeout(bar, l, L, status);
            return;
        }
        const float2* srow = rowb + buf * W;
        const float2* hrow = hb + buf * HS;
        float2 v[SF::U][SF::RAD];
        sfor<SF::U>([&](auto a) {
            constexpr int u = HCGS_CI(a);
            const int j = SF::It::j(u);
            const bool okj = SF::It::valid(u);
            sfor<SF::RAD>([&](auto r) {
                v[u][HCGS_CI(r)] = okj ? srow[j + HCGS_CI(r) * SF::M] : make_float2(0.f, 0.f);
            });
        });
        SF::run(v, xb, tw, [&](auto& vo) {
            static_assert(Shape<decltype(vo)>::R == SI::RAD && Shape<decltype(vo)>::U == SI::U,
                          "the inverse pass must start with the forward pass's last radix");
            sfor<SI::U>([&](auto a) {
                constexpr int u = HCGS_CI(a);
                const int j = SI::It::j(u);
                if (SI::It::valid(u)) {
                    sfor<SI::RAD>([&](auto rr) {
                        constexpr int r = HCGS_CI(rr);
                        float2 h = hrow[mirror(j + r * SI::M, W)];
                        if (CONJ) h.y = -h.y;
                        acc[u][r] = cadd(acc[u][r], cmul(vo[u][r], h));
                    });
                }
            });
        });
        __syncthreads();  // the buffer's rows are consumed
        if (threadIdx.x == 0 && l + 2 < L) {
            fence_proxy_async_smem();
            issue(l + 2, buf);
        }
    }
    float2* dst = out + (((size_t)b * C + c) * H + i) * W;
    SI::run(acc, xb, tw, [&](auto& vo) {
        for_outputs<W, 1, RP::T>(vo, [&](float2 x, int pos, int) { dst[pos] = x; });
    });
}

// out[b][l][c][i] = IDFT( Hsel_l * DFT(in[b][c][i]) )
template <bool CONJ, class RP>
__global__ void __launch_bounds__(RP::T, RP::MINB)
    k_rows_spread_reg(const float2* __restrict__ in, float2* __restrict__ out, int L, int C, int H,
                      const float2* __restrict__ hq, const float2* __restrict__ tw, int* __restrict__ status) {
    using namespace rfft;
    using SM = RowSmem<RP, false>;
    constexpr int W = RP::N, HS = SM::HS;
    using SF = typename RP::template SA<false>;
    using SI = typename RP::template SB<true>;
    extern __shared__ __align__(16) float2 sm[];
    float2* xb = sm;
    float2* hb = sm + SM::XS;
    float2* sp = hb + 2 * HS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sp + SM::SP);
    const int b = blockIdx.x, i = blockIdx.y, c = blockIdx.z;
    const int ky = mirror(i, H);
    const float2* h0 = hq + ((size_t)c * L * (H / 2 + 1) + ky) * HS;
    const size_t hstep = (size_t)(H / 2 + 1) * HS;
    auto issue = [&](int l, int buf) {
        mbar_expect_tx(&bar[buf], (unsigned)(HS * sizeof(float2)));
        bulk_load(hb + buf * HS, h0 + (size_t)l * hstep, HS * sizeof(float2), &bar[buf]);
    };
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
        issue(0, 0);
        if (L > 1) issue(1, 1);
    }
    __syncthreads();
    // the row's spectrum stays in shared memory (each thread its own items,
    // thread-major) rather than in registers across the plane loop
    auto spec = [&](int a, int r) -> float2& { return sp[(a * SI::RAD + r) * RP::T + threadIdx.x]; };
    {
        float2 v[SF::U][SF::RAD];
        load_row<SF>(v, in + (((size_t)b * C + c) * H + i) * W);
        SF::run(v, xb, tw, [&](auto& vo) {
            static_assert(Shape<decltype(vo)>::R == SI::RAD && Shape<decltype(vo)>::U == SI::U,
                          "the inverse pass must start with the forward pass's last radix");
            sfor<SI::U>([&](auto a) {
                sfor<SI::RAD>([&](auto r) { spec(HCGS_CI(a), HCGS_CI(r)) = vo[HCGS_CI(a)][HCGS_CI(r)]; });
            });
        });
    }
    for (int l = 0; l < L; l++) {
        const int buf = l & 1;
        const bool ok = __syncthreads_and(mbar_wait(&bar[buf], (l >> 1) & 1));
        if (!ok) {
            rows_timeout(bar, l, L, status);
            return;
        }
        const float2* hrow = hb + buf * HS;
        float2 v[SI::U][SI::RAD];
        sfor<SI::U>([&](auto a) {
            constexpr int u = HCGS_CI(a);
            const int j = SI::It::j(u);
            const bool okj = SI::It::valid(u);
            sfor<SI::RAD>([&](auto rr) {
                constexpr int r = HCGS_CI(rr);
                float2 h = okj ? hrow[mirror(j + r * SI::M, W)] : make_float2(0.f, 0.f);
                if (CONJ) h.y = -h.y;
                v[u][r] = cmul(spec(u, r), h);
            });
        });
        __syncthreads();  // the transfer-function row is consumed
        if (threadIdx.x == 0 && l + 2 < L) {
            fence_proxy_async_smem();
            issue(l + 2, buf);
        }
        float2* dst = out + ((((size_t)b * L + l) * C + c) * H + i) * W;
        SI::run(v, xb, tw, [&](auto& vo) {
            for_outputs<W, 1, RP::T>(vo, [&](float2 x, int pos, int) { dst[pos] = x; });
        });
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
    const int hw2 = hq_stride(W);
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
    const int hw2 = hq_stride(W);
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
// band_limit = 1 adds the limit of Matsushima and Shimobaba: on an n-sample
// grid du = 1/(n pitch) and H is kept where |f_x| <= 1/(lambda sqrt((2 du_x
// z)^2 + 1)) (likewise for f_y), the region where the sampled phase does not
// alias.
__global__ void k_build_hq(float2* __restrict__ hq, int H, int W, int C, int L, double px, double py, HArgs a,
                           int band_limit) {
    const int hh = H / 2 + 1, ws = hq_stride(W);
    const size_t total = (size_t)C * L * hh * ws;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e % ws);  // kx = W/2 + 1 is row padding (W odd: a mirrored value, never read)
        const int ky = (int)((e / ws) % hh);
        const int l = (int)((e / ((size_t)ws * hh)) % L);
        const int c = (int)(e / ((size_t)ws * hh * L));
        const double fx = kx / (W * px), fy = ky / (H * py);
        const double lam = a.lam[c];
        const double arg = 1.0 / (lam * lam) - (fx * fx + fy * fy);
        bool keep = arg >= 0.0;
        if (band_limit) {
            const double z = a.z[l];
            const double bx = 2.0 * z / (W * px), by = 2.0 * z / (H * py);
            keep = keep && fx <= 1.0 / (lam * sqrt(bx * bx + 1.0)) && fy <= 1.0 / (lam * sqrt(by * by + 1.0));
        }
        float2 h = make_float2(0.f, 0.f);
        if (keep) {
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
    HKey k{o->H, o->W, o->C, o->L, o->band_limit, o->pitch_x, o->pitch_y,
           std::vector<double>(o->wavelength, o->wavelength + o->C), std::vector<double>(o->plane_z, o->plane_z + o->L)};
    auto it = ctx->htab.find(k);
    if (it != ctx->htab.end()) {
        *out = (const float2*)it->second.p;
        return HCGS_OK;
    }
    DevBuf b;
    const size_t n = (size_t)o->C * o->L * (o->H / 2 + 1) * hq_stride(o->W);
    HCGS_CUDA(ctx, cudaMalloc(&b.p, n * sizeof(float2)));
    b.cap = n * sizeof(float2);
    ctx->bytes += b.cap;
    HArgs a{};
    for (int c = 0; c < o->C; c++) a.lam[c] = o->wavelength[c];
    for (int l = 0; l < o->L; l++) a.z[l] = o->plane_z[l];
    HCGS_KERNEL(ctx, "k_build_hq", 0, k_build_hq<<<1184, 256>>>((float2*)b.p, o->H, o->W, o->C, o->L, o->pitch_x, o->pitch_y, a, o->band_limit));
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

template <class CP>
static hcgs_status fft_cols_reg(hcgs_ctx* ctx, const float2* in, float2* out, int nplanes, int W, bool inverse,
                                float scale, const float2* tw, cudaStream_t st) {
    const size_t smem = (size_t)CP::smem_slots() * sizeof(float2);
    const dim3 grid((W + CP::CW - 1) / CP::CW, nplanes);
    if (inverse) {
        HCGS_CUDA(ctx, allow_smem(k_fft_cols_reg<true, CP>, smem));
        HCGS_KERNEL(ctx, "k_fft_cols", st, k_fft_cols_reg<true, CP><<<grid, CP::T, smem, st>>>(in, out, W, tw, scale));
    } else {
        HCGS_CUDA(ctx, allow_smem(k_fft_cols_reg<false, CP>, smem));
        HCGS_KERNEL(ctx, "k_fft_cols", st, k_fft_cols_reg<false, CP><<<grid, CP::T, smem, st>>>(in, out, W, tw, scale));
    }
    HCGS_LAUNCH(ctx, "k_fft_cols");
    return HCGS_OK;
}

hcgs_status fft_cols(hcgs_ctx* ctx, const float2* in, float2* out, int nplanes, int H, int W, bool inverse,
                     float scale, cudaStream_t st) {
    if (nplanes <= 0) return HCGS_OK;
    FftPlan* p;
    hcgs_status s = get_plan(ctx, H, &p);
    if (s) return s;
    if (H == 1080) return fft_cols_reg<rfft::Cols1080>(ctx, in, out, nplanes, W, inverse, scale, p->tw, st);
    if (H == 1920) return fft_cols_reg<rfft::Cols1920>(ctx, in, out, nplanes, W, inverse, scale, p->tw, st);
    if (H == 512) return fft_cols_reg<rfft::Cols512>(ctx, in, out, nplanes, W, inverse, scale, p->tw, st);
    if (H == 256) return fft_cols_reg<rfft::Cols256>(ctx, in, out, nplanes, W, inverse, scale, p->tw, st);
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

template <class CP>
static hcgs_status cols_focal_loss_reg(hcgs_ctx* ctx, float2* data, const float* I_gt, float* I_out,
                                       float* partials, int nplanes, int W, float inv_count, float scale,
                                       int* nblocks_out, const float2* tw, cudaStream_t st) {
    const size_t smem = (size_t)CP::smem_slots() * sizeof(float2);
    const dim3 grid((W + CP::CW - 1) / CP::CW, nplanes);
    *nblocks_out = grid.x * grid.y;
    if (!partials) return HCGS_OK;  // size query
    HCGS_CUDA(ctx, allow_smem(k_cols_focal_loss_reg<CP>, smem));
    HCGS_KERNEL(ctx, "k_cols_focal_loss", st, k_cols_focal_loss_reg<CP><<<grid, CP::T, smem, st>>>(data, I_gt, I_out, partials, W, tw, scale, inv_count));
    HCGS_LAUNCH(ctx, "k_cols_focal_loss");
    return HCGS_OK;
}

hcgs_status cols_focal_loss(hcgs_ctx* ctx, float2* data, const float* I_gt, float* I_out, float* partials,
                            int nplanes, int H, int W, float inv_count, float scale, int* nblocks_out,
                            cudaStream_t st) {
    FftPlan* p;
    hcgs_status s = get_plan(ctx, H, &p);
    if (s) return s;
    if (H == 1080)
        return cols_focal_loss_reg<rfft::Cols1080>(ctx, data, I_gt, I_out, partials, nplanes, W, inv_count, scale,
                                                   nblocks_out, p->tw, st);
    if (H == 1920)
        return cols_focal_loss_reg<rfft::Cols1920>(ctx, data, I_gt, I_out, partials, nplanes, W, inv_count, scale,
                                                   nblocks_out, p->tw, st);
    if (H == 512)
        return cols_focal_loss_reg<rfft::Cols512>(ctx, data, I_gt, I_out, partials, nplanes, W, inv_count, scale,
                                                  nblocks_out, p->tw, st);
    if (H == 256)
        return cols_focal_loss_reg<rfft::Cols256>(ctx, data, I_gt, I_out, partials, nplanes, W, inv_count, scale,
                                                  nblocks_out, p->tw, st);
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

template <class RP>
static hcgs_status rows_reg(hcgs_ctx* ctx, bool sum, const float2* in, float2* out, int B, int L, int C, int H,
                            const float2* hq, bool conjH, const float2* tw, cudaStream_t st) {
    const dim3 grid(B, H, C);
    int* status = ctx->d_status;
    if (sum) {
        const size_t smem = RowSmem<RP, true>::bytes;
        if (conjH) {
            HCGS_CUDA(ctx, allow_smem(k_rows_sum_reg<true, RP>, smem));
            HCGS_KERNEL(ctx, "k_rows_sum", st, k_rows_sum_reg<true, RP><<<grid, RP::T, smem, st>>>(in, out, L, C, H, hq, tw, status));
        } else {
            HCGS_CUDA(ctx, allow_smem(k_rows_sum_reg<false, RP>, smem));
            HCGS_KERNEL(ctx, "k_rows_sum", st, k_rows_sum_reg<false, RP><<<grid, RP::T, smem, st>>>(in, out, L, C, H, hq, tw, status));
        }
        HCGS_LAUNCH(ctx, "k_rows_sum");
    } else {
        const size_t smem = RowSmem<RP, false>::bytes;
        if (conjH) {
            HCGS_CUDA(ctx, allow_smem(k_rows_spread_reg<true, RP>, smem));
            HCGS_KERNEL(ctx, "k_rows_spread", st, k_rows_spread_reg<true, RP><<<grid, RP::T, smem, st>>>(in, out, L, C, H, hq, tw, status));
        } else {
            HCGS_CUDA(ctx, allow_smem(k_rows_spread_reg<false, RP>, smem));
            HCGS_KERNEL(ctx, "k_rows_spread", st, k_rows_spread_reg<false, RP><<<grid, RP::T, smem, st>>>(in, out, L, C, H, hq, tw, status));
        }
        HCGS_LAUNCH(ctx, "k_rows_spread");
    }
    return HCGS_OK;
}

static bool rows_reg_dispatch(hcgs_ctx* ctx, bool sum, const float2* in, float2* out, int B, int L, int C, int H,
                              int W, const float2* hq, bool conjH, const float2* tw, cudaStream_t st,
                              hcgs_status* res) {
    if (W == 1920) { *res = rows_reg<rfft::Rows1920>(ctx, sum, in, out, B, L, C, H, hq, conjH, tw, st); return true; }
    if (W == 1080) { *res = rows_reg<rfft::Rows1080>(ctx, sum, in, out, B, L, C, H, hq, conjH, tw, st); return true; }
    if (W == 512) { *res = rows_reg<rfft::Rows512>(ctx, sum, in, out, B, L, C, H, hq, conjH, tw, st); return true; }
    if (W == 256) { *res = rows_reg<rfft::Rows256>(ctx, sum, in, out, B, L, C, H, hq, conjH, tw, st); return true; }
    return false;
}

hcgs_status rows_sum(hcgs_ctx* ctx, const float2* in, float2* out, int B, int L, int C, int H, int W,
                     const float2* hq, bool conjH, cudaStream_t st) {
    FftPlan* p;
    hcgs_status s = get_plan(ctx, W, &p);
    if (s) return s;
    if (rows_reg_dispatch(ctx, true, in, out, B, L, C, H, W, hq, conjH, p->tw, st, &s)) return s;
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
    if (rows_reg_dispatch(ctx, false, in, out, B, L, C, H, W, hq, conjH, p->tw, st, &s)) return s;
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
// Zero embedding of P planes of H x W into 2H x 2W (field at rows H/2 ..,
// columns W/2 ..), and the crop of that window back.
__global__ void k_zero_pad(const float2* __restrict__ in, float2* __restrict__ out, int64_t P, int H, int W) {
    const int W2 = 2 * W, H2 = 2 * H, oy = H / 2, ox = W / 2;
    const int64_t total = P * H2 * W2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % W2), y = (int)((i / W2) % H2);
        const int64_t p = i / ((int64_t)W2 * H2);
        const int yy = y - oy, xx = x - ox;
        out[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? in[(p * H + yy) * W + xx] : make_float2(0.f, 0.f);
    }
}

__global__ void k_crop(const float2* __restrict__ in, float2* __restrict__ out, int64_t P, int H, int W) {
    const int oy = H / 2, ox = W / 2;
    const int64_t total = P * H * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % W), y = (int)((i / W) % H);
        const int64_t p = i / ((int64_t)W * H);
        out[i] = in[(p * 2 * H + y + oy) * 2 * W + x + ox];
    }
}

static hcgs_status pad_planes(hcgs_ctx* ctx, const float2* in, float2* out, int64_t P, int H, int W, cudaStream_t st) {
    const int64_t total = P * 4 * H * W;
    const int blocks = (int)std::min<int64_t>(148 * 16, (total + 255) / 256);
    HCGS_KERNEL(ctx, "k_zero_pad", st, k_zero_pad<<<blocks, 256, 0, st>>>(in, out, P, H, W));
    return HCGS_OK;
}

static hcgs_status crop_planes(hcgs_ctx* ctx, const float2* in, float2* out, int64_t P, int H, int W, cudaStream_t st) {
    const int64_t total = P * H * W;
    const int blocks = (int)std::min<int64_t>(148 * 16, (total + 255) / 256);
    HCGS_KERNEL(ctx, "k_crop", st, k_crop<<<blocks, 256, 0, st>>>(in, out, P, H, W));
    return HCGS_OK;
}

static hcgs_optics padded_optics(const hcgs_optics* o) {
    hcgs_optics q = *o;
    q.H = 2 * o->H;
    q.W = 2 * o->W;
    q.padding = 0;
    return q;
}

hcgs_status asm_sum(hcgs_ctx* ctx, const float2* in, float2* out, int B, const hcgs_optics* o, bool conjH,
                    cudaStream_t st) {
    if (o->padding) {
        // linear convolution: embed, propagate and sum on the 2H x 2W grid, crop
        const hcgs_optics q = padded_optics(o);
        const size_t n4 = (size_t)4 * o->H * o->W;
        HCGS_CUDA(ctx, grow(ctx, ctx->ws[6], (size_t)B * o->L * o->C * n4 * sizeof(float2), &ctx->bytes));
        HCGS_CUDA(ctx, grow(ctx, ctx->ws[7], (size_t)B * o->C * n4 * sizeof(float2), &ctx->bytes));
        float2* pin = (float2*)ctx->ws[6].p;
        float2* pout = (float2*)ctx->ws[7].p;
        hcgs_status s;
        if ((s = pad_planes(ctx, in, pin, (int64_t)B * o->L * o->C, o->H, o->W, st))) return s;
        if ((s = asm_sum(ctx, pin, pout, B, &q, conjH, st))) return s;
        return crop_planes(ctx, pout, out, (int64_t)B * o->C, o->H, o->W, st);
    }
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
    if (o->padding) {
        const hcgs_optics q = padded_optics(o);
        const size_t n4 = (size_t)4 * o->H * o->W;
        HCGS_CUDA(ctx, grow(ctx, ctx->ws[6], (size_t)B * o->C * n4 * sizeof(float2), &ctx->bytes));
        HCGS_CUDA(ctx, grow(ctx, ctx->ws[7], (size_t)B * o->L * o->C * n4 * sizeof(float2), &ctx->bytes));
        float2* pin = (float2*)ctx->ws[6].p;
        float2* pout = (float2*)ctx->ws[7].p;
        hcgs_status s;
        if ((s = pad_planes(ctx, in, pin, (int64_t)B * o->C, o->H, o->W, st))) return s;
        if ((s = asm_spread(ctx, pin, pout, B, &q, conjH, st))) return s;
        return crop_planes(ctx, pout, out, (int64_t)B * o->L * o->C, o->H, o->W, st);
    }
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
                                int band_limit, cudaStream_t st) {
    const size_t n = (size_t)C * L * (H / 2 + 1) * hq_stride(W);
    const int blocks = (int)std::min<size_t>(1184, (n + 255) / 256);
    k_build_hq<<<blocks, 256, 0, st>>>(hq, H, W, C, L, px, py, a, band_limit);
    return cudaGetLastError();
}

}  // namespace hcgs

extern "C" hcgs_status hcgs_selftest_wait_timeout(hcgs_ctx* ctx, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    hcgs::k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->d_status);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HCGS_OK : hcgs::cuda_err(ctx, e, "k_wait_selftest");
}
