// Step 3 of the render path on sm_103a: complex multi-plane compositing
// (Sec. 4.1 per-plane field equation; Algorithm 2) and its adjoint (Supp. D.4;
// Sec. 4.2: back-to-front walk, transmittance recovered by division).
//
// One CTA of one warp per (16 x 8 pixel strip, plane, view): a 16x16 tile
// is two strips, and a strip's tile lies in one 64x64 bucket of the plane's
// binning.  Four pixels per thread (one column, rows r, r + 2, r + 4, r + 6
// of the strip), evaluated as two packed FP32x2 pairs.  The warp streams the
// bucket's list (in visiting order) 32 entries at a time, keeps the entries
// whose tile rectangle covers its tile and whose footprint can reach its
// strip (exact superset test), compacts them in order into shared-memory
// slots (warp ballot), and every pixel takes the step of Algorithm 2 for
// each of them: alpha = min(alpha_max, o exp(-power)); skip when alpha <
// alpha_min; U += w alpha T; T *= 1 - alpha; stop once T < T_eps.  The warp
// leaves the list as soon as its pixels have all stopped, and writes the ids
// it kept (the strip's list) for the adjoint.
//
// The alpha arithmetic uses explicitly rounded intrinsics so that the forward
// and backward kernels take identical skip/stop decisions.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"
#include "project.cuh"

namespace hcgs {

struct RasterArgs {
    const float4* rec;
    const uint2* rects;
    const uint32_t* off;
    const uint32_t* list;
    const uint32_t* sortid;  // [V][N] Gaussian id at visiting rank
    uint32_t* slist;
    int V, N, L, H, W, tilesX, tilesY, ctX, ctY;
    float amin, amax, teps;
    float inv_amin;  // 1 / alpha_min (0 when alpha_min = 0)
    uint32_t M;      // bucket instances (device checks of the bounds-checked build)
    int* status;     // device status word
};

static RasterArgs make_raster_args(const hcgs_saved* s) {
    RasterArgs a;
    a.rec = (const float4*)s->rec.p;
    a.rects = (const uint2*)s->rects.p;
    a.off = (const uint32_t*)s->bcount.p;
    a.list = s->list;
    a.sortid = (const uint32_t*)s->sortid.p;
    a.slist = (uint32_t*)s->slist.p;
    a.V = s->V; a.N = s->N; a.L = s->L; a.H = s->H; a.W = s->W;
    a.tilesX = s->tilesX; a.tilesY = s->tilesY; a.ctX = s->ctX; a.ctY = s->ctY;
    a.amin = s->opts.alpha_min; a.amax = s->opts.alpha_max; a.teps = s->opts.T_eps;
    a.inv_amin = a.amin > 0.f ? 1.f / a.amin : 0.f;
    a.M = (uint32_t)s->M;
    a.status = nullptr;
    return a;
}

// power = 1/2 (A dx^2 + C dy^2) + B dx dy, d = pixel - mu (Supp. D.3 exponent term)
__device__ __forceinline__ float footprint_power(float px, float py, float4 r0, float Cc, float* dxo, float* dyo) {
    const float dx = __fsub_rn(px, r0.x), dy = __fsub_rn(py, r0.y);
    float p = __fmul_rn(0.5f, __fmaf_rn(r0.z, __fmul_rn(dx, dx), __fmul_rn(Cc, __fmul_rn(dy, dy))));
    p = __fmaf_rn(r0.w, __fmul_rn(dx, dy), p);
    *dxo = dx;
    *dyo = dy;
    return p;
}

template <int C>
struct RecW {
    static __device__ __forceinline__ float2 get(const float4* r, int c) {
        if (c == 0) return make_float2(r[1].z, r[1].w);
        if (c == 1) return make_float2(r[2].x, r[2].y);
        if (c == 2) return make_float2(r[2].z, r[2].w);
        return make_float2(r[3].x, r[3].y);
    }
};

constexpr int RT = 32;  // one warp per CTA: one 16 x 8 strip

// Start of a strip's kept-id list: bucket list offset beg, length n; the
// bucket's 32 strips (4 x 4 tiles, two strips each) take consecutive slices
// of n entries.  srow = strip row (tile row * 2 + half).
__device__ __forceinline__ size_t strip_list_base(uint32_t beg, uint32_t n, int tx, int srow) {
    const int local = ((srow >> 1) % COARSE * COARSE + tx % COARSE) * 2 + (srow & 1);
    return (size_t)COARSE * COARSE * 2 * beg + (size_t)local * n;
}

// Can Gaussian (mu, conic A B C, opacity o) reach alpha >= alpha_min at any
// pixel centre of the strip x in [x0, x0 + 15], y in [y0, y0 + 7]?  The
// footprint quadratic q = A dx^2 + 2 B dx dy + C dy^2 is minimised over the
// strip's (continuous) box and compared with 2 ln(o / alpha_min), with a
// relative and absolute margin far above FP32 rounding: zero when the centre
// lies in the box, else the minimum of the convex q lies on an edge, where it
// is a 1D convex problem (the unconstrained minimiser clamped to the edge).
// The box contains every pixel centre of the strip, so this never rejects a
// pixel that the per-pixel test would accept: skipping is exact.
__device__ __forceinline__ bool strip_hits(float4 r0, float Cc, float o, float x0, float y0, float amin,
                                           float inv_amin) {
    if (amin <= 0.f) return true;
    if (o < amin) return false;
    const float x1 = x0 + 15.f, y1 = y0 + 7.f;
    if (r0.x >= x0 && r0.x <= x1 && r0.y >= y0 && r0.y <= y1) return true;
    const float k2 = 2.f * __logf(o * inv_amin) * 1.001f + 1e-3f;
    const float A = r0.z, B = r0.w;
    const float sx = __fdividef(B, A), sy = __fdividef(B, Cc);
    auto q = [&](float dx, float dy) { return fmaf(A * dx, dx, fmaf(2.f * B * dx, dy, Cc * dy * dy)); };
    float m;
    {   // horizontal edges y = y0, y1
        const float d0 = y0 - r0.y, d1 = y1 - r0.y;
        const float e0 = fminf(fmaxf(r0.x - sx * d0, x0), x1) - r0.x;
        const float e1 = fminf(fmaxf(r0.x - sx * d1, x0), x1) - r0.x;
        m = fminf(q(e0, d0), q(e1, d1));
    }
    {   // vertical edges x = x0, x1
        const float d0 = x0 - r0.x, d1 = x1 - r0.x;
        const float e0 = fminf(fmaxf(r0.y - sy * d0, y0), y1) - r0.y;
        const float e1 = fminf(fmaxf(r0.y - sy * d1, y0), y1) - r0.y;
        m = fminf(m, fminf(q(d0, e0), q(d1, e1)));
    }
    return m <= k2;
}

// In the reduced-precision tiers, entries of opacity above this are still
// evaluated in FP32: the adjoint's dL/dalpha carries S / (1 - alpha), which
// multiplies the relative error of a reduced-precision alpha by
// alpha / (1 - alpha) (3 at alpha = 0.75, 99 at 0.99).  The choice depends
// on the record alone, so the forward and the adjoint make it alike.
constexpr float TIER_FP32_OPACITY = 0.75f;
template <int FT>
__device__ __forceinline__ bool tier_half(float o) {
    return FT != 0 && o <= TIER_FP32_OPACITY;
}

// Per-entry coefficients staged with the record.  FP32 evaluation: the
// base-2 exponent of o G = 2^(A' dx^2 + B' dx dy + C' dy^2 + log2 o).
// Reduced precision (tier_half): the normalised-frame factors sqrt(A),
// sqrt(C) and rho2 = 2 B / sqrt(A C).
template <int FT>
__device__ __forceinline__ float4 entry_coeffs(float4 q0, float4 q1) {
    if (tier_half<FT>(q1.y)) {
        const float sa = sqrtf(q0.z), sc = sqrtf(q1.x);
        return make_float4(sa, sc, 2.f * q0.w / (sa * sc), 0.f);
    }
    constexpr float L2E = 1.4426950408889634f;
    return make_float4(-0.5f * L2E * q0.z, -L2E * q0.w, -0.5f * L2E * q1.x, __log2f(q1.y));
}

// Stream 32 list positions [p0, p0 + 32) of the bucket for one warp: keep the
// entries whose rectangle covers tile (tx, ty) and whose footprint can reach
// the warp's strip, and compact them, in list order, into the warp's slots.
// Returns the number kept.  PF: the caller has already loaded the lane's
// list entry (s_pf) for position p0 + lane.
template <int NR, int FT, bool PF = false>
__device__ __forceinline__ int stage_warp(const RasterArgs& a, size_t vN, uint32_t beg, uint32_t p0, uint32_t n,
                                          int tx, int ty, float sx0, float sy0, float4 (*wrec)[NR + 1],
                                          uint32_t* wpos, uint32_t* wid, uint32_t* kept, uint32_t s_pf = 0u) {
    const int lane = threadIdx.x & 31;
    const uint32_t p = p0 + (uint32_t)lane;
    bool ok = false;
    uint32_t s = 0;
    float4 q0, q1;
    if (p < n && HCGS_DCHECK(a.status, beg + p < a.M)) {
        s = PF ? s_pf : a.list[beg + p];
        if (!HCGS_DCHECK(a.status, s < (uint32_t)a.N)) s = 0u;  // checked build: a stray rank reads entry 0
        const uint2 rc = a.rects[vN + s];
        ok = (uint32_t)tx >= (rc.x & 0xFFFFu) && (uint32_t)tx < (rc.x >> 16) && (uint32_t)ty >= (rc.y & 0xFFFFu) &&
             (uint32_t)ty < (rc.y >> 16);
        if (ok) {
            const float4* r = a.rec + (vN + s) * NR;
            q0 = r[0];
            q1 = r[1];
            ok = strip_hits(q0, q1.x, q1.y, sx0, sy0, a.amin, a.inv_amin);
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if (ok) {
        const int slot = __popc(m & ((1u << lane) - 1u));
        const float4* r = a.rec + (vN + s) * NR;
        wrec[slot][0] = q0;
        wrec[slot][1] = q1;
#pragma unroll
        for (int k = 2; k < NR; k++) wrec[slot][k] = r[k];
        wrec[slot][NR] = entry_coeffs<FT>(q0, q1);
        wpos[slot] = p;
        wid[slot] = s;
        kept[slot] = s;
    }
    __syncwarp();
    return __popc(m);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// The thread's pixels against one Gaussian record.  With d = pixel - mu the
// exponent term is power = 1/2 (A dx^2 + C dy^2) + B dx dy (Supp. D.3) and
// o G = o exp(-power) = 2^(A' dx^2 + B' dx dy + C' dy^2 + log2 o), with the
// coefficients A' B' C' log2 o prepared once per staged entry (k) and the
// dx terms once per entry and thread (t0 = A' dx^2 + log2 o, bdx = B' dx);
// alpha = min(alpha_max, o G).

// alpha = min(alpha_max, o G) needs the clamp only for entries whose opacity
// comes near alpha_max: below alpha_max (1 - 2^-10), o G <= o stays below
// alpha_max up to the rounding of the evaluation, and alpha = o G as evaluated.
// The choice is per entry (warp-uniform), so the forward and the adjoint
// evaluate every entry the same way.
__device__ __forceinline__ bool may_clamp(float o, float amax) { return o > amax * 0.9990234375f; }

// Reduced-precision footprint (the FP16x2 tier): the same quantities, with the
// exponent and exp() evaluated in packed half precision.  To stay well
// conditioned for footprints of any size the quadratic is formed in the
// footprint's normalised frame, u = dx sqrt(A), v = dy sqrt(C),
// q = u^2 + 2 rho u v + v^2 with rho = B / sqrt(A C) in (-1, 1), all O(1)
// inside the support.  The thread's pixels share a column, so u is fixed per
// thread and entry, and completing the square in v splits the exponent
// -q log2(e) / 2 = -c (1 - rho^2) u^2 - c w^2 (c = log2(e) / 2, w = v + rho u):
// the first part, constant along the column, is taken in FP32 into the
// factor o 2^(-c (1 - rho^2) u^2) once per thread and entry; only -c w^2,
// never larger in magnitude than the whole exponent, and its exp() run in
// packed half precision per pixel pair.  Accumulation stays FP32.
template <int FT>
struct Half2Of;
template <>
struct Half2Of<1> {
    using T = __half2;
    static __device__ __forceinline__ T from(float x) { return __float2half2_rn(x); }
    static __device__ __forceinline__ T from2(float2 x) { return __float22half2_rn(x); }
    static __device__ __forceinline__ float2 to2(T x) { return __half22float2(x); }
};
template <>
struct Half2Of<2> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ T from(float x) { return __float2bfloat162_rn(x); }
    static __device__ __forceinline__ T from2(float2 x) { return __float22bfloat162_rn(x); }
    static __device__ __forceinline__ float2 to2(T x) { return __bfloat1622float2(x); }
};

// One pixel pair: w' = sqrt(c) (dy sqrt(C) + rho u), then F 2^(-w'^2) with
// the per-thread factor F = o 2^(-c (1 - rho^2) u^2); scs = sqrt(c C),
// rus = sqrt(c) rho u.
template <int FT, bool CL>
__device__ __forceinline__ void eval_pair_h(float2 py2, float4 r0, float scs, float rus, float F, float amax,
                                            float2& dy2, float2& og2, float2& a2) {
    dy2 = __fadd2_rn(py2, f2(-r0.y));
    const auto w = Half2Of<FT>::from2(__ffma2_rn(dy2, f2(scs), f2(rus)));
    const auto e = __hmul2(__hneg2(w), w);
    const float2 G2 = Half2Of<FT>::to2(h2exp2(e));
    og2 = __fmul2_rn(f2(F), G2);
    a2 = CL ? make_float2(fminf(amax, og2.x), fminf(amax, og2.y)) : og2;
}

// Per-entry, per-thread part of the evaluation (the pixel column is fixed):
// dx and, for the FP32 tier, t0 = A' dx^2 + log2 o and bdx = B' dx.
struct EntryX {
    float dx, t0, bdx;
};
__device__ __forceinline__ EntryX entry_x(float px, float4 r0, float4 k) {
    EntryX x;
    x.dx = __fsub_rn(px, r0.x);
    x.t0 = __fmaf_rn(k.x, __fmul_rn(x.dx, x.dx), k.w);
    x.bdx = __fmul_rn(k.y, x.dx);
    return x;
}

// Both pixel pairs of a thread (rows r, r+2 and r+4, r+6 of its column).  In
// the FP32 tier the exponent is quadratic in dy, so the second pair follows
// from the first by a linear correction: e(dy + 4) - e(dy) = 4 B' dx +
// 16 C' + 8 C' dy (two packed operations instead of four).  Forward and
// adjoint both evaluate through here, so they take identical decisions.  CL:
// the entry may reach the clamp (may_clamp).
template <int FT, bool CL>
__device__ __forceinline__ void eval_entry(const EntryX& x, float2 pyA, float2 pyB, float4 r0, float4 r1, float4 k,
                                           float amax, float2& dyA, float2& ogA, float2& aA, float2& dyB,
                                           float2& ogB, float2& aB) {
    if (tier_half<FT>(r1.y)) {
        // half (FT 1) or bfloat16 (FT 2) precision for -c w^2 and its exp();
        // u = dx sqrt(A) and the factor F are fixed per thread and entry
        const float u = x.dx * k.x;
        constexpr float c = 0.72134752044448170f;  // log2(e) / 2
        constexpr float sqc = 0.84932180028801904f;  // sqrt(c)
        const float ru = 0.5f * k.z * u;            // rho u (k.z = 2 rho)
        const float F = r1.y * ex2_approx(c * fmaf(ru, ru, -u * u));
        eval_pair_h<FT == 0 ? 1 : FT, CL>(pyA, r0, sqc * k.y, sqc * ru, F, amax, dyA, ogA, aA);
        eval_pair_h<FT == 0 ? 1 : FT, CL>(pyB, r0, sqc * k.y, sqc * ru, F, amax, dyB, ogB, aB);
    } else {
        dyA = __fadd2_rn(pyA, f2(-r0.y));
        float2 e = __ffma2_rn(f2(x.bdx), dyA, f2(x.t0));
        e = __ffma2_rn(__fmul2_rn(f2(k.z), dyA), dyA, e);
        const float kc = __fmaf_rn(16.f, k.z, __fmul_rn(4.f, x.bdx));
        const float2 eB = __fadd2_rn(e, __ffma2_rn(f2(8.f * k.z), dyA, f2(kc)));
        dyB = __fadd2_rn(dyA, f2(4.f));
        ogA = make_float2(ex2_approx(e.x), ex2_approx(e.y));
        ogB = make_float2(ex2_approx(eB.x), ex2_approx(eB.y));
        aA = CL ? make_float2(fminf(amax, ogA.x), fminf(amax, ogA.y)) : ogA;
        aB = CL ? make_float2(fminf(amax, ogB.x), fminf(amax, ogB.y)) : ogB;
    }
}

// Warp reduce-scatter of 16 values: afterwards lanes 2i and 2i+1 both hold the
// warp-wide sum of value i (16 shuffles instead of 80 for a full butterfly).
__device__ __forceinline__ float warp_reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
    for (int half = 8, off = 16; half >= 1; half >>= 1, off >>= 1) {
        const bool up = lane & off;
#pragma unroll
        for (int i = 0; i < half; i++) {
            const float send = up ? v[i] : v[i + half];
            const float keep = up ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Forward step of a pixel pair that takes it (c0/c1) for one record: a pixel
// that does not take it gets alpha 0 (no add, T unchanged).
template <int C>
__device__ __forceinline__ void fwd_pair(const float4* rec, float2 a2, bool c0, bool c1, float2& T2,
                                         float2 (&accX)[C], float2 (&accY)[C]) {
    const float2 al = make_float2(c0 ? a2.x : 0.f, c1 ? a2.y : 0.f);
    const float2 wt = __fmul2_rn(al, T2);
#pragma unroll
    for (int c = 0; c < C; c++) {
        const float2 w = RecW<C>::get(rec, c);
        accX[c] = __ffma2_rn(f2(w.x), wt, accX[c]);
        accY[c] = __ffma2_rn(f2(w.y), wt, accY[c]);
    }
    T2 = __fadd2_rn(T2, make_float2(-wt.x, -wt.y));  // T (1 - alpha)
}

// A pixel is still compositing while T >= T_eps (T only changes when the
// pixel takes a step, so this is the "stop once T < T_eps" rule); pixels
// outside the image start with T = 0.
template <int C, int FT, bool NCOUNT>
__global__ void __launch_bounds__(RT, 32) k_raster_fwd(RasterArgs a, float2* __restrict__ U, float* __restrict__ Tsave,
                                                   uint32_t* __restrict__ lastsave, float* __restrict__ Tout,
                                                   int32_t* __restrict__ ncout) {
    constexpr int NR = C <= 1 ? 2 : (C <= 3 ? 3 : 4);
    __shared__ float4 srec[32][NR + 1];
    __shared__ uint32_t spos[32], sid[32];
    const int lane = threadIdx.x;
    const int strip = blockIdx.x, l = blockIdx.y, v = blockIdx.z;
    const int tx = strip % a.tilesX, ty = (strip / a.tilesX) >> 1;  // this warp's tile
    const int px = tx * TILE + (lane & 15);
    const int sy = ty * TILE + 8 * ((strip / a.tilesX) & 1);  // this warp's 16 x 8 strip starts at row sy
    const int py = sy + (lane >> 4);                 // rows py, py + 2, py + 4, py + 6
    const bool colin = px < a.W;
    const float sx0 = (float)(tx * TILE), sy0 = (float)sy;
    const uint32_t gb = ((uint32_t)(v * a.L + l) * a.ctY + ty / COARSE) * a.ctX + tx / COARSE;
    const uint32_t beg = a.off[gb], n = a.off[gb + 1] - beg;
    const size_t vN = (size_t)v * a.N;
    const float fpx = (float)px;
    const float teps = a.teps;
    // this strip's slice of the kept-id lists: the 32 strips of a bucket each
    // have room for the bucket's whole list
    uint32_t* kept = a.slist + strip_list_base(beg, n, tx, strip / a.tilesX);
    uint32_t nkept = 0;
    const float2 pyA = make_float2((float)py, (float)(py + 2)), pyB = make_float2((float)(py + 4), (float)(py + 6));
    float2 TA = make_float2(colin && py < a.H ? 1.f : 0.f, colin && py + 2 < a.H ? 1.f : 0.f);
    float2 TB = make_float2(colin && py + 4 < a.H ? 1.f : 0.f, colin && py + 6 < a.H ? 1.f : 0.f);
    float2 aAX[C], aAY[C], aBX[C], aBY[C];
#pragma unroll
    for (int c = 0; c < C; c++) aAX[c] = aAY[c] = aBX[c] = aBY[c] = f2(0.f);
    uint32_t last[4] = {0, 0, 0, 0};
    int nc[4] = {0, 0, 0, 0};
    // the list entry of the next batch is loaded one batch ahead
    uint32_t s_pf = (uint32_t)lane < n && HCGS_DCHECK(a.status, beg + lane < a.M) ? a.list[beg + lane] : 0u;
    for (uint32_t p0 = 0; p0 < n; p0 += 32) {
        const bool live = TA.x >= teps || TA.y >= teps || TB.x >= teps || TB.y >= teps;
        if (!__any_sync(0xffffffffu, live)) break;
        const uint32_t s_cur = s_pf;
        if (p0 + 32u + (uint32_t)lane < n && HCGS_DCHECK(a.status, beg + p0 + 32u + lane < a.M))
            s_pf = a.list[beg + p0 + 32u + (uint32_t)lane];
        const int nh = stage_warp<NR, FT, true>(a, vN, beg, p0, n, tx, ty, sx0, sy0, srec, spos, sid, kept + nkept,
                                                s_cur);
        for (int k = 0; k < nh; k++) {
            const float4* rec = srec[k];
            const float4 r0 = rec[0], r1 = rec[1], kk = rec[NR];
            const uint32_t pos1 = nkept + (uint32_t)k + 1u;  // staged index + 1
            auto step = [&](auto cl) {
                const EntryX x = entry_x(fpx, r0, kk);
                float2 dyA, ogA, aA, dyB, ogB, aB;
                eval_entry<FT, decltype(cl)::value>(x, pyA, pyB, r0, r1, kk, a.amax, dyA, ogA, aA, dyB, ogB, aB);
                const bool c0 = TA.x >= teps && aA.x >= a.amin, c1 = TA.y >= teps && aA.y >= a.amin;
                const bool c2 = TB.x >= teps && aB.x >= a.amin, c3 = TB.y >= teps && aB.y >= a.amin;
                fwd_pair<C>(rec, aA, c0, c1, TA, aAX, aAY);
                last[0] = c0 ? pos1 : last[0];
                last[1] = c1 ? pos1 : last[1];
                if (NCOUNT) { nc[0] += c0; nc[1] += c1; }
                fwd_pair<C>(rec, aB, c2, c3, TB, aBX, aBY);
                last[2] = c2 ? pos1 : last[2];
                last[3] = c3 ? pos1 : last[3];
                if (NCOUNT) { nc[2] += c2; nc[3] += c3; }
            };
            if (may_clamp(r1.y, a.amax)) step(std::true_type{});
            else step(std::false_type{});
        }
        nkept += (uint32_t)nh;
        __syncwarp();
    }
    const size_t plane = (size_t)v * a.L + l;
    const size_t HW = (size_t)a.H * a.W;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (!(colin && py + 2 * q < a.H)) continue;
        const size_t pix = (size_t)(py + 2 * q) * a.W + px;
        const float T = q == 0 ? TA.x : q == 1 ? TA.y : q == 2 ? TB.x : TB.y;
#pragma unroll
        for (int c = 0; c < C; c++) {
            const float2 vv = q == 0 ? make_float2(aAX[c].x, aAY[c].x)
                            : q == 1 ? make_float2(aAX[c].y, aAY[c].y)
                            : q == 2 ? make_float2(aBX[c].x, aBY[c].x)
                                     : make_float2(aBX[c].y, aBY[c].y);
            U[(plane * C + c) * HW + pix] = vv;
        }
        Tsave[plane * HW + pix] = T;
        lastsave[plane * HW + pix] = last[q];
        if (Tout) Tout[plane * HW + pix] = T;
        if (NCOUNT) ncout[plane * HW + pix] = nc[q];
    }
}

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Adjoint step of a pixel pair (c0/c1: the pixels that took this step in the
// forward) walking back-to-front (Sec. 4.2): T_k = T_{k+1} / (1 - alpha_k);
// dL/dalpha_k = sum_c Re(conj(g_c) (w_kc T_k - S_kc / (1 - alpha_k))) with
// S_k = sum_{m>k} w_m alpha_m T_m.  Since g is fixed per pixel, only the
// scalar B = sum_c Re(conj(g_c) S_c) is carried: dL/dalpha_k = T_k A_k -
// B / (1 - alpha_k) and B <- B + alpha_k T_k A_k, A_k = sum_c Re(conj(g_c) w_kc).
// Adds to the packed accumulators (one lane per pixel): dL/dw_c (gw) and the
// moments of p = -dL/dpower over the pixels, S0 = sum p, Sy = sum p dy,
// Syy = sum p dy^2; all pixels of a thread share dx, so the thread's
// gradients of mu and the conic follow from the moments once per entry.
// The reciprocal of 1 - alpha only scales gradients (no decision depends on
// it), so the hardware approximation is used.  CL as in eval_entry: for an
// entry that cannot reach the clamp the masked alpha is o G at the pixels that
// took the step and 0 elsewhere, so p = dL/dalpha * alpha.
template <int C, bool FIRST, bool CL>
__device__ __forceinline__ void bwd_pair(const float4* rec, float2 dy2, float2 og2, float2 a2, bool c0, bool c1,
                                         float amax, float2& T2, float2& B2, const float2 (&gX)[C],
                                         const float2 (&gY)[C], float2 (&gw)[2 * C], float2& S0, float2& Sy,
                                         float2& Syy) {
    const float2 al = make_float2(c0 ? a2.x : 0.f, c1 ? a2.y : 0.f);
    const float2 om = __fadd2_rn(f2(1.f), make_float2(-al.x, -al.y));
    const float2 iom = make_float2(rcp_approx(om.x), rcp_approx(om.y));
    const float2 Tk = __fmul2_rn(T2, iom);
    const float2 aT = __fmul2_rn(al, Tk);
    float2 Ak = f2(0.f);
#pragma unroll
    for (int c = 0; c < C; c++) {
        const float2 w = RecW<C>::get(rec, c);
        Ak = __ffma2_rn(gX[c], f2(w.x), __ffma2_rn(gY[c], f2(w.y), Ak));
        gw[2 * c] = FIRST ? __fmul2_rn(gX[c], aT) : __ffma2_rn(gX[c], aT, gw[2 * c]);
        gw[2 * c + 1] = FIRST ? __fmul2_rn(gY[c], aT) : __ffma2_rn(gY[c], aT, gw[2 * c + 1]);
    }
    const float2 dLda = __ffma2_rn(Tk, Ak, __fmul2_rn(make_float2(-iom.x, -iom.y), B2));
    B2 = __ffma2_rn(aT, Ak, B2);
    T2 = Tk;
    // -dL/dpower = o dL/do; a clamped alpha (o G > alpha_max) is flat in o G
    float2 p;
    if (CL) {
        const float2 dLa = make_float2(c0 && og2.x <= amax ? dLda.x : 0.f, c1 && og2.y <= amax ? dLda.y : 0.f);
        p = __fmul2_rn(dLa, og2);
    } else {
        p = __fmul2_rn(dLda, al);
    }
    const float2 pdy = __fmul2_rn(p, dy2);
    if (FIRST) {
        S0 = p;
        Sy = pdy;
        Syy = __fmul2_rn(pdy, dy2);
    } else {
        S0 = __fadd2_rn(S0, p);
        Sy = __fadd2_rn(Sy, pdy);
        Syy = __ffma2_rn(pdy, dy2, Syy);
    }
}

// The entry's 6 + 2C sums of one thread, from its accumulators: the pixel
// moments of p = -dL/dpower, d = pixel - mu (dx is the same for the thread's
// pixels; s0, sy, syy its sums of p, p dy, p dy^2), then dL/dw_c:
//   m = (sum dx p, sum dy p, sum dx^2 p, sum dx dy p, sum dy^2 p, sum p).
// With power = 1/2 (A dx^2 + C dy^2) + B dx dy the 2D gradients are linear in
// them: dL/dmu = (A m0 + B m1, B m0 + C m1), dL/dA = -m2 / 2, dL/dB = -m3,
// dL/dC = -m4 / 2, o dL/do = m5 (formed once per Gaussian in the projection
// adjoint, not per entry and thread).
template <int C>
__device__ __forceinline__ void entry_moments(float dx, float2 S0, float2 Sy, float2 Syy, const float2 (&gw)[2 * C],
                                              float (&out)[6 + 2 * C]) {
    const float s0 = S0.x + S0.y, sy = Sy.x + Sy.y;
    out[0] = dx * s0;
    out[1] = sy;
    out[2] = dx * out[0];
    out[3] = dx * sy;
    out[4] = Syy.x + Syy.y;
    out[5] = s0;
#pragma unroll
    for (int e = 0; e < 2 * C; e++) out[6 + e] = gw[e].x + gw[e].y;
}

// Loads kept entries [lo, lo + cnt) of a strip (visiting ranks from the forward
// pass) into the warp's slots: record, base-2 exponent coefficients and the
// Gaussian id (the 2D gradients are stored in Gaussian order, so that the
// projection adjoint reads them contiguously).
template <int NR, int FT>
__device__ __forceinline__ void stage_kept(const RasterArgs& a, size_t vN, const uint32_t* kept, uint32_t lo, int cnt,
                                           float4 (*wrec)[NR + 1], uint32_t* wid) {
    const int lane = threadIdx.x & 31;
    if (lane < cnt) {
        uint32_t s = kept[lo + lane];
        if (!HCGS_DCHECK(a.status, s < (uint32_t)a.N)) s = 0u;  // checked build: a stray rank reads entry 0
        const float4* r = a.rec + (vN + s) * NR;
        const float4 q0 = r[0], q1 = r[1];
        wrec[lane][0] = q0;
        wrec[lane][1] = q1;
#pragma unroll
        for (int k = 2; k < NR; k++) wrec[lane][k] = r[k];
        wrec[lane][NR] = entry_coeffs<FT>(q0, q1);
        wid[lane] = a.sortid[vN + s];
    }
    __syncwarp();
}

template <int C, int FT>
__global__ void __launch_bounds__(RT, 24) k_raster_bwd(RasterArgs a, const float* __restrict__ Tsave,
                                                    const uint32_t* __restrict__ lastsave,
                                                    const float2* __restrict__ gU, float* __restrict__ g2d) {
    constexpr int NR = C <= 1 ? 2 : (C <= 3 ? 3 : 4);
    constexpr int G = 6 + 2 * C;
    constexpr int RS = 36;  // row stride of the reduction buffer (floats)
    __shared__ float4 srec[32][NR + 1];
    __shared__ uint32_t sid[32];
    __shared__ __align__(16) float sred[G][RS];
    const int lane = threadIdx.x;
    const int strip = blockIdx.x, l = blockIdx.y, v = blockIdx.z;
    const int tx = strip % a.tilesX, ty = (strip / a.tilesX) >> 1;
    const int px = tx * TILE + (lane & 15);
    const int sy = ty * TILE + 8 * ((strip / a.tilesX) & 1);
    const int py = sy + (lane >> 4);
    const uint32_t gb = ((uint32_t)(v * a.L + l) * a.ctY + ty / COARSE) * a.ctX + tx / COARSE;
    const uint32_t beg = a.off[gb], n = a.off[gb + 1] - beg;
    const uint32_t* kept = a.slist + strip_list_base(beg, n, tx, strip / a.tilesX);
    const size_t vN = (size_t)v * a.N;
    const size_t plane = (size_t)v * a.L + l;
    const size_t HW = (size_t)a.H * a.W;
    const float fpx = (float)px;
    const float2 pyA = make_float2((float)py, (float)(py + 2)), pyB = make_float2((float)(py + 4), (float)(py + 6));
    float Tq[4] = {1.f, 1.f, 1.f, 1.f};
    uint32_t last[4] = {0, 0, 0, 0};
    float2 gq[4][C];
#pragma unroll
    for (int q = 0; q < 4; q++) {
#pragma unroll
        for (int c = 0; c < C; c++) gq[q][c] = make_float2(0.f, 0.f);
        if (px < a.W && py + 2 * q < a.H) {
            const size_t pix = (size_t)(py + 2 * q) * a.W + px;
            Tq[q] = Tsave[plane * HW + pix];
            last[q] = lastsave[plane * HW + pix];
#pragma unroll
            for (int c = 0; c < C; c++) gq[q][c] = gU[(plane * C + c) * HW + pix];
        }
    }
    float2 TA = make_float2(Tq[0], Tq[1]), TB = make_float2(Tq[2], Tq[3]);
    float2 gAX[C], gAY[C], gBX[C], gBY[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        gAX[c] = make_float2(gq[0][c].x, gq[1][c].x);
        gAY[c] = make_float2(gq[0][c].y, gq[1][c].y);
        gBX[c] = make_float2(gq[2][c].x, gq[3][c].x);
        gBY[c] = make_float2(gq[2][c].y, gq[3][c].y);
    }
    float2 BA = f2(0.f), BB = f2(0.f);  // sum_c Re(conj(g_c) S_c) per pixel
    uint32_t maxlast = max(max(last[0], last[1]), max(last[2], last[3]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxlast = max(maxlast, __shfl_xor_sync(0xffffffffu, maxlast, o));
    if (!HCGS_DCHECK(a.status, maxlast <= n)) maxlast = 0u;  // checked build: a stray length skips the strip
    for (uint32_t hi = maxlast; hi > 0;) {
        const uint32_t lo = hi > 32u ? hi - 32u : 0u;
        const int nh = (int)(hi - lo);
        stage_kept<NR, FT>(a, vN, kept, lo, nh, srec, sid);
        for (int k = nh - 1; k >= 0; k--) {  // back-to-front over the visiting order
            const float4* rec = srec[k];
            const uint32_t pos = lo + (uint32_t)k;
            const float4 r0 = rec[0], r1 = rec[1], kk = rec[NR];
            auto step = [&](auto cl) {
                constexpr bool CL = decltype(cl)::value;
                const EntryX x = entry_x(fpx, r0, kk);
                float2 dyA, ogA, aA, dyB, ogB, aB;
                eval_entry<FT, CL>(x, pyA, pyB, r0, r1, kk, a.amax, dyA, ogA, aA, dyB, ogB, aB);
                const bool c0 = pos < last[0] && aA.x >= a.amin, c1 = pos < last[1] && aA.y >= a.amin;
                const bool c2 = pos < last[2] && aB.x >= a.amin, c3 = pos < last[3] && aB.y >= a.amin;
                // no pixel of the strip took this step: zero gradient, T and B unchanged
                if (!__any_sync(0xffffffffu, c0 || c1 || c2 || c3)) return;
                // branch-free: pixels that did not take the step carry alpha 0
                // through the pair (T and B unchanged, zero gradient)
                float2 gw[2 * C], S0, Sy, Syy;
                bwd_pair<C, true, CL>(rec, dyA, ogA, aA, c0, c1, a.amax, TA, BA, gAX, gAY, gw, S0, Sy, Syy);
                bwd_pair<C, false, CL>(rec, dyB, ogB, aB, c2, c3, a.amax, TB, BB, gBX, gBY, gw, S0, Sy, Syy);
                float gv[G];
                entry_moments<C>(x.dx, S0, Sy, Syy, gw, gv);
                // warp sum of the G values: each lane writes its column of the
                // G x 32 buffer, lane (e, h) adds the 16 values of row e in
                // half h, one shuffle joins the halves
                float* red = &sred[0][0];
#pragma unroll
                for (int e = 0; e < G; e++) red[e * RS + lane] = gv[e];
                __syncwarp();
                const int e = lane >> 1, h = lane & 1;
                // lanes past the last row read it again (branch-free) and discard
                const float4* row = reinterpret_cast<const float4*>(red + (e < G ? e : G - 1) * RS + 16 * h);
                const float4 u0 = row[0], u1 = row[1], u2 = row[2], u3 = row[3];
                const float2 s0 = __fadd2_rn(make_float2(u0.x, u0.y), make_float2(u0.z, u0.w));
                const float2 s1 = __fadd2_rn(make_float2(u1.x, u1.y), make_float2(u1.z, u1.w));
                const float2 s2 = __fadd2_rn(make_float2(u2.x, u2.y), make_float2(u2.z, u2.w));
                const float2 s3 = __fadd2_rn(make_float2(u3.x, u3.y), make_float2(u3.z, u3.w));
                const float2 s4 = __fadd2_rn(__fadd2_rn(s0, s1), __fadd2_rn(s2, s3));
                float sum = s4.x + s4.y;
                sum += __shfl_xor_sync(0xffffffffu, sum, 1);
                // slot 5 holds o dL/do = sum p (the projection adjoint needs no more)
                if (!h && e < G) atomicAdd(g2d + (vN + sid[k]) * G + e, sum);
                __syncwarp();
            };
            if (may_clamp(r1.y, a.amax)) step(std::true_type{});
            else step(std::false_type{});
        }
        __syncwarp();
        hi = lo;
    }
}

// ---------------------------------------------------------------------------
// Dense plane-weight gradient (rho_grad = 1).  For plane l and a Gaussian n
// assigned elsewhere, compositing with continuous weights (alpha_eff = alpha
// rho_l) has, at rho_{n,l} = 0, dU_l/drho_{n,l} = o G (w_n T_l - S_l) at every
// pixel whose plane-l walk reaches n (alpha = min(alpha_max, o G) >= alpha_min,
// not yet stopped), T_l the plane's transmittance at n's place in the
// visiting order and S_l = U_l - (the plane's field in front of n).  One warp
// per (16 x 8 strip, plane l, view): pass A forms U_l at the warp's pixels
// from the plane's own list (the forward's decisions); pass B walks the tile's
// all-plane list in visiting order, advancing T and the prefix on plane-l
// entries and reducing the others' terms over the strip into drho[n][l].
// ---------------------------------------------------------------------------
template <int C, int FT>
__global__ void __launch_bounds__(RT) k_raster_rho_dense(RasterArgs a, const uint32_t* __restrict__ aoff,
                                                         const uint32_t* __restrict__ alist,
                                                         const int* __restrict__ planes,
                                                         const uint32_t* __restrict__ sortid,
                                                         const float2* __restrict__ gU, float* __restrict__ drho) {
    constexpr int NR = C <= 1 ? 2 : (C <= 3 ? 3 : 4);
    __shared__ float4 srec[32][NR + 1];
    __shared__ uint32_t spos[32], sid[32], skept[32];
    const int lane = threadIdx.x;
    const int strip = blockIdx.x, l = blockIdx.y, v = blockIdx.z;
    const int tx = strip % a.tilesX, ty = (strip / a.tilesX) >> 1;
    const int px = tx * TILE + (lane & 15);
    const int sy = ty * TILE + 8 * ((strip / a.tilesX) & 1);
    const int py = sy + (lane >> 4);
    const bool colin = px < a.W;
    const float sx0 = (float)(tx * TILE), sy0 = (float)sy;
    const size_t vN = (size_t)v * a.N;
    const float fpx = (float)px;
    const float teps = a.teps;
    const float2 pyA = make_float2((float)py, (float)(py + 2)), pyB = make_float2((float)(py + 4), (float)(py + 6));
    const float2 T0A = make_float2(colin && py < a.H ? 1.f : 0.f, colin && py + 2 < a.H ? 1.f : 0.f);
    const float2 T0B = make_float2(colin && py + 4 < a.H ? 1.f : 0.f, colin && py + 6 < a.H ? 1.f : 0.f);
    // pass A: U_l at the warp's pixels
    float2 uAX[C], uAY[C], uBX[C], uBY[C];
#pragma unroll
    for (int c = 0; c < C; c++) uAX[c] = uAY[c] = uBX[c] = uBY[c] = f2(0.f);
    {
        const uint32_t gb = ((uint32_t)(v * a.L + l) * a.ctY + ty / COARSE) * a.ctX + tx / COARSE;
        const uint32_t beg = a.off[gb], n = a.off[gb + 1] - beg;
        float2 TA = T0A, TB = T0B;
        for (uint32_t p0 = 0; p0 < n; p0 += 32) {
            const bool live = TA.x >= teps || TA.y >= teps || TB.x >= teps || TB.y >= teps;
            if (!__any_sync(0xffffffffu, live)) break;
            const int nh = stage_warp<NR, FT>(a, vN, beg, p0, n, tx, ty, sx0, sy0, srec, spos, sid, skept);
            for (int k = 0; k < nh; k++) {
                const float4* rec = srec[k];
                const float4 r0 = rec[0], r1 = rec[1], kk = rec[NR];
                const EntryX x = entry_x(fpx, r0, kk);
                float2 dyA, ogA, aA, dyB, ogB, aB;
                if (may_clamp(r1.y, a.amax)) eval_entry<FT, true>(x, pyA, pyB, r0, r1, kk, a.amax, dyA, ogA, aA, dyB, ogB, aB);
                else eval_entry<FT, false>(x, pyA, pyB, r0, r1, kk, a.amax, dyA, ogA, aA, dyB, ogB, aB);
                const bool c0 = TA.x >= teps && aA.x >= a.amin, c1 = TA.y >= teps && aA.y >= a.amin;
                const bool c2 = TB.x >= teps && aB.x >= a.amin, c3 = TB.y >= teps && aB.y >= a.amin;
                fwd_pair<C>(rec, aA, c0, c1, TA, uAX, uAY);
                fwd_pair<C>(rec, aB, c2, c3, TB, uBX, uBY);
            }
            __syncwarp();
        }
    }
    // upstream gradient at the warp's pixels
    const size_t HW = (size_t)a.H * a.W;
    const size_t pbase = ((size_t)v * a.L + l) * C;
    float2 gq[4][C];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const bool in = colin && py + 2 * q < a.H;
        const size_t pix = (size_t)(py + 2 * q) * a.W + px;
#pragma unroll
        for (int c = 0; c < C; c++) gq[q][c] = in ? gU[(pbase + c) * HW + pix] : make_float2(0.f, 0.f);
    }
    // pass B: every plane's Gaussians of the tile, in visiting order
    const uint32_t gba = ((uint32_t)v * a.ctY + ty / COARSE) * a.ctX + tx / COARSE;
    const uint32_t beg = aoff[gba], n = aoff[gba + 1] - beg;
    RasterArgs aa = a;
    aa.list = alist;
    float2 TA = T0A, TB = T0B;
    float2 pAX[C], pAY[C], pBX[C], pBY[C];  // prefix of the plane's field
#pragma unroll
    for (int c = 0; c < C; c++) pAX[c] = pAY[c] = pBX[c] = pBY[c] = f2(0.f);
    for (uint32_t p0 = 0; p0 < n; p0 += 32) {
        const bool live = TA.x >= teps || TA.y >= teps || TB.x >= teps || TB.y >= teps;
        if (!__any_sync(0xffffffffu, live)) break;
        const int nh = stage_warp<NR, FT>(aa, vN, beg, p0, n, tx, ty, sx0, sy0, srec, spos, sid, skept);
        for (int k = 0; k < nh; k++) {
            const float4* rec = srec[k];
            const float4 r0 = rec[0], r1 = rec[1], kk = rec[NR];
            const uint32_t srank = sid[k];
            const bool own = planes[vN + srank] == l;  // warp-uniform
            const EntryX x = entry_x(fpx, r0, kk);
            float2 dyA, ogA, aA, dyB, ogB, aB;
            if (may_clamp(r1.y, a.amax)) eval_entry<FT, true>(x, pyA, pyB, r0, r1, kk, a.amax, dyA, ogA, aA, dyB, ogB, aB);
            else eval_entry<FT, false>(x, pyA, pyB, r0, r1, kk, a.amax, dyA, ogA, aA, dyB, ogB, aB);
            const bool c0 = TA.x >= teps && aA.x >= a.amin, c1 = TA.y >= teps && aA.y >= a.amin;
            const bool c2 = TB.x >= teps && aB.x >= a.amin, c3 = TB.y >= teps && aB.y >= a.amin;
            if (own) {
                fwd_pair<C>(rec, aA, c0, c1, TA, pAX, pAY);
                fwd_pair<C>(rec, aB, c2, c3, TB, pBX, pBY);
            } else {
                // o G sum_c Re(conj(g_c) (w_c T - (U_c - prefix_c))) over the reached pixels
                float acc = 0.f;
                const float Tq[4] = {TA.x, TA.y, TB.x, TB.y};
                const float og[4] = {ogA.x, ogA.y, ogB.x, ogB.y};
                const bool cq[4] = {c0, c1, c2, c3};
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    float d = 0.f;
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        const float2 w = RecW<C>::get(rec, c);
                        const float ux = q == 0 ? uAX[c].x : q == 1 ? uAX[c].y : q == 2 ? uBX[c].x : uBX[c].y;
                        const float uy = q == 0 ? uAY[c].x : q == 1 ? uAY[c].y : q == 2 ? uBY[c].x : uBY[c].y;
                        const float qx = q == 0 ? pAX[c].x : q == 1 ? pAX[c].y : q == 2 ? pBX[c].x : pBX[c].y;
                        const float qy = q == 0 ? pAY[c].x : q == 1 ? pAY[c].y : q == 2 ? pBY[c].x : pBY[c].y;
                        d = fmaf(gq[q][c].x, fmaf(w.x, Tq[q], -(ux - qx)), d);
                        d = fmaf(gq[q][c].y, fmaf(w.y, Tq[q], -(uy - qy)), d);
                    }
                    acc = fmaf(cq[q] ? og[q] : 0.f, d, acc);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0 && acc != 0.f) atomicAdd(&drho[(size_t)sortid[vN + srank] * a.L + l], acc);
            }
        }
        __syncwarp();
    }
}

hcgs_status raster_forward(hcgs_ctx* ctx, hcgs_saved* s, float2* U, float* T_out, int32_t* nc_out,
                           cudaStream_t st) {
    const size_t pl = (size_t)s->V * s->L * s->H * s->W;
    HCGS_CUDA(ctx, grow(ctx, s->Tfin, pl * sizeof(float), &s->bytes));
    HCGS_CUDA(ctx, grow(ctx, s->last, pl * sizeof(uint32_t), &s->bytes));
    HCGS_CUDA(ctx, grow(ctx, s->slist, (size_t)COARSE * COARSE * 2 * s->M * sizeof(uint32_t) + 16, &s->bytes));
    RasterArgs a = make_raster_args(s);
    a.status = ctx->d_status;
    dim3 grid(s->tilesX * s->tilesY * 2, s->L, s->V);  // 16 x 8 pixel strips
    float* Ts = (float*)s->Tfin.p;
    uint32_t* ls = (uint32_t*)s->last.p;
    const int ft = s->opts.footprint;
#define HCGS_FWD_T(CC, FTV)                                                                                                 \
    if (nc_out)                                                                                                             \
        HCGS_KERNEL(ctx, "k_raster_fwd", st, (k_raster_fwd<CC, FTV, true><<<grid, RT, 0, st>>>(a, U, Ts, ls, T_out, nc_out)));  \
    else                                                                                                                    \
        HCGS_KERNEL(ctx, "k_raster_fwd", st, (k_raster_fwd<CC, FTV, false><<<grid, RT, 0, st>>>(a, U, Ts, ls, T_out, nc_out)))
#define HCGS_FWD(CC)                          \
    if (ft == 1) {                            \
        HCGS_FWD_T(CC, 1);                    \
    } else if (ft == 2) {                     \
        HCGS_FWD_T(CC, 2);                    \
    } else {                                  \
        HCGS_FWD_T(CC, 0);                    \
    }
    switch (s->C) {
        case 1: HCGS_FWD(1); break;
        case 2: HCGS_FWD(2); break;
        case 3: HCGS_FWD(3); break;
        default: HCGS_FWD(4); break;
    }
#undef HCGS_FWD
#undef HCGS_FWD_T
    HCGS_LAUNCH(ctx, "k_raster_fwd");
    return HCGS_OK;
}

hcgs_status raster_backward(hcgs_ctx* ctx, hcgs_saved* s, const float2* gU, cudaStream_t st) {
    const size_t ng = (size_t)s->V * s->N * g2d_count(s->C);
    HCGS_CUDA(ctx, grow(ctx, s->g2d, ng * sizeof(float), &s->bytes));
    HCGS_CUDA(ctx, cudaMemsetAsync(s->g2d.p, 0, ng * sizeof(float), st));
    RasterArgs a = make_raster_args(s);
    a.status = ctx->d_status;
    dim3 grid(s->tilesX * s->tilesY * 2, s->L, s->V);  // 16 x 8 pixel strips
    const float* Ts = (const float*)s->Tfin.p;
    const uint32_t* ls = (const uint32_t*)s->last.p;
    float* g2 = (float*)s->g2d.p;
    const int ft = s->opts.footprint;
#define HCGS_BWD(CC)                                                                                              \
    if (ft == 1)                                                                                                  \
        HCGS_KERNEL(ctx, "k_raster_bwd", st, (k_raster_bwd<CC, 1><<<grid, RT, 0, st>>>(a, Ts, ls, gU, g2)));      \
    else if (ft == 2)                                                                                             \
        HCGS_KERNEL(ctx, "k_raster_bwd", st, (k_raster_bwd<CC, 2><<<grid, RT, 0, st>>>(a, Ts, ls, gU, g2)));      \
    else                                                                                                          \
        HCGS_KERNEL(ctx, "k_raster_bwd", st, (k_raster_bwd<CC, 0><<<grid, RT, 0, st>>>(a, Ts, ls, gU, g2)))
    switch (s->C) {
        case 1: HCGS_BWD(1); break;
        case 2: HCGS_BWD(2); break;
        case 3: HCGS_BWD(3); break;
        default: HCGS_BWD(4); break;
    }
#undef HCGS_BWD
    HCGS_LAUNCH(ctx, "k_raster_bwd");
    if (s->opts.rho_grad) {
        const size_t nd = (size_t)s->N * s->L;
        HCGS_CUDA(ctx, grow(ctx, s->drho, (nd > 0 ? nd : 1) * sizeof(float), &s->bytes));
        HCGS_CUDA(ctx, cudaMemsetAsync(s->drho.p, 0, (nd > 0 ? nd : 1) * sizeof(float), st));
        const uint32_t* aoff = (const uint32_t*)s->abcount.p;
        const int* pl = (const int*)s->planes.p;
        const uint32_t* sid = (const uint32_t*)s->sortid.p;
        float* dr = (float*)s->drho.p;
#define HCGS_DENSE(CC)                                                                                            \
    if (ft == 1)                                                                                                  \
        HCGS_KERNEL(ctx, "k_raster_rho_dense", st,                                                                \
                    (k_raster_rho_dense<CC, 1><<<grid, RT, 0, st>>>(a, aoff, s->alist, pl, sid, gU, dr)));        \
    else if (ft == 2)                                                                                             \
        HCGS_KERNEL(ctx, "k_raster_rho_dense", st,                                                                \
                    (k_raster_rho_dense<CC, 2><<<grid, RT, 0, st>>>(a, aoff, s->alist, pl, sid, gU, dr)));        \
    else                                                                                                          \
        HCGS_KERNEL(ctx, "k_raster_rho_dense", st,                                                                \
                    (k_raster_rho_dense<CC, 0><<<grid, RT, 0, st>>>(a, aoff, s->alist, pl, sid, gU, dr)))
        switch (s->C) {
            case 1: HCGS_DENSE(1); break;
            case 2: HCGS_DENSE(2); break;
            case 3: HCGS_DENSE(3); break;
            default: HCGS_DENSE(4); break;
        }
#undef HCGS_DENSE
        HCGS_LAUNCH(ctx, "k_raster_rho_dense");
    }
    return HCGS_OK;
}

}  // namespace hcgs
