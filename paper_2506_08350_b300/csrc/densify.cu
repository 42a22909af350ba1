// Densification of Algorithm 1 (Supp. D.2): statistics of the screen-space mean
// gradient, the per-Gaussian decision (prune / keep / clone / split), and the
// compaction that writes the new parameter arrays with phase-aware copies;
// plus the counter-based generator (Philox4x32-10, Salmon et al. 2011) that
// draws the copies' noise.
//
// Rules (those of 3DGS, which Sec. 5 adopts with a 300-step period):
//   statistic  s_n = sum over views where n is visible of
//              |(dL/dmu_x W/2, dL/dmu_y H/2)|, d_n = number of such views;
//   prune      sigmoid(logit) < prune_opacity, or max scale > prune_scale (> 0);
//   densify    s_n / d_n >= grad_threshold:
//              split when max scale > split_scale: two children with means
//              mu + R diag(s) z_k, log-scales - log(split_shrink), phases
//              phi + phase_noise z'_k, everything else copied, parent removed;
//              clone otherwise: the parent, then a copy with phases
//              phi + phase_noise z'_0.
// Outputs follow the input order (offsets from an exclusive scan of 0/1/2).
#include <cmath>

#include "common.cuh"
#include "project.cuh"

namespace hcgs {

// ---------------------------------------------------------------------------
// Philox4x32-10: 10 rounds of two 32 x 32 -> 64-bit products, the word
// permutation and the key, bumped by the Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// block b of the stream (seed, stream): counter (b, stream, 0, 0), key = seed
__global__ void k_philox(uint64_t seed, uint32_t stream, int64_t n, int normal, void* __restrict__ out) {
    const int64_t nb = (n + 3) / 4;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)b, stream, 0u, 0u), key);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
        if (normal == 0) {
            uint32_t* o = (uint32_t*)out;
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (4 * b + i < n) o[4 * b + i] = ws[i];
        } else if (normal == 2) {
            // uniforms (w + 1/2) 2^-32 in (0, 1), rounded to float
            float* o = (float*)out;
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (4 * b + i < n) o[4 * b + i] = (float)(((double)ws[i] + 0.5) * 0x1p-32);
        } else {
            // Box-Muller on the word pairs (in double: the draws are few)
            float* o = (float*)out;
#pragma unroll
            for (int p = 0; p < 2; p++) {
                const double u = ((double)ws[2 * p] + 0.5) * 0x1p-32;
                const double v = ((double)ws[2 * p + 1] + 0.5) * 0x1p-32;
                const double r = sqrt(-2.0 * log(u));
                double sn, cs;
                sincospi(2.0 * v, &sn, &cs);
                if (4 * b + 2 * p < n) o[4 * b + 2 * p] = (float)(r * cs);
                if (4 * b + 2 * p + 1 < n) o[4 * b + 2 * p + 1] = (float)(r * sn);
            }
        }
    }
}

hcgs_status philox(hcgs_ctx* ctx, uint64_t seed, uint32_t stream_id, int64_t n, int normal, void* out,
                   cudaStream_t st) {
    const int64_t nb = (n + 3) / 4;
    const int blocks = (int)std::min<int64_t>(148 * 8, (nb + 255) / 256);
    HCGS_KERNEL(ctx, "k_philox", st, k_philox<<<blocks, 256, 0, st>>>(seed, stream_id, n, normal, out));
    return HCGS_OK;
}

// ---------------------------------------------------------------------------
// statistics: per Gaussian, over the views of the last backward pass
// ---------------------------------------------------------------------------
__global__ void k_densify_accum(const uint32_t* __restrict__ rank, const float* __restrict__ g2d,
                                const float4* __restrict__ rec, int NR, int V, int N, int G, float hw, float hh,
                                float* __restrict__ accum, float* __restrict__ denom) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f, d = 0.f;
    for (int v = 0; v < V; v++) {
        const uint32_t r = rank[(size_t)v * N + n];
        if (r == 0xFFFFFFFFu) continue;
        const size_t e = (size_t)v * N + r;
        const float* g = g2d + ((size_t)v * N + n) * G;
        // dL/dmu from the pixel moments sum dx p, sum dy p and the conic A, B, C
        // of the record: (A m0 + B m1, B m0 + C m1)
        const float4 q0 = rec[e * NR], q1 = rec[e * NR + 1];
        const float gx = fmaf(q0.z, g[0], q0.w * g[1]), gy = fmaf(q0.w, g[0], q1.x * g[1]);
        s += sqrtf(gx * hw * (gx * hw) + gy * hh * (gy * hh));
        d += 1.f;
    }
    if (d > 0.f) {
        accum[n] += s;
        denom[n] += d;
    }
}

hcgs_status densify_accumulate(hcgs_ctx* ctx, hcgs_saved* s, float* accum, float* denom, cudaStream_t st) {
    if (s->N == 0) return HCGS_OK;
    HCGS_KERNEL(ctx, "k_densify_accum", st,
                k_densify_accum<<<(s->N + 255) / 256, 256, 0, st>>>(
                    (const uint32_t*)s->rank.p, (const float*)s->g2d.p, (const float4*)s->rec.p,
                    rec_count(s->C), s->V, s->N, g2d_count(s->C),
                    0.5f * (float)s->W, 0.5f * (float)s->H, accum, denom));
    return HCGS_OK;
}

// ---------------------------------------------------------------------------
// decision and output counts
// ---------------------------------------------------------------------------
enum { D_KEEP = 0, D_PRUNE = 1, D_CLONE = 2, D_SPLIT = 3 };

__global__ void k_densify_decide(const float* __restrict__ log_scales, const float* __restrict__ opacity_logits,
                                 const float* __restrict__ accum, const float* __restrict__ denom, int N,
                                 hcgs_densify_opts o, int32_t* __restrict__ action, uint32_t* __restrict__ count) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const float op = 1.f / (1.f + expf(-opacity_logits[n]));
    const float smax = expf(fmaxf(log_scales[3 * n], fmaxf(log_scales[3 * n + 1], log_scales[3 * n + 2])));
    const float d = denom[n];
    const float avg = d > 0.f ? accum[n] / d : 0.f;
    int a = D_KEEP;
    if (avg >= o.grad_threshold) a = smax > o.split_scale ? D_SPLIT : D_CLONE;
    if (op < o.prune_opacity || (o.prune_scale > 0.f && smax > o.prune_scale)) a = D_PRUNE;
    action[n] = a;
    count[n] = a == D_PRUNE ? 0u : (a == D_KEEP ? 1u : 2u);
}

__global__ void k_offsets_tail(const uint32_t* __restrict__ count, uint32_t* __restrict__ offsets, int N) {
    offsets[N] = offsets[N - 1] + count[N - 1];
}

// offsets[N] = the total after the exclusive scan of count (N >= 1)
hcgs_status densify_offsets_tail(hcgs_ctx* ctx, const uint32_t* count, uint32_t* offsets, int N, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_offsets_tail", st, k_offsets_tail<<<1, 1, 0, st>>>(count, offsets, N));
    return HCGS_OK;
}

hcgs_status densify_decide(hcgs_ctx* ctx, const hcgs_gaussians* g, const float* accum, const float* denom,
                           const hcgs_densify_opts& o, int32_t* action, uint32_t* count, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_densify_decide", st,
                k_densify_decide<<<(g->N + 255) / 256, 256, 0, st>>>(g->log_scales, g->opacity_logits, accum, denom,
                                                                     g->N, o, action, count));
    return HCGS_OK;
}

// ---------------------------------------------------------------------------
// compaction with copies
// ---------------------------------------------------------------------------
struct DensifyExtras {
    const float* in[HCGS_DENSIFY_MAX_EXTRA];
    float* out[HCGS_DENSIFY_MAX_EXTRA];
    int width[HCGS_DENSIFY_MAX_EXTRA];
    int k;
};

__global__ void k_densify_apply(hcgs_gaussians gi, int C, int L, const int32_t* __restrict__ action,
                                const uint32_t* __restrict__ offset, const float* __restrict__ noise,
                                hcgs_densify_opts o, hcgs_gaussian_grads go, DensifyExtras ex) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= gi.N) return;
    const int a = action[n];
    if (a == D_PRUNE) return;
    const size_t j = offset[n];
    const int NZ = 3 + C;
    // a plain copy of Gaussian n to output slot m
    auto copy = [&](size_t m) {
        for (int i = 0; i < 3; i++) go.means[3 * m + i] = gi.means[3 * (size_t)n + i];
        for (int i = 0; i < 3; i++) go.log_scales[3 * m + i] = gi.log_scales[3 * (size_t)n + i];
        for (int i = 0; i < 4; i++) go.quats[4 * m + i] = gi.quats[4 * (size_t)n + i];
        go.opacity_logits[m] = gi.opacity_logits[n];
        for (int c = 0; c < C; c++) go.amplitude[C * m + c] = gi.amplitude[C * (size_t)n + c];
        for (int c = 0; c < C; c++) go.phase[C * m + c] = gi.phase[C * (size_t)n + c];
        for (int l = 0; l < L; l++) go.plane_logits[L * m + l] = gi.plane_logits[L * (size_t)n + l];
    };
    auto extras = [&](size_t m, bool keep) {
        for (int e = 0; e < ex.k; e++)
            for (int i = 0; i < ex.width[e]; i++)
                ex.out[e][(size_t)ex.width[e] * m + i] = keep ? ex.in[e][(size_t)ex.width[e] * n + i] : 0.f;
    };
    const float* z = noise + (size_t)n * 2 * NZ;
    if (a == D_KEEP || a == D_CLONE) {
        copy(j);
        extras(j, true);
    }
    if (a == D_CLONE) {
        copy(j + 1);
        for (int c = 0; c < C; c++) go.phase[C * (j + 1) + c] += o.phase_noise * z[3 + c];
        extras(j + 1, false);
    }
    if (a == D_SPLIT) {
        // rotation of the normalised quaternion (w, x, y, z) and the scales
        const float* q = gi.quats + 4 * (size_t)n;
        const float qn = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        const float w = q[0] * qn, x = q[1] * qn, y = q[2] * qn, zq = q[3] * qn;
        const float R[9] = {1.f - 2.f * (y * y + zq * zq), 2.f * (x * y - w * zq), 2.f * (x * zq + w * y),
                            2.f * (x * y + w * zq), 1.f - 2.f * (x * x + zq * zq), 2.f * (y * zq - w * x),
                            2.f * (x * zq - w * y), 2.f * (y * zq + w * x), 1.f - 2.f * (x * x + y * y)};
        float s[3];
        for (int i = 0; i < 3; i++) s[i] = expf(gi.log_scales[3 * (size_t)n + i]);
        const float shrink = logf(o.split_shrink);
        for (int k = 0; k < 2; k++) {
            const size_t m = j + k;
            const float* zk = z + k * NZ;
            copy(m);
            for (int i = 0; i < 3; i++) {
                const float d = R[3 * i] * (s[0] * zk[0]) + R[3 * i + 1] * (s[1] * zk[1]) + R[3 * i + 2] * (s[2] * zk[2]);
                go.means[3 * m + i] += d;
                go.log_scales[3 * m + i] -= shrink;
            }
            for (int c = 0; c < C; c++) go.phase[C * m + c] += o.phase_noise * zk[3 + c];
            extras(m, false);
        }
    }
}

hcgs_status densify_apply(hcgs_ctx* ctx, const hcgs_gaussians* gi, int C, int L, const int32_t* action,
                          const uint32_t* offset, const float* noise, const hcgs_densify_opts& o,
                          const hcgs_gaussian_grads& go, int n_extra, const float* const* extra_in,
                          float* const* extra_out, const int* extra_width, cudaStream_t st) {
    DensifyExtras ex{};
    ex.k = n_extra;
    for (int e = 0; e < n_extra; e++) {
        ex.in[e] = extra_in[e];
        ex.out[e] = extra_out[e];
        ex.width[e] = extra_width[e];
    }
    HCGS_KERNEL(ctx, "k_densify_apply", st,
                k_densify_apply<<<(gi->N + 127) / 128, 128, 0, st>>>(*gi, C, L, action, offset, noise, o, go, ex));
    return HCGS_OK;
}

}  // namespace hcgs
