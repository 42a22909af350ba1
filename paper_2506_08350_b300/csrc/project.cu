// Steps 1-2 of the render path on sm_103a: projection of the Gaussians
// (Sec. 3 Eq. gaussian_projection / gaussian_projection_2d; Eq.
// hard_assignment), depth sort, and binning into coarse 64x64-pixel buckets
// per plane; plus the adjoint of the projection (Supp. D.4, Eq. ste).
//
// Binning design.  Instead of materialising one (tile, depth) key per
// Gaussian and covered 16x16 tile and sorting those (Algorithm 2 preprocessing),
// the Gaussians are sorted once by depth (N keys per view), and each visible
// Gaussian emits one instance per covered 64x64 bucket of its plane, in
// visiting order.  A stable radix sort by bucket id then yields per-bucket
// lists already in visiting order.  The rasterizer streams a bucket's list and
// keeps the entries whose 16x16-tile rectangle covers its tile.  This moves
// ~16x fewer instances than per-tile binning, needs no per-tile sort, and the
// result does not depend on tiling because every candidate is still tested
// per pixel with the support rule o G >= alpha_min.
#include <cmath>

#include "common.cuh"
#include "project.cuh"

namespace hcgs {

// ---------------------------------------------------------------------------
// projection
// ---------------------------------------------------------------------------
__global__ void k_prep_w(const float* __restrict__ amp, const float* __restrict__ ph, float2* __restrict__ w,
                         int N, int C, int* __restrict__ status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * C) return;
    (void)HCGS_DCHECK(status, isfinite(amp[i]) && isfinite(ph[i]));  // non-finite appearance (checked build)
    float s, c;
    sincosf(ph[i], &s, &c);
    w[i] = make_float2(amp[i] * c, amp[i] * s);
}

__global__ void k_project(ProjArgs a, const float* __restrict__ means, const float* __restrict__ log_scales,
                          const float* __restrict__ quats, const float* __restrict__ opacity_logits,
                          const float* __restrict__ plane_logits, const float* __restrict__ cam,
                          float4* __restrict__ proj, uint2* __restrict__ rectn, uint32_t* __restrict__ dkey,
                          uint32_t* __restrict__ dval) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)a.V * a.N) return;
    const int v = (int)(i / a.N), n = (int)(i - (size_t)v * a.N);
    ProjF P;
    project_one(a, means + 3 * n, log_scales + 3 * n, quats + 4 * n, opacity_logits[n], cam + 20 * v, P);
#ifdef HCGS_CHECKED
    {   // a Gaussian with a non-finite parameter is reported (and culled)
        bool fin = isfinite(opacity_logits[n]);
        for (int k = 0; k < 3; k++) fin = fin && isfinite(means[3 * n + k]) && isfinite(log_scales[3 * n + k]);
        for (int k = 0; k < 4; k++) fin = fin && isfinite(quats[4 * n + k]);
        for (int l = 0; l < a.L; l++) fin = fin && isfinite(plane_logits[(size_t)n * a.L + l]);
        if (v == 0) HCGS_DCHECK(a.status, fin);
        if (!fin) P.valid = false;
    }
#endif
    int plane = 0;
    {
        const float* r = plane_logits + (size_t)n * a.L;
        float best = r[0];
        for (int l = 1; l < a.L; l++)
            if (r[l] > best) { best = r[l]; plane = l; }  // ties keep the lowest index
    }
    uint2 rect = make_uint2(0u, 0u);  // empty
    if (P.valid) {
        int tx0 = 0, tx1 = a.tilesX, ty0 = 0, ty1 = a.tilesY;
        bool any = true;
        if (a.amin > 0.f) {
            if (P.o < a.amin) {
                any = false;
            } else {
                // support {d : d^T conic d <= 2 ln(o / alpha_min)}: its bounding box,
                // padded so that FP32 rounding never loses a support pixel
                const float k2 = 2.f * logf(P.o / a.amin);
                const float rx = sqrtf(k2 * P.cov[0]) * 1.0001f + 0.01f;
                const float ry = sqrtf(k2 * P.cov[2]) * 1.0001f + 0.01f;
                const float fx0 = floorf((P.mu.x - rx) * (1.f / TILE)), fx1 = floorf((P.mu.x + rx) * (1.f / TILE));
                const float fy0 = floorf((P.mu.y - ry) * (1.f / TILE)), fy1 = floorf((P.mu.y + ry) * (1.f / TILE));
                tx0 = (int)fmaxf(fx0, 0.f);
                ty0 = (int)fmaxf(fy0, 0.f);
                tx1 = (int)fminf(fx1 + 1.f, (float)a.tilesX);
                ty1 = (int)fminf(fy1 + 1.f, (float)a.tilesY);
                any = tx0 < tx1 && ty0 < ty1;
            }
        }
        if (any) rect = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
    }
    proj[2 * i] = make_float4(P.mu.x, P.mu.y, P.conic[0], P.conic[1]);
    proj[2 * i + 1] = make_float4(P.conic[2], P.o, P.depth, __int_as_float(plane));
    rectn[i] = rect;
    // The visiting order's key: the camera-space depth rounded once to FP32.
    // It is formed in FP64 from the FP32 inputs (each product exact), so that
    // Gaussians closer in depth than the rounding error of an FP32 evaluation
    // are still ordered by their depths; equal keys go by index (the sort is
    // stable).  depth >= near_z > 0, so the float bits order like the values.
    if (P.valid) {
        const float* Vm = cam + 20 * v;
        const float* mn = means + 3 * n;
        const double zd = fma((double)Vm[8], (double)mn[0],
                              fma((double)Vm[9], (double)mn[1], fma((double)Vm[10], (double)mn[2], (double)Vm[11])));
        dkey[i] = __float_as_uint(__double2float_rn(zd));
    } else {
        dkey[i] = 0xFFFFFFFFu;
    }
    dval[i] = (uint32_t)n;
}

// Number of visible Gaussians per view: culled ones carry the key ~0u and
// sort last, so it is the position of the first ~0u key (binary search).
__global__ void k_count_visible(const uint32_t* __restrict__ sorted_keys, int N, uint32_t* __restrict__ nvalid) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= gridDim.x * blockDim.x) return;
    const uint32_t* k = sorted_keys + (size_t)v * N;
    int lo = 0, hi = N;  // first index with key == ~0u lies in [lo, hi]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (k[mid] == 0xFFFFFFFFu) hi = mid;
        else lo = mid + 1;
    }
    nvalid[v] = (uint32_t)lo;
}

// Gaussians in visiting order: records for the rasterizer, ranks, and the
// number of coarse buckets each one touches.
__global__ void k_gather(ProjArgs a, const uint32_t* __restrict__ sorted_id, const uint32_t* __restrict__ nvalid,
                         const float4* __restrict__ proj, const uint2* __restrict__ rectn,
                         const float2* __restrict__ w, int order, uint32_t* __restrict__ rank,
                         uint32_t* __restrict__ sortid, float4* __restrict__ rec, uint2* __restrict__ rects,
                         int* __restrict__ planes, uint32_t* __restrict__ ccount) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)a.V * a.N) return;
    const int v = (int)(i / a.N), s = (int)(i - (size_t)v * a.N);
    const int m = (int)nvalid[v];
    const uint32_t n = sorted_id[i];
    const size_t vn = (size_t)v * a.N;
    if (!HCGS_DCHECK(a.status, n < (uint32_t)a.N && m <= a.N)) return;
    if (s >= m) {
        rank[vn + n] = 0xFFFFFFFFu;
        ccount[i] = 0u;
        return;
    }
    const int s2 = order == 1 ? m - 1 - s : s;
    rank[vn + n] = (uint32_t)s2;
    sortid[vn + s2] = n;
    const float4 p0 = proj[2 * (vn + n)], p1 = proj[2 * (vn + n) + 1];
    const int NR = rec_count(a.C);
    float4* r = rec + (vn + s2) * NR;
    const float2* wn = w + (size_t)n * a.C;
    r[0] = p0;
    r[1] = make_float4(p1.x, p1.y, wn[0].x, wn[0].y);
    if (a.C >= 2) r[2] = make_float4(wn[1].x, wn[1].y, a.C >= 3 ? wn[2].x : 0.f, a.C >= 3 ? wn[2].y : 0.f);
    if (a.C >= 4) r[3] = make_float4(wn[3].x, wn[3].y, 0.f, 0.f);
    const uint2 rc = rectn[vn + n];
    rects[vn + s2] = rc;
    planes[vn + s2] = __float_as_int(p1.w);
    const uint32_t tx0 = rc.x & 0xFFFFu, tx1 = rc.x >> 16, ty0 = rc.y & 0xFFFFu, ty1 = rc.y >> 16;
    uint32_t cnt = 0;
    if (tx0 < tx1 && ty0 < ty1) {
        const uint32_t cx0 = tx0 / COARSE, cx1 = (tx1 + COARSE - 1) / COARSE;
        const uint32_t cy0 = ty0 / COARSE, cy1 = (ty1 + COARSE - 1) / COARSE;
        cnt = (cx1 - cx0) * (cy1 - cy0);
    }
    ccount[vn + s2] = cnt;
}

// One instance per (visible Gaussian, covered coarse bucket), in visiting
// order: entry i = (view, rank) owns positions [coff[i], coff[i] + n_i) for
// its buckets [cx0, cx0 + cw) x [cy0, cy0 + ch), row by row.  A warp's 32
// entries own one contiguous range, so the warp writes it 32 instances at a
// time (coalesced), each lane finding the entry that owns its position by a
// binary search over the warp's running counts, instead of one entry per lane.
struct InstSrc {
    uint32_t cnt = 0, start = 0, cw = 1, cx0 = 0, cy0 = 0, kb = 0, s = 0;
};

// The instance source of entry i (view v, visiting rank s): its bucket
// rectangle; kb = the id of the entry's bucket row block (view, plane).
__device__ __forceinline__ InstSrc inst_source(const ProjArgs& a, size_t i, const uint32_t* __restrict__ coff,
                                               const uint2* __restrict__ rects, const int* __restrict__ planes,
                                               const uint32_t* __restrict__ nvalid) {
    InstSrc r;
    if (i >= (size_t)a.V * a.N) return r;
    const int v = (int)(i / a.N), s = (int)(i - (size_t)v * a.N);
    if (s >= (int)nvalid[v]) return r;
    const uint2 rc = rects[i];
    const uint32_t tx0 = rc.x & 0xFFFFu, tx1 = rc.x >> 16, ty0 = rc.y & 0xFFFFu, ty1 = rc.y >> 16;
    if (!(tx0 < tx1 && ty0 < ty1)) return r;
    r.cx0 = tx0 / COARSE;
    r.cy0 = ty0 / COARSE;
    r.cw = (tx1 + COARSE - 1) / COARSE - r.cx0;
    r.cnt = r.cw * ((ty1 + COARSE - 1) / COARSE - r.cy0);
    r.start = coff[i];
    // planes == nullptr: the all-plane lists (bucket id without the plane)
    r.kb = planes ? ((uint32_t)v * a.L + (uint32_t)planes[i]) * a.ctY : (uint32_t)v * a.ctY;
    r.s = (uint32_t)s;
    return r;
}

__device__ __forceinline__ void emit_instances(const InstSrc& e, uint32_t ctX, uint32_t* __restrict__ ikey,
                                               uint32_t* __restrict__ ival, const ProjArgs& a) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t inc = e.cnt;  // inclusive running count over the warp's lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, inc, o);
        if (lane >= o) inc += y;
    }
    const uint32_t total = __shfl_sync(full, inc, 31);
    const uint32_t excl = inc - e.cnt;
    for (uint32_t b0 = 0; b0 < total; b0 += 32) {
        const uint32_t idx = b0 + (uint32_t)lane;
        int j = 0;  // the owner: the number of lanes whose running count is <= idx
#pragma unroll
        for (int b = 16; b > 0; b >>= 1) {
            const uint32_t x = __shfl_sync(full, inc, j + b - 1);
            if (x <= idx) j += b;
        }
        const uint32_t k = idx - __shfl_sync(full, excl, j);
        const uint32_t start = __shfl_sync(full, e.start, j), w = __shfl_sync(full, e.cw, j);
        const uint32_t x0 = __shfl_sync(full, e.cx0, j), y0 = __shfl_sync(full, e.cy0, j);
        const uint32_t kb = __shfl_sync(full, e.kb, j), sv = __shfl_sync(full, e.s, j);
        if (idx < total && HCGS_DCHECK(a.status, start + k < a.M)) {
            const uint32_t dy = k / w, dx = k - dy * w;
            ikey[start + k] = (kb + y0 + dy) * ctX + x0 + dx;
            ival[start + k] = sv;
        }
    }
}

__global__ void k_inst_gen(ProjArgs a, const uint32_t* __restrict__ coff, const uint2* __restrict__ rects,
                           const int* __restrict__ planes, const uint32_t* __restrict__ nvalid,
                           uint32_t* __restrict__ ikey, uint32_t* __restrict__ ival) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i - (threadIdx.x & 31) >= (size_t)a.V * a.N) return;  // the whole warp is past the end
    emit_instances(inst_source(a, i, coff, rects, planes, nvalid), (uint32_t)a.ctX, ikey, ival, a);
}

// The same instances with the plane left out of the bucket id (per view and
// coarse tile, every plane's Gaussians), for the dense plane-weight gradient.
__global__ void k_inst_gen_all(ProjArgs a, const uint32_t* __restrict__ coff, const uint2* __restrict__ rects,
                               const uint32_t* __restrict__ nvalid, uint32_t* __restrict__ ikey,
                               uint32_t* __restrict__ ival) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i - (threadIdx.x & 31) >= (size_t)a.V * a.N) return;
    emit_instances(inst_source(a, i, coff, rects, nullptr, nvalid), (uint32_t)a.ctX, ikey, ival, a);
}

// Bucket start offsets from the sorted bucket ids: off[b] = first position
// whose id >= b; off[NB] = M.
__global__ void k_bucket_bounds(const uint32_t* __restrict__ key, uint32_t M, uint32_t NB, uint32_t* __restrict__ off) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i > M) return;
    const int64_t prev = i > 0 ? (int64_t)key[i - 1] : -1;
    const int64_t cur = i < M ? (int64_t)key[i] : (int64_t)NB;
    for (int64_t b = prev + 1; b <= cur; b++) off[b] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort (8-bit digits), segmented: segments of a fixed length,
// or (segoff given) segment s = [segoff[s], segoff[s + 1]) whose keys all lie
// in [s keystep, (s + 1) keystep) and are sorted on key - s keystep.  The
// segment is the most significant part of the order (the scan of the
// histograms runs segment-major), so the result is the stable sort of the
// whole array when the input is already grouped by segment.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_IPT = 16;
constexpr int RS_KPB = RS_THREADS * RS_IPT;

struct RsSeg {
    size_t so, len;   // start and length of this block's segment
    uint32_t kb;      // subtracted from the keys before the digit is taken
};
__device__ __forceinline__ RsSeg rs_segment(int seg, size_t seglen, const uint32_t* segoff, uint32_t keystep) {
    RsSeg r;
    if (segoff) {
        r.so = segoff[seg];
        r.len = segoff[seg + 1] - segoff[seg];
        r.kb = (uint32_t)seg * keystep;
    } else {
        r.so = (size_t)seg * seglen;
        r.len = seglen;
        r.kb = 0u;
    }
    return r;
}

__global__ void k_rs_hist(const uint32_t* __restrict__ keys, size_t seglen, const uint32_t* __restrict__ segoff,
                          uint32_t keystep, int shift, uint32_t mask, int nblk, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    const int seg = blockIdx.y, blk = blockIdx.x;
    h[threadIdx.x] = 0;
    __syncthreads();
    const RsSeg sg = rs_segment(seg, seglen, segoff, keystep);
    const size_t beg = (size_t)blk * RS_KPB;
    const uint32_t* k = keys + sg.so;
#pragma unroll
    for (int r = 0; r < RS_IPT; r++) {
        const size_t idx = beg + (size_t)r * RS_THREADS + threadIdx.x;
        if (idx < sg.len) atomicAdd(&h[((k[idx] - sg.kb) >> shift) & mask], 1u);
    }
    __syncthreads();
    hist[((size_t)seg * 256 + threadIdx.x) * nblk + blk] = h[threadIdx.x];
}

// One pass of the stable scatter.  Warp w owns the block's elements
// [256 w, 256 w + 256) and ranks them in input order, 32 at a time, against
// its own digit counters (warp match; the leader of each digit group advances
// the counter and broadcasts the old value), with no block barrier between
// rounds.  One scan over (digit, warp) then gives every element its place in
// the block's digit-sorted order; the elements are staged in shared memory in
// that order and written out so that consecutive threads write consecutive
// addresses of a digit's output run (instead of 4-byte writes scattered over
// 256 runs).
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           size_t seglen, const uint32_t* __restrict__ segoff,
                                                           uint32_t keystep, int shift, uint32_t mask, int nblk,
                                                           const uint32_t* __restrict__ pos) {
    constexpr int NW = RS_THREADS / 32, PW = RS_KPB / NW;  // warps, elements per warp
    __shared__ uint32_t wh[NW][256];  // per-warp digit counters, then per-warp bases within a digit
    __shared__ uint32_t gbase[256], loff[256], wsum[NW];
    __shared__ uint32_t sk[RS_KPB], sv[RS_KPB];
    const int seg = blockIdx.y, blk = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const RsSeg sg = rs_segment(seg, seglen, segoff, keystep);
    const size_t beg = (size_t)blk * RS_KPB;
    if (beg >= sg.len) return;  // past the end of a shorter segment (uniform over the block)
    const size_t so = sg.so;
    const uint32_t kb = sg.kb;
    const int nb = (int)min((size_t)RS_KPB, sg.len - beg);  // elements of this block
    for (int e = t; e < NW * 256; e += RS_THREADS) (&wh[0][0])[e] = 0;
    gbase[t] = pos[((size_t)seg * 256 + t) * nblk + blk];
    uint32_t key[RS_IPT], val[RS_IPT], rk[RS_IPT];
#pragma unroll
    for (int r = 0; r < RS_IPT; r++) {
        const int i = warp * PW + r * 32 + lane;
        key[r] = i < nb ? kin[so + beg + i] : 0u;
        val[r] = i < nb ? vin[so + beg + i] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_IPT; r++) {
        const bool ok = warp * PW + r * 32 + lane < nb;
        const uint32_t d = ok ? (((key[r] - kb) >> shift) & mask) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        const uint32_t lrank = __popc(peers & lt);
        uint32_t old = (ok && lrank == 0) ? wh[warp][d] : 0u;
        old = __shfl_sync(0xffffffffu, old, leader);
        if (ok && lrank == 0) wh[warp][d] = old + __popc(peers);
        rk[r] = old + lrank;
        __syncwarp();
    }
    __syncthreads();
    // thread t = digit t: bases of the warps within the digit, and the
    // block's exclusive scan of the digit totals
    {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const uint32_t x = wh[w][t];
            wh[w][t] = c;
            c += x;
        }
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t wb = 0;
        for (int w = 0; w < warp; w++) wb += wsum[w];
        loff[t] = wb + inc - c;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_IPT; r++) {
        if (warp * PW + r * 32 + lane < nb) {
            const uint32_t d = ((key[r] - kb) >> shift) & mask;
            const uint32_t lp = loff[d] + wh[warp][d] + rk[r];
            sk[lp] = key[r];
            sv[lp] = val[r];
        }
    }
    __syncthreads();
    for (int i = t; i < nb; i += RS_THREADS) {
        const uint32_t k = sk[i];
        const uint32_t d = ((k - kb) >> shift) & mask;
        const uint32_t p = gbase[d] + (uint32_t)i - loff[d];
        kout[p] = k;
        vout[p] = sv[i];
    }
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 counts
// ---------------------------------------------------------------------------
constexpr int SC_THREADS = 512;
constexpr int SC_IPT = 8;
constexpr int SC_EPB = SC_THREADS * SC_IPT;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* total) {
    __shared__ uint32_t ws[SC_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < SC_THREADS / 32 ? ws[lane] : 0u;
        uint32_t vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        if (lane < SC_THREADS / 32) ws[lane] = vi - v;
        if (lane == SC_THREADS / 32 - 1) *total = vi;
    }
    __syncthreads();
    const uint32_t r = ws[warp] + inc - x;
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, size_t n, uint32_t* __restrict__ bsum) {
    const size_t beg = (size_t)blockIdx.x * SC_EPB + (size_t)threadIdx.x * SC_IPT;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SC_IPT; k++)
        if (beg + k < n) s += in[beg + k];
    __shared__ uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Second pass: block b starts from the sum of the block sums before it
// (summed here, in 64 bits, by the whole block: no separate pass over the
// block sums), scans its own elements and writes them; the last block also
// writes the 64-bit total (for overflow detection).
__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, size_t n,
                             const uint32_t* __restrict__ bsum, int nb, unsigned long long* __restrict__ total64) {
    __shared__ unsigned long long red[SC_THREADS / 32];
    __shared__ unsigned long long base_s;
    unsigned long long part = 0;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += SC_THREADS) part += bsum[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < SC_THREADS / 32; w++) t += red[w];
        base_s = t;
        if ((int)blockIdx.x == nb - 1) *total64 = t + bsum[nb - 1];
    }
    __syncthreads();
    const uint32_t base = (uint32_t)base_s;
    const size_t beg = (size_t)blockIdx.x * SC_EPB + (size_t)threadIdx.x * SC_IPT;
    uint32_t v[SC_IPT];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SC_IPT; k++) {
        v[k] = beg + k < n ? in[beg + k] : 0u;
        s += v[k];
    }
    __shared__ uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot) + base;
#pragma unroll
    for (int k = 0; k < SC_IPT; k++)
        if (beg + k < n) {
            out[beg + k] = run;
            run += v[k];
        }
}

static size_t scan_bsum_bytes(size_t n) {
    const size_t nb = (n + SC_EPB - 1) / SC_EPB;
    return ((nb * sizeof(uint32_t) + 7) / 8) * 8;
}

hcgs_status exclusive_scan(hcgs_ctx* ctx, hcgs_saved* s, const uint32_t* in, uint32_t* out, size_t n,
                           cudaStream_t st) {
    if (n == 0) return HCGS_OK;
    const size_t nb = (n + SC_EPB - 1) / SC_EPB;
    HCGS_CUDA(ctx, grow(ctx, s->scan, scan_bsum_bytes(n) + 8, &s->bytes));
    uint32_t* bsum = (uint32_t*)s->scan.p;
    unsigned long long* t64 = (unsigned long long*)((char*)s->scan.p + scan_bsum_bytes(n));
    HCGS_KERNEL(ctx, "k_scan_reduce", st, k_scan_reduce<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, n, bsum));
    HCGS_KERNEL(ctx, "k_scan_apply", st,
                k_scan_apply<<<(unsigned)nb, SC_THREADS, 0, st>>>(in, out, n, bsum, (int)nb, t64));
    HCGS_LAUNCH(ctx, "exclusive_scan");
    return HCGS_OK;
}

// the 64-bit total of the last exclusive_scan over n elements
static const unsigned long long* scan_total_ptr(hcgs_saved* s, size_t n) {
    return (const unsigned long long*)((char*)s->scan.p + scan_bsum_bytes(n));
}

// Segments of the bucket-instance array by view (instances are generated
// view-major: view v owns [coff[v N], coff[(v + 1) N])): segoff[v] for
// v < V, segoff[V] = M, and segoff[V + 1] = the most instances of one view.
__global__ void k_view_segments(const uint32_t* __restrict__ coff, const unsigned long long* __restrict__ total,
                                int V, int N, uint32_t* __restrict__ segoff) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const uint32_t M = (uint32_t)*total;
    uint32_t prev = 0, most = 0;
    for (int v = 0; v <= V; v++) {
        const uint32_t o = v < V ? coff[(size_t)v * N] : M;
        segoff[v] = o;
        if (v > 0) most = max(most, o - prev);
        prev = o;
    }
    segoff[V + 1] = most;
}

// keys / vals hold two buffers of ``total`` elements each (the passes
// ping-pong between them); *which tells the one holding the result.  Without
// segoff: nseg segments of seglen elements; with segoff (device, nseg + 1
// offsets): seglen is the longest segment.
hcgs_status radix_sort(hcgs_ctx* ctx, hcgs_saved* s, uint32_t* keys, uint32_t* vals, int nseg, size_t seglen,
                       size_t total, const uint32_t* segoff, uint32_t keystep, int nbits, int* which,
                       cudaStream_t st) {
    *which = 0;
    if (seglen == 0 || nseg == 0) return HCGS_OK;
    const int nblk = (int)((seglen + RS_KPB - 1) / RS_KPB);
    const size_t nh = (size_t)nseg * 256 * nblk;
    HCGS_CUDA(ctx, grow(ctx, s->hist, nh * sizeof(uint32_t), &s->bytes));
    uint32_t* hist = (uint32_t*)s->hist.p;
    int cur = 0;
    // as few passes of at most 8 bits as cover nbits, the bits split evenly
    // between them (13 bits: 7 + 6 rather than 8 + 5, so that the first
    // pass scatters into fewer, longer runs)
    const int npass = (nbits + 7) / 8;
    const int width = (nbits + npass - 1) / npass;
    for (int shift = 0; shift < nbits; shift += width) {
        const uint32_t mask = (1u << width) - 1u;
        uint32_t* kin = keys + (size_t)cur * total;
        uint32_t* vin = vals + (size_t)cur * total;
        uint32_t* kout = keys + (size_t)(1 - cur) * total;
        uint32_t* vout = vals + (size_t)(1 - cur) * total;
        dim3 grid(nblk, nseg);
        HCGS_KERNEL(ctx, "k_rs_hist", st,
                    k_rs_hist<<<grid, RS_THREADS, 0, st>>>(kin, seglen, segoff, keystep, shift, mask, nblk, hist));
        HCGS_LAUNCH(ctx, "k_rs_hist");
        hcgs_status e = exclusive_scan(ctx, s, hist, hist, nh, st);
        if (e) return e;
        HCGS_KERNEL(ctx, "k_rs_scatter", st,
                    k_rs_scatter<<<grid, RS_THREADS, 0, st>>>(kin, vin, kout, vout, seglen, segoff, keystep, shift,
                                                              mask, nblk, hist));
        HCGS_LAUNCH(ctx, "k_rs_scatter");
        cur = 1 - cur;
    }
    *which = cur;
    return HCGS_OK;
}

// ---------------------------------------------------------------------------
// orchestration of steps 1-2
// ---------------------------------------------------------------------------
static int bits_for(uint64_t n) {
    int b = 1;
    while ((1ull << b) < n) b++;
    return b;
}

hcgs_status project_and_bin(hcgs_ctx* ctx, hcgs_saved* s, const hcgs_gaussians* g, const float* viewmats,
                            const float* intr, cudaStream_t st) {
    const int V = s->V, N = s->N, C = s->C, L = s->L;
    const size_t VN = (size_t)V * N;
    const int NR = rec_count(C);
    size_t* ob = &s->bytes;
    HCGS_CUDA(ctx, grow(ctx, s->w, (size_t)N * C * sizeof(float2), ob));
    HCGS_CUDA(ctx, grow(ctx, s->proj, VN * 2 * sizeof(float4), ob));
    HCGS_CUDA(ctx, grow(ctx, s->rectn, VN * sizeof(uint2), ob));
    HCGS_CUDA(ctx, grow(ctx, s->dkey, 2 * VN * sizeof(uint32_t), ob));
    HCGS_CUDA(ctx, grow(ctx, s->dval, 2 * VN * sizeof(uint32_t), ob));
    HCGS_CUDA(ctx, grow(ctx, s->nvalid, V * sizeof(uint32_t), ob));
    HCGS_CUDA(ctx, grow(ctx, s->rank, VN * sizeof(uint32_t), ob));
    HCGS_CUDA(ctx, grow(ctx, s->sortid, VN * sizeof(uint32_t), ob));
    HCGS_CUDA(ctx, grow(ctx, s->rec, VN * NR * sizeof(float4), ob));
    HCGS_CUDA(ctx, grow(ctx, s->rects, VN * sizeof(uint2), ob));
    HCGS_CUDA(ctx, grow(ctx, s->planes, VN * sizeof(int), ob));
    HCGS_CUDA(ctx, grow(ctx, s->ccount, VN * sizeof(uint32_t), ob));
    HCGS_CUDA(ctx, grow(ctx, s->cam, (size_t)V * 20 * sizeof(float), ob));
    const size_t NB = (size_t)V * L * s->ctX * s->ctY;
    HCGS_CUDA(ctx, grow(ctx, s->bcount, (NB + 1) * sizeof(uint32_t), ob));

    float* cam = (float*)s->cam.p;
    for (int v = 0; v < V; v++) {
        HCGS_CUDA(ctx, cudaMemcpyAsync(cam + 20 * v, viewmats + 16 * v, 16 * sizeof(float), cudaMemcpyDeviceToDevice, st));
        HCGS_CUDA(ctx, cudaMemcpyAsync(cam + 20 * v + 16, intr + 4 * v, 4 * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    ProjArgs a = make_proj_args(s);
    a.status = ctx->d_status;
    const int T = 256;
    HCGS_KERNEL(ctx, "k_prep_w", st, k_prep_w<<<(N * C + T - 1) / T, T, 0, st>>>(g->amplitude, g->phase, (float2*)s->w.p, N, C, ctx->d_status));
    const unsigned gridVN = (unsigned)((VN + T - 1) / T);
    uint32_t* dkey = (uint32_t*)s->dkey.p;
    uint32_t* dval = (uint32_t*)s->dval.p;
    HCGS_KERNEL(ctx, "k_project", st, k_project<<<gridVN, T, 0, st>>>(a, g->means, g->log_scales, g->quats, g->opacity_logits, g->plane_logits, cam,
                                    (float4*)s->proj.p, (uint2*)s->rectn.p, dkey, dval));
    HCGS_LAUNCH(ctx, "k_project");
    int which = 0;
    hcgs_status e = radix_sort(ctx, s, dkey, dval, V, N, VN, nullptr, 0u, 32, &which, st);
    if (e) return e;
    HCGS_KERNEL(ctx, "k_count_visible", st, k_count_visible<<<V, 1, 0, st>>>(dkey + (size_t)which * VN, N, (uint32_t*)s->nvalid.p));
    HCGS_KERNEL(ctx, "k_gather", st, k_gather<<<gridVN, T, 0, st>>>(a, dval + (size_t)which * VN, (const uint32_t*)s->nvalid.p,
                                   (const float4*)s->proj.p, (const uint2*)s->rectn.p, (const float2*)s->w.p,
                                   s->opts.order, (uint32_t*)s->rank.p, (uint32_t*)s->sortid.p, (float4*)s->rec.p,
                                   (uint2*)s->rects.p, (int*)s->planes.p, (uint32_t*)s->ccount.p));
    HCGS_LAUNCH(ctx, "k_gather");
    uint32_t* coff = (uint32_t*)s->ccount.p;
    if ((e = exclusive_scan(ctx, s, coff, coff, VN, st))) return e;
    HCGS_CUDA(ctx, grow(ctx, s->segoff, (size_t)(V + 2) * sizeof(uint32_t), ob));
    uint32_t* segoff = (uint32_t*)s->segoff.p;
    HCGS_KERNEL(ctx, "k_view_segments", st, k_view_segments<<<1, 32, 0, st>>>(coff, scan_total_ptr(s, VN), V, N, segoff));
    // the instance count sizes the instance buffers and the longest view the
    // sort's grid: one readback
    HCGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, scan_total_ptr(s, VN), 8, cudaMemcpyDeviceToHost, st));
    HCGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 3, segoff + V + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    // the device status word rides along: a bounded wait that ran out in an
    // earlier launch of this context is reported here
    HCGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 2, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HCGS_CUDA(ctx, cudaStreamSynchronize(st));
    if (ctx->h_pinned[2] != 0) {
        const uint32_t w = ctx->h_pinned[2];
        HCGS_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
        if (w & STATUS_DEVICE_CHECK) {
            set_err(ctx, HCGS_ERR_DEVICE_CHECK, "a device-side bounds or input check failed in an earlier launch");
            return HCGS_ERR_DEVICE_CHECK;
        }
        set_err(ctx, HCGS_ERR_TIMEOUT, "a bounded device wait ran out in an earlier launch");
        return HCGS_ERR_TIMEOUT;
    }
    const unsigned long long M = *(unsigned long long*)ctx->h_pinned;
    if (M >= (1ull << 31)) {
        set_err(ctx, HCGS_ERR_CAPACITY, "more than 2^31 bucket instances");
        return HCGS_ERR_CAPACITY;
    }
    s->M = M;
    a.M = (uint32_t)M;
    const size_t Mc = M > 0 ? (size_t)M : 1;
    HCGS_CUDA(ctx, grow(ctx, s->ikey, 2 * Mc * sizeof(uint32_t), ob));
    HCGS_CUDA(ctx, grow(ctx, s->ival, 2 * Mc * sizeof(uint32_t), ob));
    uint32_t* ikey = (uint32_t*)s->ikey.p;
    uint32_t* ival = (uint32_t*)s->ival.p;
    HCGS_KERNEL(ctx, "k_inst_gen", st, k_inst_gen<<<gridVN, T, 0, st>>>(a, coff, (const uint2*)s->rects.p, (const int*)s->planes.p,
                                     (const uint32_t*)s->nvalid.p, ikey, ival));
    HCGS_LAUNCH(ctx, "k_inst_gen");
    // bucket ids are view-major (v L ctY ctX + within-view bucket) and the
    // instances already grouped by view: each view's segment is sorted on its
    // within-view bucket (fewer key bits, fewer passes than the whole id)
    const uint32_t NBv = (uint32_t)(L * s->ctX * s->ctY);
    const size_t most = ctx->h_pinned[3];
    if ((e = radix_sort(ctx, s, ikey, ival, V, most, (size_t)M, segoff, NBv, bits_for(NBv), &which, st))) return e;
    const uint32_t* skey = ikey + (size_t)which * M;
    s->list = ival + (size_t)which * M;
    HCGS_KERNEL(ctx, "k_bucket_bounds", st, k_bucket_bounds<<<(unsigned)((M + 1 + T - 1) / T), T, 0, st>>>(skey, (uint32_t)M, (uint32_t)NB,
                                                                  (uint32_t*)s->bcount.p));
    HCGS_LAUNCH(ctx, "k_bucket_bounds");
    if (s->opts.rho_grad) {
        // all-plane lists: the same instances bucketed by (view, coarse tile)
        const size_t NBA = (size_t)V * s->ctX * s->ctY;
        HCGS_CUDA(ctx, grow(ctx, s->akey, 2 * Mc * sizeof(uint32_t), ob));
        HCGS_CUDA(ctx, grow(ctx, s->aval, 2 * Mc * sizeof(uint32_t), ob));
        HCGS_CUDA(ctx, grow(ctx, s->abcount, (NBA + 1) * sizeof(uint32_t), ob));
        uint32_t* akey = (uint32_t*)s->akey.p;
        uint32_t* aval = (uint32_t*)s->aval.p;
        HCGS_KERNEL(ctx, "k_inst_gen_all", st, k_inst_gen_all<<<gridVN, T, 0, st>>>(a, coff, (const uint2*)s->rects.p,
                                                                             (const uint32_t*)s->nvalid.p, akey, aval));
        const uint32_t NBAv = (uint32_t)(s->ctX * s->ctY);
        if ((e = radix_sort(ctx, s, akey, aval, V, most, (size_t)M, segoff, NBAv, bits_for(NBAv), &which, st)))
            return e;
        s->alist = aval + (size_t)which * M;
        HCGS_KERNEL(ctx, "k_bucket_bounds", st,
                    k_bucket_bounds<<<(unsigned)((M + 1 + T - 1) / T), T, 0, st>>>(akey + (size_t)which * M, (uint32_t)M,
                                                                                (uint32_t)NBA, (uint32_t*)s->abcount.p));
    }
    return HCGS_OK;
}

// ---------------------------------------------------------------------------
// adjoint of the projection (Supp. D.4) and of the plane argmax (Eq. ste)
// ---------------------------------------------------------------------------
__global__ void k_project_bwd(ProjArgs a, const float* __restrict__ means, const float* __restrict__ log_scales,
                              const float* __restrict__ quats, const float* __restrict__ opacity_logits,
                              const float* __restrict__ amplitude, const float* __restrict__ phase,
                              const float* __restrict__ plane_logits, const float* __restrict__ cam,
                              const uint32_t* __restrict__ rank, const float* __restrict__ g2d, float ste_tau,
                              const float* __restrict__ drho_dense, hcgs_gaussian_grads gr, int accumulate) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= a.N) return;
    const int C = a.C, G = g2d_count(C);
    float gm[3] = {0, 0, 0}, gls[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0};
    float gsig[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // dL/dSigma summed over the views
    bool any = false;
    float gol = 0.f, drho = 0.f;
    float gwr[MAX_C] = {0, 0, 0, 0}, gwi[MAX_C] = {0, 0, 0, 0};
    for (int v = 0; v < a.V; v++) {
        const uint32_t s = rank[(size_t)v * a.N + n];
        if (s == 0xFFFFFFFFu) continue;
        const float* g = g2d + ((size_t)v * a.N + n) * G;
        for (int c = 0; c < C; c++) {
            gwr[c] += g[6 + 2 * c];
            gwi[c] += g[7 + 2 * c];
        }
        ProjF P;
        project_one(a, means + 3 * n, log_scales + 3 * n, quats + 4 * n, opacity_logits[n], cam + 20 * v, P);
        if (!P.valid) continue;
        // slot 5 holds o dL/do: dL/dlogit = o (1 - o) dL/do, and dL/drho =
        // o G dL/dalpha summed = o dL/do for the assigned plane
        const float ogo = g[5];
        gol += ogo * (1.f - P.o);
        drho += ogo;
        // the rasterizer's adjoint leaves the pixel moments of p = -dL/dpower
        // (sum dx p, sum dy p, sum dx^2 p, sum dx dy p, sum dy^2 p); with
        // power = 1/2 (A dx^2 + C dy^2) + B dx dy, d = pixel - mu:
        const float A = P.conic[0], B = P.conic[1], Cc = P.conic[2];
        const float2 gmu = make_float2(fmaf(A, g[0], B * g[1]), fmaf(B, g[0], Cc * g[1]));
        project_one_backward(a, P, cam + 20 * v, gmu, -0.5f * g[2], -g[3], -0.5f * g[4], gm, gsig);
        any = true;
    }
    if (any) {
        ProjF Q;
        sigma_factors(log_scales + 3 * n, quats + 4 * n, Q);
        sigma_backward(Q, gsig, gls, gq);
    }
    // appearance: w_c = a_c (cos phi_c, sin phi_c)
    for (int c = 0; c < C; c++) {
        float sn, cs;
        sincosf(phase[n * C + c], &sn, &cs);
        const float ga = gwr[c] * cs + gwi[c] * sn;
        const float gp = amplitude[n * C + c] * (-gwr[c] * sn + gwi[c] * cs);
        if (accumulate) {
            gr.amplitude[n * C + c] += ga;
            gr.phase[n * C + c] += gp;
        } else {
            gr.amplitude[n * C + c] = ga;
            gr.phase[n * C + c] = gp;
        }
    }
    // straight-through plane logits: elementwise product with softmax(rho'/tau)
    const float* r = plane_logits + (size_t)n * a.L;
    int am = 0;
    float mx = r[0];
    for (int l = 1; l < a.L; l++)
        if (r[l] > mx) { mx = r[l]; am = l; }
    float Z = 0.f;
    for (int l = 0; l < a.L; l++) Z += expf((r[l] - mx) / ste_tau);
    const float sm_a = 1.f / Z;  // softmax at the argmax: exp(0) / Z
    for (int l = 0; l < a.L; l++) {
        // dense mode: the unassigned planes' weights, times their softmax values
        const float gv = l == am ? drho * sm_a
                                 : (drho_dense ? drho_dense[(size_t)n * a.L + l] * (expf((r[l] - mx) / ste_tau) / Z)
                                               : 0.f);
        if (accumulate) gr.plane_logits[(size_t)n * a.L + l] += gv;
        else gr.plane_logits[(size_t)n * a.L + l] = gv;
    }
    if (accumulate) {
        for (int k = 0; k < 3; k++) { gr.means[3 * n + k] += gm[k]; gr.log_scales[3 * n + k] += gls[k]; }
        for (int k = 0; k < 4; k++) gr.quats[4 * n + k] += gq[k];
        gr.opacity_logits[n] += gol;
    } else {
        for (int k = 0; k < 3; k++) { gr.means[3 * n + k] = gm[k]; gr.log_scales[3 * n + k] = gls[k]; }
        for (int k = 0; k < 4; k++) gr.quats[4 * n + k] = gq[k];
        gr.opacity_logits[n] = gol;
    }
}

hcgs_status project_backward(hcgs_ctx* ctx, hcgs_saved* s, const hcgs_gaussians* g,
                             const hcgs_gaussian_grads* gr, int accumulate, cudaStream_t st) {
    ProjArgs a = make_proj_args(s);
    a.status = ctx->d_status;
    HCGS_KERNEL(ctx, "k_project_bwd", st, k_project_bwd<<<(s->N + 127) / 128, 128, 0, st>>>(a, g->means, g->log_scales, g->quats, g->opacity_logits,
                                                      g->amplitude, g->phase, g->plane_logits,
                                                      (const float*)s->cam.p, (const uint32_t*)s->rank.p,
                                                      (const float*)s->g2d.p, s->opts.ste_tau,
                                                      s->opts.rho_grad ? (const float*)s->drho.p : nullptr, *gr,
                                                      accumulate));
    HCGS_LAUNCH(ctx, "k_project_bwd");
    return HCGS_OK;
}

}  // namespace hcgs
