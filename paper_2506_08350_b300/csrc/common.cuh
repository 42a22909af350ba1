// Internal declarations shared by the libhcgs translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "hcgs.h"

namespace hcgs {

constexpr int TILE = 16;            // tile edge in pixels (Sec. 4.2)
constexpr int MAX_C = 4;            // wavelengths
constexpr int MAX_L = 16;           // depth planes
constexpr int MAX_FFT = 4096;       // longest supported transform
constexpr int MAX_STAGES = 16;
constexpr int COARSE = 4;          // fine tiles per coarse-bucket edge (64 x 64 px)

// Device scratch buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Mixed-radix plan for one transform length (radices 2, 3, 4, 5, 8).
struct FftPlan {
    int n = 0;
    int nst = 0;
    int radix[MAX_STAGES] = {0};
    float2* tw = nullptr;  // device [n]: exp(-2 pi i m / n), formed in FP64
};

struct FftPlanArg {  // by-value kernel argument
    int n, nst;
    int radix[MAX_STAGES];
};

// Per-(geometry, optics) transfer-function table: quadrant of H_z, because
// H depends on f_x^2 and f_y^2 only.  Hq[c][l][H/2+1][hq_stride(W)] float2.
struct HKey {
    int H, W, C, L, band_limit;
    double px, py;
    std::vector<double> lam, z;
    bool operator<(const HKey& o) const {
        return std::tie(H, W, C, L, band_limit, px, py, lam, z) <
               std::tie(o.H, o.W, o.C, o.L, o.band_limit, o.px, o.py, o.lam, o.z);
    }
};

// Per-launch CUDA events, recorded only while profiling is on.
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
struct Prof {
    bool on = false;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
};

}  // namespace hcgs

struct hcgs_ctx {
    hcgs::Prof prof;
    int device = 0;
    std::string last_error;
    size_t bytes = 0;
    hcgs::DevBuf ws[10];                             // workspace slots (6, 7: zero-padded grids; 8, 9: phase-only conversion)
    hcgs::DevBuf selftest;                           // target of hcgs_selftest_device_check
    std::vector<cudaStream_t> streams;               // streams this context's kernels were launched on
    std::map<int, hcgs::FftPlan> plans;              // FFT plans by length
    std::map<hcgs::HKey, hcgs::DevBuf> htab;         // transfer-function tables
    int* d_status = nullptr;                         // device status word
    uint32_t* h_pinned = nullptr;                    // pinned host words
    hcgs_saved* scratch_saved = nullptr;             // used when render_view gets NULL
};

struct hcgs_saved {
    // geometry of the last hcgs_project
    int V = 0, N = 0, L = 0, C = 0, H = 0, W = 0;
    int tilesX = 0, tilesY = 0, ctX = 0, ctY = 0;  // fine and coarse tile grids
    int valid = 0;         // 1 after hcgs_project
    int rastered = 0;      // 1 after hcgs_rasterize_planes
    int have_g2d = 0;      // 1 after hcgs_rasterize_planes_backward
    hcgs_raster_opts opts{};
    hcgs_optics optics{};
    std::vector<double> lam, z;
    uint64_t M = 0;        // coarse-bucket instances over all views
    // buffers
    hcgs::DevBuf w;        // [N][C] float2: c e^{j phi}
    hcgs::DevBuf proj;     // [V][N][2] float4 projected record, by Gaussian id
    hcgs::DevBuf rectn;    // [V][N] uint2 fine-tile rectangle, by Gaussian id
    hcgs::DevBuf dkey;     // [2][V][N] uint32 depth keys (sort ping-pong)
    hcgs::DevBuf dval;     // [2][V][N] uint32 Gaussian ids
    hcgs::DevBuf nvalid;   // [V] uint32 number of visible Gaussians per view
    hcgs::DevBuf segoff;   // [V + 2] uint32 first instance of each view, M, the most instances of a view
    hcgs::DevBuf rank;     // [V][N] uint32 visiting rank of Gaussian n (~0u if culled)
    hcgs::DevBuf sortid;   // [V][N] uint32 Gaussian id at visiting rank s
    hcgs::DevBuf rec;      // [V][N][NR] float4 records in visiting order
    hcgs::DevBuf rects;    // [V][N] uint2 fine-tile rectangle in visiting order
    hcgs::DevBuf planes;   // [V][N] int32 plane in visiting order
    hcgs::DevBuf ccount;   // [V*N] uint32 coarse tiles per record, then offsets
    hcgs::DevBuf bcount;   // [V*L*CT + 1] uint32 bucket counts, then offsets
    hcgs::DevBuf ikey;     // [2][M] uint32 instance bucket ids (sort ping-pong)
    hcgs::DevBuf ival;     // [2][M] uint32 instance visiting ranks
    hcgs::DevBuf hist;     // radix-sort block histograms
    hcgs::DevBuf scan;     // scan partials
    hcgs::DevBuf Tfin;     // [V][L][H][W] float
    hcgs::DevBuf last;     // [V][L][H][W] uint32: staged index after the last contributor
    hcgs::DevBuf slist;    // [32 M] uint32: per 16x8 strip, the Gaussians its forward pass kept, in order
    hcgs::DevBuf U;        // [V][L][C][H][W] float2 when the caller gives no plane buffer
    hcgs::DevBuf g2d;      // [V][N][G2D] float (Gaussian order): pixel moments of -dL/dpower 5, o dL/do, dL/dw 2C
    hcgs::DevBuf gU;       // [V][L][C][H][W] float2 plane gradients
    hcgs::DevBuf cam;      // [V][20] float copies of the view matrices and intrinsics
    // dense plane-weight gradient (opts.rho_grad = 1 only)
    hcgs::DevBuf akey, aval;  // [2][M] all-plane instance bucket ids / ranks (sort ping-pong)
    hcgs::DevBuf abcount;     // [V*CT + 1] all-plane bucket offsets
    hcgs::DevBuf drho;        // [N][L] float dL/drho of the unassigned planes, summed over views
    const uint32_t* alist = nullptr;  // sorted all-plane instance ranks (points into aval)
    const uint32_t* list = nullptr;  // sorted instance ranks (points into ival)
    size_t bytes = 0;
};

namespace hcgs {

// Row stride (complex elements) of the transfer-function quadrant table:
// W/2 + 1 rounded up to even, so that every row starts on a 16-byte boundary
// and spans a multiple of 16 bytes (whole rows are moved by bulk copies).
__host__ __device__ constexpr int hq_stride(int W) { return (W / 2 + 2) & ~1; }

// ---- bulk asynchronous copies into shared memory, completed on mbarriers ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// the calling thread arrives and announces `bytes` of copies for this phase
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// dst (shared) and src (global) 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// orders earlier generic-proxy accesses of shared memory before later bulk copies
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Waits for phase `parity` of the barrier for at most ~1 s of SM clock;
// false if it did not complete by then.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const uint32_t a = smem_addr(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}
// status word bits set by kernels (read back by the host at its next sync)
constexpr int STATUS_WAIT_TIMEOUT = 1;
constexpr int STATUS_DEVICE_CHECK = 2;  // a bounds / input check failed (HCGS_CHECKED builds)

// Device-side checks of the bounds-checked build (HCGS_CHECKED): a failed
// check records STATUS_DEVICE_CHECK in the status word and evaluates to
// false, so the caller skips the access it guards.  In the regular build the
// check compiles away (true).
#ifdef HCGS_CHECKED
#define HCGS_DCHECK(status, cond) ((cond) ? true : (atomicOr((status), hcgs::STATUS_DEVICE_CHECK), false))
#else
#define HCGS_DCHECK(status, cond) true
#endif

// ---- error plumbing ----
struct Err {
    hcgs_status s;
    std::string msg;
};
bool set_err(hcgs_ctx* ctx, hcgs_status s, const std::string& m);
hcgs_status cuda_err(hcgs_ctx* ctx, cudaError_t e, const char* what);
cudaError_t grow(hcgs_ctx* ctx, DevBuf& b, size_t bytes, size_t* owner_bytes);
void free_buf(DevBuf& b);
// Guard bands of the bounds-checked build: every buffer the library grows
// carries GUARD_BYTES of a fixed pattern after its capacity; hcgs_check_status
// verifies them.  Empty in the regular build.
constexpr size_t GUARD_BYTES = 256;
constexpr unsigned char GUARD_FILL = 0xA5;

#define HCGS_CUDA(ctx, call)                                        \
    do {                                                            \
        cudaError_t e__ = (call);                                   \
        if (e__ != cudaSuccess) return hcgs::cuda_err(ctx, e__, #call); \
    } while (0)
#define HCGS_LAUNCH(ctx, what)                                      \
    do {                                                            \
        cudaError_t e__ = cudaGetLastError();                       \
        if (e__ != cudaSuccess) return hcgs::cuda_err(ctx, e__, what); \
    } while (0)

// ---- per-kernel timing ----
void prof_begin(hcgs_ctx* ctx, const char* name, cudaStream_t st);
void prof_end(hcgs_ctx* ctx, cudaStream_t st);
// Launch a kernel between two profiling events.
#define HCGS_KERNEL(ctx, name, st, ...)        \
    do {                                       \
        hcgs::prof_begin(ctx, name, st);       \
        __VA_ARGS__;                           \
        hcgs::prof_end(ctx, st);               \
        HCGS_LAUNCH(ctx, name);                \
    } while (0)

// ---- FFT / ASM (fft.cu) ----
bool fft_supported(int n);
hcgs_status get_plan(hcgs_ctx* ctx, int n, FftPlan** out);
hcgs_status get_htab(hcgs_ctx* ctx, const hcgs_optics* o, const float2** out);
// Batched column transforms of `nplanes` H x W complex planes (in place allowed).
hcgs_status fft_cols(hcgs_ctx* ctx, const float2* in, float2* out, int nplanes, int H, int W, bool inverse,
                     float scale, cudaStream_t st);
// sum mode: out[b][c] = IDFT_rows( sum_l Hsel(c,l) DFT_rows(in[b][l][c]) ), unscaled.
hcgs_status rows_sum(hcgs_ctx* ctx, const float2* in, float2* out, int B, int L, int C, int H, int W,
                     const float2* hq, bool conjH, cudaStream_t st);
// spread mode: out[b][l][c] = IDFT_rows( Hsel(c,l) DFT_rows(in[b][c]) ), unscaled.
hcgs_status rows_spread(hcgs_ctx* ctx, const float2* in, float2* out, int B, int L, int C, int H, int W,
                        const float2* hq, bool conjH, cudaStream_t st);
// Column pass of the focal-stack loss: inverse column DFT (scaled), intensity,
// loss partials, dL/dV, forward column DFT of dL/dV, in place.
hcgs_status cols_focal_loss(hcgs_ctx* ctx, float2* data, const float* I_gt, float* I_out, float* partials,
                            int nplanes, int H, int W, float inv_count, float scale, int* nblocks_out,
                            cudaStream_t st);
hcgs_status asm_sum(hcgs_ctx* ctx, const float2* in, float2* out, int B, const hcgs_optics* o, bool conjH,
                    cudaStream_t st);
hcgs_status asm_spread(hcgs_ctx* ctx, const float2* in, float2* out, int B, const hcgs_optics* o, bool conjH,
                       cudaStream_t st);

// ---- projection / sort / binning / raster (project.cu, sort.cu, raster.cu) ----
hcgs_status project_and_bin(hcgs_ctx* ctx, hcgs_saved* s, const hcgs_gaussians* g, const float* viewmats,
                            const float* intr, cudaStream_t st);
hcgs_status raster_forward(hcgs_ctx* ctx, hcgs_saved* s, float2* U, float* T_out, int32_t* nc_out,
                           cudaStream_t st);
hcgs_status raster_backward(hcgs_ctx* ctx, hcgs_saved* s, const float2* gU, cudaStream_t st);
hcgs_status project_backward(hcgs_ctx* ctx, hcgs_saved* s, const hcgs_gaussians* g,
                             const hcgs_gaussian_grads* gr, int accumulate, cudaStream_t st);
// Stable LSD radix sort of nseg contiguous segments of (key, value) pairs on
// key bits [0, nbits); returns the buffer index (0 or 1) holding the result.
// keys/vals point at [2][total] ping-pong storage.  Without segoff the
// segments are seglen long; with segoff (device, nseg + 1 offsets; seglen =
// the longest segment) segment s is sorted on key - s keystep.
hcgs_status radix_sort(hcgs_ctx* ctx, hcgs_saved* s, uint32_t* keys, uint32_t* vals, int nseg, size_t seglen,
                       size_t total, const uint32_t* segoff, uint32_t keystep, int nbits, int* which,
                       cudaStream_t st);
// Exclusive scan of n uint32 counts (in place allowed); writes the total to
// out[n] when with_total is set.  Totals must stay below 2^32.
hcgs_status exclusive_scan(hcgs_ctx* ctx, hcgs_saved* s, const uint32_t* in, uint32_t* out, size_t n,
                           cudaStream_t st);

// ---- training pieces (train.cu) ----
hcgs_status adam(hcgs_ctx* ctx, float* p, const float* g, float* m, float* v, int64_t n, int step, float lr,
                 float b1, float b2, float eps, cudaStream_t st);
// Up to OPT_MAX parameter arrays updated by one optimiser launch (the unused
// pointers of an array are NULL: gp and n for Adam).
constexpr int OPT_MAX = 16, OPT_THREADS = 256, OPT_EPB = 4 * OPT_THREADS;
struct OptArrays {
    float* p[OPT_MAX];
    const float* g[OPT_MAX];
    float* m[OPT_MAX];
    float* v[OPT_MAX];
    float* gp[OPT_MAX];
    float* n[OPT_MAX];
    int64_t count[OPT_MAX];
    float lr[OPT_MAX];
    int64_t first[OPT_MAX + 1];  // first block of each array (filled by opt_blocks)
    int k;
};
int64_t opt_blocks(OptArrays& A);
hcgs_status adam_multi(hcgs_ctx* ctx, OptArrays& A, int step, float b1, float b2, float eps, cudaStream_t st);
hcgs_status reduce_sum(hcgs_ctx* ctx, const float* partials, int n, float scale, float* out, cudaStream_t st);
hcgs_status mlp_fwd(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* const* W, const float* const* b,
                    float* y, cudaStream_t st);
hcgs_status mlp_bwd(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* const* W, const float* const* b,
                    const float* gy, float* const* gW, float* const* gb, cudaStream_t st);
hcgs_status mlp_mse(hcgs_ctx* ctx, const float* y, const float* tgt, int N, int K, float* loss, float* gy,
                    cudaStream_t st);
hcgs_status cast_bf16(hcgs_ctx* ctx, const float* src, uint16_t* dst, int64_t n, cudaStream_t st);

// ---- densification (densify.cu) ----
hcgs_status philox(hcgs_ctx* ctx, uint64_t seed, uint32_t stream_id, int64_t n, int normal, void* out,
                   cudaStream_t st);
hcgs_status densify_accumulate(hcgs_ctx* ctx, hcgs_saved* s, float* accum, float* denom, cudaStream_t st);
hcgs_status densify_decide(hcgs_ctx* ctx, const hcgs_gaussians* g, const float* accum, const float* denom,
                           const hcgs_densify_opts& o, int32_t* action, uint32_t* count, cudaStream_t st);
hcgs_status densify_offsets_tail(hcgs_ctx* ctx, const uint32_t* count, uint32_t* offsets, int N, cudaStream_t st);
hcgs_status densify_apply(hcgs_ctx* ctx, const hcgs_gaussians* gi, int C, int L, const int32_t* action,
                          const uint32_t* offset, const float* noise, const hcgs_densify_opts& o,
                          const hcgs_gaussian_grads& go, int n_extra, const float* const* extra_in,
                          float* const* extra_out, const int* extra_width, cudaStream_t st);

// ---- the paper's objective and optimiser (objective.cu) ----
hcgs_status ssim_recon_loss(hcgs_ctx* ctx, float2* V, float* I, const float* Igt, const float* M, int B, int L,
                            int C, int H, int W, float lam, float* dmap, float* partials, int* nblocks_out,
                            float* gI, cudaStream_t st, int plain = 0);
hcgs_status phasor(hcgs_ctx* ctx, const float* phi, float2* P, int64_t n, cudaStream_t st);
hcgs_status split_parts(hcgs_ctx* ctx, const float2* U, float* out, int64_t n, cudaStream_t st);
hcgs_status merge_parts(hcgs_ctx* ctx, const float* g, float2* out, int64_t n, cudaStream_t st);
hcgs_status phase_grad(hcgs_ctx* ctx, const float* phi, const float2* gP, float* gphi, int64_t n, cudaStream_t st);
hcgs_status phase_of(hcgs_ctx* ctx, const float2* P, float* phi, int64_t n, cudaStream_t st);
hcgs_status scale(hcgs_ctx* ctx, const float* x, float s, float* out, int64_t n, cudaStream_t st);
int focal_field_blocks(int64_t n);
hcgs_status focal_field(hcgs_ctx* ctx, float2* V, const float* Igt, float* Iout, int64_t n, float* partials,
                        cudaStream_t st);
hcgs_status adan(hcgs_ctx* ctx, float* p, const float* g, float* gp, float* m, float* v, float* n, int64_t count,
                 int step, float lr, float b1, float b2, float b3, float eps, float wd, cudaStream_t st);
hcgs_status adan_multi(hcgs_ctx* ctx, OptArrays& A, int step, float b1, float b2, float b3, float eps, float wd,
                       cudaStream_t st);

}  // namespace hcgs
