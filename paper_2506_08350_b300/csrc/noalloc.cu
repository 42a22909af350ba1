// Allocation-free inverse propagation: hcgs_asm_propagate_noalloc.
//
// Same computation as the inverse-propagation form of hcgs_asm_propagate
// (sign = -1, reduce_planes = 0): out_l = IDFT(conj(H_{Z_l}) DFT(in)), with the
// same kernels (k_fft_cols, k_rows_spread, k_build_hq).  The difference is
// where the working memory comes from: the column spectrum of `in`, the
// transfer-function table and the two twiddle tables live in one file-scope
// device array of fixed size instead of buffers the library allocates.  It is
// for callers that cannot call cudaMalloc: for example a host application
// whose device memory is entirely managed by its own pool allocator (a
// cudaMalloc from inside a library would fail or fragment that pool), or a
// display loop that allocates everything at start-up and must not stall on
// cudaMalloc/cudaFree, which synchronise the device, in the middle of a frame.
//
// The array occupies NOALLOC_SCRATCH_COMPLEX complex64 values (32 MiB) on
// every GPU that loads this library, until the process exits.  Every call
// shares it and it keeps the last call's contents; each call rewrites all the
// parts it reads before reading them, so nothing needs to start at zero.
// Calls whose kernels overlap on the GPU (two streams, two threads) race on
// the array and must be serialised by the caller.
#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "fft.cuh"

namespace hcgs {
namespace {

constexpr size_t NOALLOC_SCRATCH_COMPLEX = size_t(4) << 20;  // 4 Mi complex64 = 32 MiB
static __device__ __align__(256) float2 g_noalloc_scratch[NOALLOC_SCRATCH_COMPLEX];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
// The array's device address, looked up once per device and CUDA context: a
// context that is destroyed and created again (cudaDeviceReset) reloads the
// module, so the address is keyed on the context's process-unique id (a new
// context never reuses an old id, unlike its handle).
struct NoallocAddr {
    unsigned long long ctx_id;
    float2* p;
};
NoallocAddr g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Id of the calling thread's current context, through the driver entry
// points the runtime hands out (no link-time dependency on libcuda).
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
bool current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) != cudaSuccess ||
            q0 != cudaDriverEntryPointSuccess || !f0)
            return false;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || !f1)
            return false;
        get_current = (CtxGetCurrentFn)f0;
        get_id = (CtxGetIdFn)f1;
    }
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// do the byte ranges [a, a + na) and [b, b + nb) share a byte?
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

// exp(-2 pi i m / n), formed in FP64 and rounded to FP32
__global__ void k_noalloc_twiddles(float2* __restrict__ tw, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(-2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
}

// complex elements rounded up to a 512-byte boundary
size_t round64(size_t n) { return (n + 63) & ~size_t(63); }

bool optics_ok(const hcgs_optics* o) {
    if (!o || o->H < 1 || o->W < 1 || o->C < 1 || o->C > MAX_C || o->L < 1 || o->L > MAX_L) return false;
    if (!(o->pitch_x > 0) || !(o->pitch_y > 0) || !o->wavelength || !o->plane_z) return false;
    if (o->band_limit != 0 && o->band_limit != 1) return false;
    if (o->padding != 0) return false;  // the zero-padded grids need the context's workspace
    for (int c = 0; c < o->C; c++)
        if (!(o->wavelength[c] > 0)) return false;
    return true;
}

FftPlanArg plan_for(int n) {
    FftPlanArg p;
    p.n = n;
    for (int s = 0; s < MAX_STAGES; s++) p.radix[s] = 0;
    factor_radices(n, p.radix, &p.nst);
    return p;
}

}  // namespace
}  // namespace hcgs

using namespace hcgs;

extern "C" hcgs_status hcgs_asm_propagate_noalloc(const float* in, int B, const hcgs_optics* o, float* out,
                                                  void* stream) {
    if (!in || !out || B < 1 || !optics_ok(o)) return HCGS_ERR_INVALID_ARG;
    const int H = o->H, W = o->W, C = o->C, L = o->L;
    const size_t nS = (size_t)B * C * H * W;
    // `out` is written while `in` is still being read: no shared byte
    if (overlaps(in, nS * sizeof(float2), out, nS * L * sizeof(float2))) return HCGS_ERR_INVALID_ARG;
    if (!fft_supported(o->H) || !fft_supported(o->W)) return HCGS_ERR_UNSUPPORTED_SIZE;
    const size_t nH = (size_t)C * L * (H / 2 + 1) * hq_stride(W);
    const size_t need = round64(nS) + round64(nH) + round64(H) + round64(W);
    if (need > NOALLOC_SCRATCH_COMPLEX) return HCGS_ERR_CAPACITY;

    // set-up, once per device and context, with that device current: the
    // device address of the static array (its host-side name is only a
    // stand-in)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return HCGS_ERR_CUDA;
    float2* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        unsigned long long cid = 0;
        // no context current yet on this thread: cudaSetDevice makes the
        // device's primary context current (it allocates nothing)
        if (!current_context_id(&cid) && (cudaSetDevice(dev) != cudaSuccess || !current_context_id(&cid)))
            return HCGS_ERR_CUDA;
        if (!g_noalloc_addr[dev].p || g_noalloc_addr[dev].ctx_id != cid) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HCGS_ERR_CUDA;
            g_noalloc_addr[dev].p = (float2*)p;
            g_noalloc_addr[dev].ctx_id = cid;
        }
        base = g_noalloc_addr[dev].p;
    }
    float2* S1 = base;
    float2* hq = S1 + round64(nS);
    float2* twH = hq + round64(nH);
    float2* twW = twH + round64(H);
    cudaStream_t st = (cudaStream_t)stream;

    k_noalloc_twiddles<<<(H + 255) / 256, 256, 0, st>>>(twH, H);
    k_noalloc_twiddles<<<(W + 255) / 256, 256, 0, st>>>(twW, W);
    if (cudaGetLastError() != cudaSuccess) return HCGS_ERR_CUDA;
    HArgs a{};
    for (int c = 0; c < C; c++) a.lam[c] = o->wavelength[c];
    for (int l = 0; l < L; l++) a.z[l] = o->plane_z[l];
    const FftPlanArg pH = plan_for(H), pW = plan_for(W);
    if (launch_build_hq_raw(hq, H, W, C, L, o->pitch_x, o->pitch_y, a, o->band_limit, st) != cudaSuccess ||
        launch_fft_cols_raw(false, (const float2*)in, S1, B * C, H, W, pH, twH, 1.f, st) != cudaSuccess ||
        launch_rows_spread_conj_raw(S1, (float2*)out, B, L, C, H, W, hq, pW, twW, st) != cudaSuccess ||
        launch_fft_cols_raw(true, (const float2*)out, (float2*)out, B * L * C, H, W, pH, twH,
                            1.f / (float)((size_t)H * W), st) != cudaSuccess)
        return HCGS_ERR_CUDA;
    return HCGS_OK;
}
