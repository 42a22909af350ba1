// C ABI of libhcgs: argument validation, scratch management and the
// orchestration of the render path.  See include/hcgs.h for the contract.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

#include "common.cuh"
#include "project.cuh"

using namespace hcgs;

namespace hcgs {

bool set_err(hcgs_ctx* ctx, hcgs_status s, const std::string& m) {
    if (ctx) ctx->last_error = std::string(hcgs_status_string(s)) + ": " + m;
    return false;
}

hcgs_status cuda_err(hcgs_ctx* ctx, cudaError_t e, const char* what) {
    set_err(ctx, HCGS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return HCGS_ERR_CUDA;
}

#ifdef HCGS_CHECKED
// registry of guarded allocations: base -> (capacity, device); the guard band
// follows the capacity
static std::mutex g_guard_mu;
static std::map<void*, std::pair<size_t, int>> g_guards;
#endif

cudaError_t grow(hcgs_ctx* ctx, DevBuf& b, size_t bytes, size_t* owner_bytes) {
    if (bytes <= b.cap) return cudaSuccess;
    if (b.p) {
        *owner_bytes -= b.cap;
        free_buf(b);
    }
#ifdef HCGS_CHECKED
    const size_t guard = GUARD_BYTES;
#else
    const size_t guard = 0;
#endif
    const size_t want = bytes + bytes / 8;  // slack against small growth steps
    cudaError_t e = cudaMalloc(&b.p, want + guard);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&b.p, bytes + guard);
        if (e != cudaSuccess) return e;
        b.cap = bytes;
    } else {
        b.cap = want;
    }
#ifdef HCGS_CHECKED
    e = cudaMemset((char*)b.p + b.cap, GUARD_FILL, guard);
    if (e != cudaSuccess) return e;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        std::lock_guard<std::mutex> lk(g_guard_mu);
        g_guards[b.p] = std::make_pair(b.cap, dev);
    }
#endif
    *owner_bytes += b.cap;
    (void)ctx;
    return cudaSuccess;
}

void prof_begin(hcgs_ctx* ctx, const char* name, cudaStream_t st) {
    if (!ctx) return;
    // the streams this context's work was enqueued on: releasing a saved
    // state or the context waits for them, not for the whole device
    if (ctx->streams.empty() || ctx->streams.back() != st) {
        bool seen = false;
        for (cudaStream_t x : ctx->streams) seen = seen || x == st;
        if (!seen) ctx->streams.push_back(st);
    }
    if (!ctx->prof.on) return;
    Prof& P = ctx->prof;
    if (P.used + 2 > P.pool.size()) {
        for (int k = 0; k < 64; k++) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            P.pool.push_back(e);
        }
    }
    ProfRec r{name, P.pool[P.used], P.pool[P.used + 1]};
    P.used += 2;
    cudaEventRecord(r.a, st);
    P.recs.push_back(r);
}

void prof_end(hcgs_ctx* ctx, cudaStream_t st) {
    if (!ctx || !ctx->prof.on || ctx->prof.recs.empty()) return;
    cudaEventRecord(ctx->prof.recs.back().b, st);
}

void free_buf(DevBuf& b) {
    if (b.p) {
#ifdef HCGS_CHECKED
        {
            std::lock_guard<std::mutex> lk(g_guard_mu);
            g_guards.erase(b.p);
        }
#endif
        cudaFree(b.p);
    }
    b.p = nullptr;
    b.cap = 0;
}

#ifdef HCGS_CHECKED
// one block per guarded buffer: any byte of its guard band that differs from
// the fill pattern marks the status word; the band is then filled again, so
// that the context stays usable after the report
__global__ void k_check_guards(unsigned char* const* __restrict__ guards, int n, int* __restrict__ status) {
    const int g = blockIdx.x;
    if (g >= n) return;
    unsigned char* p = guards[g];
    bool bad = false;
    for (int i = threadIdx.x; i < (int)GUARD_BYTES; i += blockDim.x) bad |= p[i] != GUARD_FILL;
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicOr(status, STATUS_DEVICE_CHECK);
        for (int i = threadIdx.x; i < (int)GUARD_BYTES; i += blockDim.x) p[i] = GUARD_FILL;
    }
}

// index check of the self-test: idx = n is out of the checked range [0, n),
// while the buffer holds 2 n elements, so the store stays inside the
// allocation even if the check were missing
__global__ void k_selftest_index(float* __restrict__ buf, int n, int idx, int* __restrict__ status) {
    if (threadIdx.x == 0 && HCGS_DCHECK(status, idx < n)) buf[idx] = 1.f;
}
// a store into the guard band of buf (inside its allocation)
__global__ void k_selftest_guard(unsigned char* __restrict__ guard) {
    if (threadIdx.x == 0) guard[GUARD_BYTES / 2] = (unsigned char)(GUARD_FILL ^ 0xFF);
}
#endif

}  // namespace hcgs

// ---------------------------------------------------------------------------
// validation helpers
// ---------------------------------------------------------------------------
#define REQUIRE(ctx, cond, msg)                                   \
    do {                                                          \
        if (!(cond)) {                                            \
            hcgs::set_err(ctx, HCGS_ERR_INVALID_ARG, msg);        \
            return HCGS_ERR_INVALID_ARG;                          \
        }                                                         \
    } while (0)

static hcgs_status check_optics(hcgs_ctx* ctx, const hcgs_optics* o) {
    REQUIRE(ctx, o, "optics is NULL");
    REQUIRE(ctx, o->H >= 1 && o->W >= 1, "H and W must be >= 1");
    REQUIRE(ctx, o->C >= 1 && o->C <= MAX_C, "C must be in [1, 4]");
    REQUIRE(ctx, o->L >= 1 && o->L <= MAX_L, "L must be in [1, 16]");
    REQUIRE(ctx, o->pitch_x > 0 && o->pitch_y > 0, "pitch must be > 0");
    REQUIRE(ctx, o->wavelength && o->plane_z, "wavelength and plane_z must be host arrays");
    for (int c = 0; c < o->C; c++) REQUIRE(ctx, o->wavelength[c] > 0, "wavelengths must be > 0");
    REQUIRE(ctx, o->band_limit == 0 || o->band_limit == 1, "band_limit must be 0 or 1");
    REQUIRE(ctx, o->padding == 0 || o->padding == 1, "padding must be 0 or 1");
    if (!fft_supported(o->H) || !fft_supported(o->W)) {
        set_err(ctx, HCGS_ERR_UNSUPPORTED_SIZE, "H and W must be 2^a 3^b 5^c and <= 4096");
        return HCGS_ERR_UNSUPPORTED_SIZE;
    }
    if (o->padding && (!fft_supported(2 * o->H) || !fft_supported(2 * o->W))) {
        set_err(ctx, HCGS_ERR_UNSUPPORTED_SIZE, "with padding, 2H and 2W must be 2^a 3^b 5^c and <= 4096");
        return HCGS_ERR_UNSUPPORTED_SIZE;
    }
    return HCGS_OK;
}

static hcgs_status check_opts(hcgs_ctx* ctx, const hcgs_raster_opts* r) {
    REQUIRE(ctx, r, "opts is NULL");
    REQUIRE(ctx, r->tile == 16, "tile must be 16");
    REQUIRE(ctx, r->alpha_min >= 0.f && r->alpha_max <= 1.f && r->alpha_min < r->alpha_max,
            "need 0 <= alpha_min < alpha_max <= 1");
    REQUIRE(ctx, r->T_eps >= 0.f, "T_eps must be >= 0");
    REQUIRE(ctx, r->near_z > 0.f, "near_z must be > 0");
    REQUIRE(ctx, r->cov2d_dilation >= 0.f, "cov2d_dilation must be >= 0");
    REQUIRE(ctx, r->ste_tau > 0.f, "ste_tau must be > 0");
    REQUIRE(ctx, r->order == 0 || r->order == 1, "order must be 0 or 1");
    REQUIRE(ctx, r->footprint >= 0 && r->footprint <= 2, "footprint must be 0, 1 or 2");
    REQUIRE(ctx, r->rho_grad == 0 || r->rho_grad == 1, "rho_grad must be 0 or 1");
    return HCGS_OK;
}

static hcgs_status check_gauss(hcgs_ctx* ctx, const hcgs_gaussians* g) {
    REQUIRE(ctx, g, "gaussians is NULL");
    REQUIRE(ctx, g->N >= 0, "N must be >= 0");
    if (g->N > 0)
        REQUIRE(ctx, g->means && g->log_scales && g->quats && g->opacity_logits && g->amplitude && g->phase &&
                         g->plane_logits,
                "a Gaussian parameter array is NULL");
    return HCGS_OK;
}

static cudaStream_t S(void* p) { return (cudaStream_t)p; }

#define TRY(x)                        \
    do {                              \
        hcgs_status st__ = (x);       \
        if (st__ != HCGS_OK) return st__; \
    } while (0)

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" {

const char* hcgs_status_string(hcgs_status s) {
    switch (s) {
        case HCGS_OK: return "HCGS_OK";
        case HCGS_ERR_INVALID_ARG: return "HCGS_ERR_INVALID_ARG";
        case HCGS_ERR_CUDA: return "HCGS_ERR_CUDA";
        case HCGS_ERR_CAPACITY: return "HCGS_ERR_CAPACITY";
        case HCGS_ERR_UNSUPPORTED_SIZE: return "HCGS_ERR_UNSUPPORTED_SIZE";
        case HCGS_ERR_DEVICE_CHECK: return "HCGS_ERR_DEVICE_CHECK";
        case HCGS_ERR_TIMEOUT: return "HCGS_ERR_TIMEOUT";
        case HCGS_ERR_STATE: return "HCGS_ERR_STATE";
    }
    return "HCGS_ERR_UNKNOWN";
}

hcgs_status hcgs_ctx_create(hcgs_ctx** out, int device) {
    if (!out) return HCGS_ERR_INVALID_ARG;
    *out = nullptr;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return HCGS_ERR_CUDA;
    hcgs_ctx* c = new hcgs_ctx();
    c->device = device;
    if (cudaMalloc(&c->d_status, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&c->h_pinned, 64) != cudaSuccess) {
        delete c;
        return HCGS_ERR_CUDA;
    }
    cudaMemset(c->d_status, 0, sizeof(int));
    *out = c;
    return HCGS_OK;
}

static void saved_free(hcgs_saved* s) {
    DevBuf* bufs[] = {&s->w, &s->proj, &s->rectn, &s->dkey, &s->dval, &s->nvalid, &s->rank, &s->sortid, &s->rec,
                      &s->rects, &s->planes, &s->ccount, &s->bcount, &s->ikey, &s->ival, &s->hist, &s->scan,
                      &s->Tfin, &s->last, &s->slist, &s->U, &s->g2d, &s->gU, &s->cam, &s->akey, &s->aval,
                      &s->abcount, &s->drho, &s->segoff};
    for (DevBuf* b : bufs) free_buf(*b);
    s->bytes = 0;
}

// waits for the work this context enqueued (on every stream it used)
static void wait_ctx_streams(hcgs_ctx* ctx) {
    for (cudaStream_t st : ctx->streams)
        if (cudaStreamSynchronize(st) != cudaSuccess) cudaGetLastError();  // a stream destroyed since: nothing to wait for
}

void hcgs_ctx_destroy(hcgs_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    wait_ctx_streams(ctx);
    for (auto& b : ctx->ws) free_buf(b);
    free_buf(ctx->selftest);
    for (auto& kv : ctx->plans) cudaFree(kv.second.tw);
    for (auto& kv : ctx->htab) free_buf(kv.second);
    if (ctx->scratch_saved) {
        saved_free(ctx->scratch_saved);
        delete ctx->scratch_saved;
    }
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_pinned);
    delete ctx;
}

hcgs_status hcgs_profile_enable(hcgs_ctx* ctx, int on) {
    REQUIRE(ctx, ctx, "ctx is NULL");
    ctx->prof.on = on != 0;
    ctx->prof.recs.clear();
    ctx->prof.used = 0;
    return HCGS_OK;
}

hcgs_status hcgs_profile_summary(hcgs_ctx* ctx, int max, int* n_out, const char** names, double* ms,
                                 int64_t* launches) {
    REQUIRE(ctx, ctx && n_out, "NULL argument");
    cudaSetDevice(ctx->device);
    std::vector<std::string> order;
    std::map<std::string, std::pair<double, int64_t>> agg;
    for (const ProfRec& r : ctx->prof.recs) {
        HCGS_CUDA(ctx, cudaEventSynchronize(r.b));
        float t = 0.f;
        HCGS_CUDA(ctx, cudaEventElapsedTime(&t, r.a, r.b));
        auto it = agg.find(r.name);
        if (it == agg.end()) {
            order.push_back(r.name);
            agg[r.name] = {t, 1};
        } else {
            it->second.first += t;
            it->second.second += 1;
        }
    }
    int n = 0;
    for (const std::string& k : order) {
        if (n >= max) break;
        // names point at the string literals the launch sites pass
        for (const ProfRec& r : ctx->prof.recs)
            if (k == r.name) { names[n] = r.name; break; }
        ms[n] = agg[k].first;
        launches[n] = agg[k].second;
        n++;
    }
    *n_out = n;
    ctx->prof.recs.clear();
    ctx->prof.used = 0;
    return HCGS_OK;
}

const char* hcgs_last_error(hcgs_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

size_t hcgs_ctx_bytes(hcgs_ctx* ctx) {
    if (!ctx) return 0;
    size_t b = ctx->bytes;
    if (ctx->scratch_saved) b += ctx->scratch_saved->bytes;
    return b;
}

int hcgs_is_checked_build(void) {
#ifdef HCGS_CHECKED
    return 1;
#else
    return 0;
#endif
}

hcgs_status hcgs_check_status(hcgs_ctx* ctx, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t st = S(stream);
#ifdef HCGS_CHECKED
    {
        std::vector<unsigned char*> gp;
        {
            std::lock_guard<std::mutex> lk(g_guard_mu);
            for (auto& kv : g_guards)
                if (kv.second.second == ctx->device) gp.push_back((unsigned char*)kv.first + kv.second.first);
        }
        if (!gp.empty()) {
            unsigned char** d = nullptr;
            HCGS_CUDA(ctx, cudaMalloc(&d, gp.size() * sizeof(unsigned char*)));
            cudaError_t e = cudaMemcpyAsync(d, gp.data(), gp.size() * sizeof(unsigned char*), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) {
                k_check_guards<<<(unsigned)gp.size(), 128, 0, st>>>(d, (int)gp.size(), ctx->d_status);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            cudaFree(d);
            HCGS_CUDA(ctx, e);
        }
    }
#endif
    HCGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned + 2, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HCGS_CUDA(ctx, cudaStreamSynchronize(st));
    const uint32_t w = ctx->h_pinned[2];
    if (w) {
        HCGS_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
        HCGS_CUDA(ctx, cudaStreamSynchronize(st));
    }
    if (w & STATUS_DEVICE_CHECK) {
        set_err(ctx, HCGS_ERR_DEVICE_CHECK, "a device-side bounds, input or guard-band check failed");
        return HCGS_ERR_DEVICE_CHECK;
    }
    if (w & STATUS_WAIT_TIMEOUT) {
        set_err(ctx, HCGS_ERR_TIMEOUT, "a bounded device wait ran out");
        return HCGS_ERR_TIMEOUT;
    }
    return HCGS_OK;
}

hcgs_status hcgs_selftest_device_check(hcgs_ctx* ctx, int kind, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, kind == 0 || kind == 1, "kind must be 0 (index check) or 1 (guard band)");
#ifdef HCGS_CHECKED
    cudaSetDevice(ctx->device);
    cudaStream_t st = S(stream);
    const int n = 32;
    HCGS_CUDA(ctx, grow(ctx, ctx->selftest, 2 * n * sizeof(float), &ctx->bytes));
    if (kind == 0)
        HCGS_KERNEL(ctx, "k_selftest_index", st, k_selftest_index<<<1, 32, 0, st>>>((float*)ctx->selftest.p, n, n, ctx->d_status));
    else
        HCGS_KERNEL(ctx, "k_selftest_guard", st, k_selftest_guard<<<1, 32, 0, st>>>((unsigned char*)ctx->selftest.p + ctx->selftest.cap));
    return HCGS_OK;
#else
    (void)stream;
    set_err(ctx, HCGS_ERR_STATE, "device checks exist only in the bounds-checked build (libhcgs_checked.so)");
    return HCGS_ERR_STATE;
#endif
}

hcgs_status hcgs_saved_create(hcgs_ctx* ctx, hcgs_saved** out) {
    REQUIRE(ctx, ctx && out, "NULL argument");
    *out = new hcgs_saved();
    return HCGS_OK;
}

hcgs_status hcgs_saved_release(hcgs_ctx* ctx, hcgs_saved* s) {
    if (!s) return HCGS_OK;
    if (ctx) {
        cudaSetDevice(ctx->device);
        wait_ctx_streams(ctx);  // the saved state's buffers are used only by this context's launches
    } else {
        cudaDeviceSynchronize();  // no context to ask which streams used it
    }
    saved_free(s);
    delete s;
    return HCGS_OK;
}

// ---------------------------------------------------------------------------
// steps
// ---------------------------------------------------------------------------
hcgs_status hcgs_project(hcgs_ctx* ctx, const hcgs_gaussians* g, int V, const float* viewmats,
                         const float* intrinsics, const hcgs_optics* optics, const hcgs_raster_opts* opts,
                         hcgs_saved* s, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    TRY(check_gauss(ctx, g));
    TRY(check_optics(ctx, optics));
    TRY(check_opts(ctx, opts));
    REQUIRE(ctx, s, "saved is NULL");
    REQUIRE(ctx, V >= 1, "V must be >= 1");
    REQUIRE(ctx, viewmats && intrinsics, "viewmats / intrinsics is NULL");
    cudaSetDevice(ctx->device);
    s->V = V;
    s->N = g->N;
    s->C = optics->C;
    s->L = optics->L;
    s->H = optics->H;
    s->W = optics->W;
    s->tilesX = (optics->W + TILE - 1) / TILE;
    s->tilesY = (optics->H + TILE - 1) / TILE;
    s->ctX = (s->tilesX + COARSE - 1) / COARSE;
    s->ctY = (s->tilesY + COARSE - 1) / COARSE;
    s->opts = *opts;
    s->optics = *optics;
    s->lam.assign(optics->wavelength, optics->wavelength + optics->C);
    s->z.assign(optics->plane_z, optics->plane_z + optics->L);
    s->optics.wavelength = s->lam.data();
    s->optics.plane_z = s->z.data();
    s->valid = 0;
    s->rastered = 0;
    s->have_g2d = 0;
    if ((uint64_t)V * optics->L * s->ctX * s->ctY >= (1ull << 32)) {
        set_err(ctx, HCGS_ERR_CAPACITY, "too many buckets");
        return HCGS_ERR_CAPACITY;
    }
    if (g->N == 0) {
        // empty scene: every bucket is empty
        const size_t NB = (size_t)V * s->L * s->ctX * s->ctY;
        HCGS_CUDA(ctx, grow(ctx, s->bcount, (NB + 1) * sizeof(uint32_t), &s->bytes));
        HCGS_CUDA(ctx, grow(ctx, s->ival, 8, &s->bytes));
        HCGS_CUDA(ctx, cudaMemsetAsync(s->bcount.p, 0, (NB + 1) * sizeof(uint32_t), S(stream)));
        s->list = (const uint32_t*)s->ival.p;
        s->M = 0;
    } else {
        TRY(project_and_bin(ctx, s, g, viewmats, intrinsics, S(stream)));
    }
    s->valid = 1;
    return HCGS_OK;
}

hcgs_status hcgs_rasterize_planes(hcgs_ctx* ctx, hcgs_saved* s, float* U, float* T_final, int32_t* n_contrib,
                                  void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, s && U, "NULL argument");
    if (!s->valid) {
        set_err(ctx, HCGS_ERR_STATE, "hcgs_project has not run on this saved state");
        return HCGS_ERR_STATE;
    }
    cudaSetDevice(ctx->device);
    TRY(raster_forward(ctx, s, (float2*)U, T_final, n_contrib, S(stream)));
    s->rastered = 1;
    return HCGS_OK;
}

hcgs_status hcgs_asm_propagate(hcgs_ctx* ctx, const float* in, int B, const hcgs_optics* o, int sign,
                               int reduce_planes, float* out, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    TRY(check_optics(ctx, o));
    REQUIRE(ctx, in && out && in != out, "in/out must be distinct non-NULL device arrays");
    REQUIRE(ctx, B >= 1, "B must be >= 1");
    cudaSetDevice(ctx->device);
    if (sign == 1 && reduce_planes == 1) return asm_sum(ctx, (const float2*)in, (float2*)out, B, o, false, S(stream));
    if (sign == -1 && reduce_planes == 0)
        return asm_spread(ctx, (const float2*)in, (float2*)out, B, o, true, S(stream));
    set_err(ctx, HCGS_ERR_INVALID_ARG, "supported forms: (sign=+1, reduce_planes=1), (sign=-1, reduce_planes=0)");
    return HCGS_ERR_INVALID_ARG;
}

hcgs_status hcgs_asm_propagate_backward(hcgs_ctx* ctx, const float* g_out, int B, const hcgs_optics* o, int sign,
                                        int reduce_planes, float* g_in, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    TRY(check_optics(ctx, o));
    REQUIRE(ctx, g_out && g_in && g_out != g_in, "g_out/g_in must be distinct non-NULL device arrays");
    REQUIRE(ctx, B >= 1, "B must be >= 1");
    cudaSetDevice(ctx->device);
    // (F^-1 D F)^H = F^-1 conj(D) F, and conj(H_Z) = H_{-Z} inside the band
    if (sign == 1 && reduce_planes == 1)
        return asm_spread(ctx, (const float2*)g_out, (float2*)g_in, B, o, true, S(stream));
    if (sign == -1 && reduce_planes == 0)
        return asm_sum(ctx, (const float2*)g_out, (float2*)g_in, B, o, false, S(stream));
    set_err(ctx, HCGS_ERR_INVALID_ARG, "supported forms: (sign=+1, reduce_planes=1), (sign=-1, reduce_planes=0)");
    return HCGS_ERR_INVALID_ARG;
}

hcgs_status hcgs_render_view(hcgs_ctx* ctx, const hcgs_gaussians* g, int V, const float* viewmats,
                             const float* intrinsics, const hcgs_optics* o, const hcgs_raster_opts* opts,
                             float* hologram, float* planes, hcgs_saved* saved, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, hologram, "hologram is NULL");
    hcgs_saved* s = saved;
    if (!s) {
        if (!ctx->scratch_saved) ctx->scratch_saved = new hcgs_saved();
        s = ctx->scratch_saved;
    }
    TRY(hcgs_project(ctx, g, V, viewmats, intrinsics, o, opts, s, stream));
    float2* U = (float2*)planes;
    if (!U) {
        const size_t F = (size_t)V * o->L * o->C * o->H * o->W;
        HCGS_CUDA(ctx, grow(ctx, s->U, F * sizeof(float2), &s->bytes));
        U = (float2*)s->U.p;
    }
    TRY(raster_forward(ctx, s, U, nullptr, nullptr, S(stream)));
    s->rastered = 1;
    return asm_sum(ctx, U, (float2*)hologram, V, &s->optics, false, S(stream));
}

hcgs_status hcgs_rasterize_planes_backward(hcgs_ctx* ctx, hcgs_saved* s, const float* gU, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, s && gU, "NULL argument");
    if (!s->valid || !s->rastered) {
        set_err(ctx, HCGS_ERR_STATE, "the forward rasterization has not run on this saved state");
        return HCGS_ERR_STATE;
    }
    cudaSetDevice(ctx->device);
    TRY(raster_backward(ctx, s, (const float2*)gU, S(stream)));
    s->have_g2d = 1;
    return HCGS_OK;
}

static hcgs_status check_grads(hcgs_ctx* ctx, const hcgs_gaussian_grads* gr) {
    REQUIRE(ctx, gr, "grads is NULL");
    REQUIRE(ctx, gr->means && gr->log_scales && gr->quats && gr->opacity_logits && gr->amplitude && gr->phase &&
                     gr->plane_logits,
            "a gradient array is NULL");
    return HCGS_OK;
}

hcgs_status hcgs_project_backward(hcgs_ctx* ctx, hcgs_saved* s, const hcgs_gaussians* g,
                                  const hcgs_gaussian_grads* gr, int accumulate, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, s, "saved is NULL");
    TRY(check_gauss(ctx, g));
    if (!s->have_g2d || g->N != s->N) {
        set_err(ctx, HCGS_ERR_STATE, "needs hcgs_rasterize_planes_backward on the same Gaussians first");
        return HCGS_ERR_STATE;
    }
    if (g->N == 0) return HCGS_OK;
    TRY(check_grads(ctx, gr));
    cudaSetDevice(ctx->device);
    return project_backward(ctx, s, g, gr, accumulate, S(stream));
}

hcgs_status hcgs_render_view_backward(hcgs_ctx* ctx, hcgs_saved* saved, const hcgs_gaussians* g,
                                      const float* g_hologram, const hcgs_gaussian_grads* gr, int accumulate,
                                      void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    hcgs_saved* s = saved ? saved : ctx->scratch_saved;
    REQUIRE(ctx, s && g_hologram, "NULL argument");
    if (!s->valid || !s->rastered) {
        set_err(ctx, HCGS_ERR_STATE, "hcgs_render_view has not run on this saved state");
        return HCGS_ERR_STATE;
    }
    TRY(check_gauss(ctx, g));
    REQUIRE(ctx, g->N == s->N, "N differs from the forward call");
    cudaSetDevice(ctx->device);
    const size_t F = (size_t)s->V * s->L * s->C * s->H * s->W;
    HCGS_CUDA(ctx, grow(ctx, s->gU, F * sizeof(float2), &s->bytes));
    TRY(asm_spread(ctx, (const float2*)g_hologram, (float2*)s->gU.p, s->V, &s->optics, true, S(stream)));
    TRY(raster_backward(ctx, s, (const float2*)s->gU.p, S(stream)));
    s->have_g2d = 1;
    if (g->N == 0) return HCGS_OK;
    TRY(check_grads(ctx, gr));
    return project_backward(ctx, s, g, gr, accumulate, S(stream));
}

hcgs_status hcgs_focal_stack_loss(hcgs_ctx* ctx, const float* hologram, const float* I_gt, int B,
                                  const hcgs_optics* o, float* loss, float* g_hologram, float* I_out,
                                  void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    TRY(check_optics(ctx, o));
    REQUIRE(ctx, hologram && I_gt && loss, "NULL argument");
    REQUIRE(ctx, B >= 1, "B must be >= 1");
    cudaSetDevice(ctx->device);
    if (o->padding) {
        // zero-padded propagation: V by the general route, then the loss on V
        const size_t nF = (size_t)B * o->L * o->C * o->H * o->W;
        cudaStream_t st = S(stream);
        HCGS_CUDA(ctx, grow(ctx, ctx->ws[2], nF * sizeof(float2), &ctx->bytes));
        const int nb = focal_field_blocks((int64_t)nF);
        HCGS_CUDA(ctx, grow(ctx, ctx->ws[3], (size_t)nb * sizeof(float), &ctx->bytes));
        float2* V = (float2*)ctx->ws[2].p;
        TRY(asm_spread(ctx, (const float2*)hologram, V, B, o, true, st));
        TRY(focal_field(ctx, V, I_gt, I_out, (int64_t)nF, (float*)ctx->ws[3].p, st));
        TRY(reduce_sum(ctx, (const float*)ctx->ws[3].p, nb, (float)(1.0 / (double)nF), loss, st));
        if (g_hologram) TRY(asm_sum(ctx, V, (float2*)g_hologram, B, o, false, st));
        return HCGS_OK;
    }
    const float2* hq;
    TRY(get_htab(ctx, o, &hq));
    const size_t planeN = (size_t)o->H * o->W;
    const size_t nP = (size_t)B * o->C * planeN, nF = (size_t)B * o->L * o->C * planeN;
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[1], nP * sizeof(float2), &ctx->bytes));
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[2], nF * sizeof(float2), &ctx->bytes));
    float2* S1 = (float2*)ctx->ws[1].p;
    float2* S2 = (float2*)ctx->ws[2].p;
    cudaStream_t st = S(stream);
    const float inv_count = (float)(1.0 / (double)nF);
    int nblocks = 0;
    TRY(cols_focal_loss(ctx, nullptr, nullptr, nullptr, nullptr, B * o->L * o->C, o->H, o->W, inv_count, 0.f,
                        &nblocks, st));
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[3], (size_t)nblocks * sizeof(float), &ctx->bytes));
    TRY(fft_cols(ctx, (const float2*)hologram, S1, B * o->C, o->H, o->W, false, 1.f, st));
    TRY(rows_spread(ctx, S1, S2, B, o->L, o->C, o->H, o->W, hq, true, st));
    TRY(cols_focal_loss(ctx, S2, I_gt, I_out, (float*)ctx->ws[3].p, B * o->L * o->C, o->H, o->W, inv_count,
                        1.f / (float)planeN, &nblocks, st));
    TRY(reduce_sum(ctx, (const float*)ctx->ws[3].p, nblocks, inv_count, loss, st));
    if (g_hologram) {
        TRY(rows_sum(ctx, S2, (float2*)g_hologram, B, o->L, o->C, o->H, o->W, hq, false, st));
        TRY(fft_cols(ctx, (float2*)g_hologram, (float2*)g_hologram, B * o->C, o->H, o->W, true,
                     1.f / (float)planeN, st));
    }
    return HCGS_OK;
}

// Workspace of the SSIM passes: dmap (3 n floats), then the intensities (n)
// when the caller gives no I_out; ws[3] takes the block partials.
static hcgs_status paper_loss_ws(hcgs_ctx* ctx, size_t n, bool need_I, int nblocks, float** dmap, float** I) {
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[4], (need_I ? 4 : 3) * n * sizeof(float), &ctx->bytes));
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[3], (size_t)nblocks * sizeof(float), &ctx->bytes));
    *dmap = (float*)ctx->ws[4].p;
    *I = need_I ? *dmap + 3 * n : nullptr;
    return HCGS_OK;
}

hcgs_status hcgs_paper_loss(hcgs_ctx* ctx, const float* hologram, const float* I_gt, const float* masks, int B,
                            const hcgs_optics* o, float lambda_ssim, float* loss, float* g_hologram, float* I_out,
                            void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    TRY(check_optics(ctx, o));
    REQUIRE(ctx, hologram && I_gt && loss, "NULL argument");
    REQUIRE(ctx, B >= 1, "B must be >= 1");
    REQUIRE(ctx, lambda_ssim >= 0.f && std::isfinite(lambda_ssim), "lambda_ssim must be finite and >= 0");
    cudaSetDevice(ctx->device);
    const float2* hq = nullptr;
    if (!o->padding) TRY(get_htab(ctx, o, &hq));
    const size_t planeN = (size_t)o->H * o->W;
    const size_t nP = (size_t)B * o->C * planeN, nF = (size_t)B * o->L * o->C * planeN;
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[1], nP * sizeof(float2), &ctx->bytes));
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[2], nF * sizeof(float2), &ctx->bytes));
    float2* S1 = (float2*)ctx->ws[1].p;
    float2* V = (float2*)ctx->ws[2].p;
    cudaStream_t st = S(stream);
    int nblocks = 0;
    TRY(ssim_recon_loss(ctx, nullptr, nullptr, nullptr, nullptr, B, o->L, o->C, o->H, o->W, 0.f, nullptr, nullptr,
                        &nblocks, nullptr, st));
    float *dmap, *Iws;
    TRY(paper_loss_ws(ctx, nF, I_out == nullptr, nblocks, &dmap, &Iws));
    float* I = I_out ? I_out : Iws;
    if (o->padding) {
        TRY(asm_spread(ctx, (const float2*)hologram, V, B, o, true, st));
    } else {
        // V_l = ASM(P, -z_l) for every plane: column DFT, row DFT x conj(H), inverse rows, inverse columns
        TRY(fft_cols(ctx, (const float2*)hologram, S1, B * o->C, o->H, o->W, false, 1.f, st));
        TRY(rows_spread(ctx, S1, V, B, o->L, o->C, o->H, o->W, hq, true, st));
        TRY(fft_cols(ctx, V, V, B * o->L * o->C, o->H, o->W, true, 1.f / (float)planeN, st));
    }
    // I = |V|^2, loss partials, and dL/dV = 2 (dL/dI) V in place over V
    TRY(ssim_recon_loss(ctx, V, I, I_gt, masks, B, o->L, o->C, o->H, o->W, lambda_ssim, dmap,
                        (float*)ctx->ws[3].p, &nblocks, nullptr, st));
    TRY(reduce_sum(ctx, (const float*)ctx->ws[3].p, nblocks, (float)(1.0 / (double)nF), loss, st));
    if (g_hologram && o->padding) {
        TRY(asm_sum(ctx, V, (float2*)g_hologram, B, o, false, st));
    } else if (g_hologram) {
        // dL/dP = sum over planes of the adjoint propagation of dL/dV
        TRY(fft_cols(ctx, V, V, B * o->L * o->C, o->H, o->W, false, 1.f, st));
        TRY(rows_sum(ctx, V, (float2*)g_hologram, B, o->L, o->C, o->H, o->W, hq, false, st));
        TRY(fft_cols(ctx, (float2*)g_hologram, (float2*)g_hologram, B * o->C, o->H, o->W, true,
                     1.f / (float)planeN, st));
    }
    return HCGS_OK;
}

hcgs_status hcgs_paper_loss_intensities(hcgs_ctx* ctx, const float* I, const float* I_gt, const float* masks, int B,
                                        int L, int C, int H, int W, float lambda_ssim, float* loss, float* g_I,
                                        void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, I && I_gt && loss && g_I, "NULL argument");
    REQUIRE(ctx, B >= 1 && L >= 1 && C >= 1 && H >= 1 && W >= 1, "sizes must be >= 1");
    REQUIRE(ctx, (double)B * L * C * H * W < 2147483648.0 / 4, "too many values");
    REQUIRE(ctx, lambda_ssim >= 0.f && std::isfinite(lambda_ssim), "lambda_ssim must be finite and >= 0");
    cudaSetDevice(ctx->device);
    cudaStream_t st = S(stream);
    const size_t n = (size_t)B * L * C * H * W;
    int nblocks = 0;
    TRY(ssim_recon_loss(ctx, nullptr, nullptr, nullptr, nullptr, B, L, C, H, W, 0.f, nullptr, nullptr, &nblocks,
                        nullptr, st));
    float *dmap, *unused;
    TRY(paper_loss_ws(ctx, n, false, nblocks, &dmap, &unused));
    TRY(ssim_recon_loss(ctx, nullptr, (float*)I, I_gt, masks, B, L, C, H, W, lambda_ssim, dmap,
                        (float*)ctx->ws[3].p, &nblocks, g_I, st));
    return reduce_sum(ctx, (const float*)ctx->ws[3].p, nblocks, (float)(1.0 / (double)n), loss, st);
}

hcgs_status hcgs_adan_step(hcgs_ctx* ctx, float* p, const float* g, float* g_prev, float* m, float* v, float* n,
                           int64_t count, int step, float lr, float beta1, float beta2, float beta3, float eps,
                           float weight_decay, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, count >= 0, "count must be >= 0");
    if (count == 0) return HCGS_OK;
    REQUIRE(ctx, p && g && g_prev && m && v && n, "NULL argument");
    REQUIRE(ctx, step >= 1, "step counts from 1");
    REQUIRE(ctx, beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && beta3 >= 0.f && beta3 < 1.f &&
                     eps >= 0.f && weight_decay >= 0.f,
            "bad Adan constants");
    cudaSetDevice(ctx->device);
    return adan(ctx, p, g, g_prev, m, v, n, count, step, lr, beta1, beta2, beta3, eps, weight_decay, S(stream));
}

static hcgs_status check_densify_opts(hcgs_ctx* ctx, const hcgs_densify_opts* o) {
    REQUIRE(ctx, o, "densify opts is NULL");
    REQUIRE(ctx, std::isfinite(o->grad_threshold) && std::isfinite(o->split_scale) &&
                     std::isfinite(o->prune_opacity) && std::isfinite(o->prune_scale) &&
                     std::isfinite(o->phase_noise) && o->split_shrink > 1.f && std::isfinite(o->split_shrink),
            "densify opts must be finite, split_shrink > 1");
    return HCGS_OK;
}

hcgs_status hcgs_densify_accumulate(hcgs_ctx* ctx, hcgs_saved* s, float* accum, float* denom, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, s && accum && denom, "NULL argument");
    if (!s->have_g2d) {
        set_err(ctx, HCGS_ERR_STATE, "needs the backward pass of the compositor on this saved state first");
        return HCGS_ERR_STATE;
    }
    cudaSetDevice(ctx->device);
    return densify_accumulate(ctx, s, accum, denom, S(stream));
}

hcgs_status hcgs_densify_plan(hcgs_ctx* ctx, const hcgs_gaussians* g, const float* accum, const float* denom,
                              const hcgs_densify_opts* opts, int32_t* action, uint32_t* offsets, int64_t* n_out,
                              void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    TRY(check_gauss(ctx, g));
    TRY(check_densify_opts(ctx, opts));
    REQUIRE(ctx, offsets && n_out, "NULL argument");
    REQUIRE(ctx, g->N < (1 << 30), "N must be < 2^30 (the output count is uint32)");
    if (g->N > 0) REQUIRE(ctx, accum && denom && action, "NULL argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = S(stream);
    if (g->N > 0) {
        HCGS_CUDA(ctx, grow(ctx, ctx->ws[5], (size_t)g->N * sizeof(uint32_t), &ctx->bytes));
        uint32_t* count = (uint32_t*)ctx->ws[5].p;
        TRY(densify_decide(ctx, g, accum, denom, *opts, action, count, st));
        if (!ctx->scratch_saved) ctx->scratch_saved = new hcgs_saved();
        TRY(exclusive_scan(ctx, ctx->scratch_saved, count, offsets, (size_t)g->N, st));
        TRY(densify_offsets_tail(ctx, count, offsets, g->N, st));
    } else {
        HCGS_CUDA(ctx, cudaMemsetAsync(offsets, 0, sizeof(uint32_t), st));
    }
    HCGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_pinned, offsets + g->N, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    HCGS_CUDA(ctx, cudaStreamSynchronize(st));
    *n_out = (int64_t)ctx->h_pinned[0];
    return HCGS_OK;
}

hcgs_status hcgs_densify_apply(hcgs_ctx* ctx, const hcgs_gaussians* g_in, int C, int L, const int32_t* action,
                               const uint32_t* offsets, const float* noise, const hcgs_densify_opts* opts,
                               const hcgs_gaussian_grads* g_out, int n_extra, const float* const* extra_in,
                               float* const* extra_out, const int* extra_width, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    TRY(check_gauss(ctx, g_in));
    TRY(check_densify_opts(ctx, opts));
    REQUIRE(ctx, C >= 1 && C <= MAX_C && L >= 1 && L <= MAX_L, "bad C or L");
    REQUIRE(ctx, n_extra >= 0 && n_extra <= HCGS_DENSIFY_MAX_EXTRA, "n_extra out of range");
    if (g_in->N == 0) return HCGS_OK;
    REQUIRE(ctx, action && offsets && noise && g_out, "NULL argument");
    TRY(check_grads(ctx, g_out));
    REQUIRE(ctx, g_out->means != g_in->means && g_out->phase != g_in->phase, "g_out must not alias g_in");
    if (n_extra > 0) REQUIRE(ctx, extra_in && extra_out && extra_width, "NULL extra array list");
    for (int e = 0; e < n_extra; e++) {
        REQUIRE(ctx, extra_in[e] && extra_out[e] && extra_in[e] != extra_out[e], "bad extra array");
        REQUIRE(ctx, extra_width[e] >= 1 && extra_width[e] <= 64, "extra width must be 1..64");
    }
    cudaSetDevice(ctx->device);
    return densify_apply(ctx, g_in, C, L, action, offsets, noise, *opts, *g_out, n_extra, extra_in, extra_out,
                         extra_width, S(stream));
}

hcgs_status hcgs_philox(hcgs_ctx* ctx, uint64_t seed, uint32_t stream_id, int64_t n, int kind, void* out,
                        void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, n >= 0 && n < ((int64_t)1 << 34), "n out of range");
    REQUIRE(ctx, kind >= 0 && kind <= 2, "kind must be 0 (words), 1 (normals) or 2 (uniforms)");
    if (n == 0) return HCGS_OK;
    REQUIRE(ctx, out, "NULL argument");
    cudaSetDevice(ctx->device);
    return philox(ctx, seed, stream_id, n, kind, out, S(stream));
}

hcgs_status hcgs_phase_only_loss(hcgs_ctx* ctx, const float* U_target, const float* phase, int B,
                                 const hcgs_optics* o, float lambda_ssim, float* loss, float* g_phase, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    TRY(check_optics(ctx, o));
    REQUIRE(ctx, U_target && phase && loss, "NULL argument");
    REQUIRE(ctx, B >= 1, "B must be >= 1");
    REQUIRE(ctx, lambda_ssim >= 0.f && std::isfinite(lambda_ssim), "lambda_ssim must be finite and >= 0");
    cudaSetDevice(ctx->device);
    cudaStream_t st = S(stream);
    const int64_t nP = (int64_t)B * o->C * o->H * o->W, nF = nP * o->L;
    // e^{j phi} and its fields on the planes
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[8], (size_t)nP * sizeof(float2), &ctx->bytes));
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[2], (size_t)nF * sizeof(float2), &ctx->bytes));
    HCGS_CUDA(ctx, grow(ctx, ctx->ws[9], (size_t)6 * nF * sizeof(float), &ctx->bytes));
    float2* Pphi = (float2*)ctx->ws[8].p;
    float2* Uphi = (float2*)ctx->ws[2].p;
    float* X = (float*)ctx->ws[9].p;  // parts of U_phi [2][nF]
    float* Y = X + 2 * nF;             // parts of the target
    float* gX = Y + 2 * nF;
    TRY(phasor(ctx, phase, Pphi, nP, st));
    TRY(asm_spread(ctx, Pphi, Uphi, B, o, true, st));
    TRY(split_parts(ctx, Uphi, X, nF, st));
    TRY(split_parts(ctx, (const float2*)U_target, Y, nF, st));
    // the parts are 2 B L C real images: squared error (weight 1) + SSIM
    int nblocks = 0;
    TRY(ssim_recon_loss(ctx, nullptr, nullptr, nullptr, nullptr, 2 * B, o->L, o->C, o->H, o->W, 0.f, nullptr,
                        nullptr, &nblocks, nullptr, st, 1));
    float *dmap, *unused;
    TRY(paper_loss_ws(ctx, (size_t)(2 * nF), false, nblocks, &dmap, &unused));
    TRY(ssim_recon_loss(ctx, nullptr, X, Y, nullptr, 2 * B, o->L, o->C, o->H, o->W, lambda_ssim, dmap,
                        (float*)ctx->ws[3].p, &nblocks, gX, st, 1));
    TRY(reduce_sum(ctx, (const float*)ctx->ws[3].p, nblocks, (float)(1.0 / (double)(2 * nF)), loss, st));
    if (g_phase) {
        TRY(merge_parts(ctx, gX, Uphi, nF, st));
        TRY(asm_sum(ctx, Uphi, Pphi, B, o, false, st));
        TRY(phase_grad(ctx, phase, Pphi, g_phase, nP, st));
    }
    return HCGS_OK;
}

hcgs_status hcgs_scale(hcgs_ctx* ctx, const float* x, int64_t n, float s, float* out, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, n >= 0, "n must be >= 0");
    if (n == 0) return HCGS_OK;
    REQUIRE(ctx, x && out, "NULL argument");
    cudaSetDevice(ctx->device);
    return scale(ctx, x, s, out, n, S(stream));
}

hcgs_status hcgs_phase_hologram(hcgs_ctx* ctx, const float* phase, int64_t n, float* hologram, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, n >= 0, "n must be >= 0");
    if (n == 0) return HCGS_OK;
    REQUIRE(ctx, hologram && phase, "NULL argument");
    cudaSetDevice(ctx->device);
    return phasor(ctx, phase, (float2*)hologram, n, S(stream));
}

hcgs_status hcgs_hologram_phase(hcgs_ctx* ctx, const float* hologram, int64_t n, float* phase, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, n >= 0, "n must be >= 0");
    if (n == 0) return HCGS_OK;
    REQUIRE(ctx, hologram && phase, "NULL argument");
    cudaSetDevice(ctx->device);
    return phase_of(ctx, (const float2*)hologram, phase, n, S(stream));
}

hcgs_status hcgs_adam_step(hcgs_ctx* ctx, float* p, const float* g, float* m, float* v, int64_t n, int step,
                           float lr, float beta1, float beta2, float eps, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, n >= 0, "n must be >= 0");
    if (n == 0) return HCGS_OK;
    REQUIRE(ctx, p && g && m && v, "NULL argument");
    REQUIRE(ctx, step >= 1, "step counts from 1");
    REQUIRE(ctx, beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f, "bad Adam constants");
    cudaSetDevice(ctx->device);
    return adam(ctx, p, g, m, v, n, step, lr, beta1, beta2, eps, S(stream));
}

hcgs_status hcgs_adam_step_multi(hcgs_ctx* ctx, int k, float* const* p, const float* const* g, float* const* m,
                                 float* const* v, const int64_t* count, const float* lr, int step, float beta1,
                                 float beta2, float eps, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, k >= 0 && k <= OPT_MAX, "k must be in [0, 16]");
    if (k == 0) return HCGS_OK;
    REQUIRE(ctx, p && g && m && v && count && lr, "NULL argument");
    REQUIRE(ctx, step >= 1, "step counts from 1");
    REQUIRE(ctx, beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f, "bad Adam constants");
    OptArrays A{};
    A.k = k;
    for (int a = 0; a < k; a++) {
        REQUIRE(ctx, count[a] >= 0, "count must be >= 0");
        REQUIRE(ctx, count[a] == 0 || (p[a] && g[a] && m[a] && v[a]), "NULL array");
        A.p[a] = p[a]; A.g[a] = g[a]; A.m[a] = m[a]; A.v[a] = v[a];
        A.count[a] = count[a];
        A.lr[a] = lr[a];
    }
    cudaSetDevice(ctx->device);
    return adam_multi(ctx, A, step, beta1, beta2, eps, S(stream));
}

hcgs_status hcgs_adan_step_multi(hcgs_ctx* ctx, int k, float* const* p, const float* const* g, float* const* g_prev,
                                 float* const* m, float* const* v, float* const* n, const int64_t* count,
                                 const float* lr, int step, float beta1, float beta2, float beta3, float eps,
                                 float weight_decay, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, k >= 0 && k <= OPT_MAX, "k must be in [0, 16]");
    if (k == 0) return HCGS_OK;
    REQUIRE(ctx, p && g && g_prev && m && v && n && count && lr, "NULL argument");
    REQUIRE(ctx, step >= 1, "step counts from 1");
    REQUIRE(ctx, beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && beta3 >= 0.f && beta3 < 1.f &&
                     eps >= 0.f && weight_decay >= 0.f,
            "bad Adan constants");
    OptArrays A{};
    A.k = k;
    for (int a = 0; a < k; a++) {
        REQUIRE(ctx, count[a] >= 0, "count must be >= 0");
        REQUIRE(ctx, count[a] == 0 || (p[a] && g[a] && g_prev[a] && m[a] && v[a] && n[a]), "NULL array");
        A.p[a] = p[a]; A.g[a] = g[a]; A.gp[a] = g_prev[a]; A.m[a] = m[a]; A.v[a] = v[a]; A.n[a] = n[a];
        A.count[a] = count[a];
        A.lr[a] = lr[a];
    }
    cudaSetDevice(ctx->device);
    return adan_multi(ctx, A, step, beta1, beta2, beta3, eps, weight_decay, S(stream));
}

hcgs_status hcgs_mlp_forward(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* W1, const uint16_t* W2,
                             const uint16_t* W3, const uint16_t* W4, const float* b1, const float* b2,
                             const float* b3, const float* b4, float* y, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, N >= 0 && N <= (1 << 30), "N must be in [0, 2^30]");
    if (N == 0) return HCGS_OK;
    REQUIRE(ctx, x && W1 && W2 && W3 && W4 && b1 && b2 && b3 && b4 && y, "NULL argument");
    cudaSetDevice(ctx->device);
    const uint16_t* W[4] = {W1, W2, W3, W4};
    const float* b[4] = {b1, b2, b3, b4};
    return mlp_fwd(ctx, x, N, W, b, y, S(stream));
}

hcgs_status hcgs_mlp_backward(hcgs_ctx* ctx, const uint16_t* x, int N, const uint16_t* W1, const uint16_t* W2,
                              const uint16_t* W3, const uint16_t* W4, const float* b1, const float* b2,
                              const float* b3, const float* b4, const float* gy, float* gW1, float* gW2,
                              float* gW3, float* gW4, float* gb1, float* gb2, float* gb3, float* gb4,
                              void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, N >= 0 && N <= (1 << 30), "N must be in [0, 2^30]");
    REQUIRE(ctx, x && W1 && W2 && W3 && W4 && b1 && b2 && b3 && b4 && gy, "NULL argument");
    REQUIRE(ctx, gW1 && gW2 && gW3 && gW4 && gb1 && gb2 && gb3 && gb4, "NULL gradient argument");
    cudaSetDevice(ctx->device);
    const uint16_t* W[4] = {W1, W2, W3, W4};
    const float* b[4] = {b1, b2, b3, b4};
    float* gW[4] = {gW1, gW2, gW3, gW4};
    float* gb[4] = {gb1, gb2, gb3, gb4};
    return mlp_bwd(ctx, x, N, W, b, gy, gW, gb, S(stream));
}

hcgs_status hcgs_mlp_mse_loss(hcgs_ctx* ctx, const float* y, const float* target, int N, int K, float* loss,
                              float* gy, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, N >= 1 && K >= 1 && K <= 16, "need N >= 1 and 1 <= K <= 16");
    REQUIRE(ctx, y && target && loss && gy, "NULL argument");
    cudaSetDevice(ctx->device);
    return mlp_mse(ctx, y, target, N, K, loss, gy, S(stream));
}

hcgs_status hcgs_cast_bf16(hcgs_ctx* ctx, const float* src, uint16_t* dst, int64_t n, void* stream) {
    if (!ctx) return HCGS_ERR_INVALID_ARG;
    REQUIRE(ctx, n >= 0, "n must be >= 0");
    if (n == 0) return HCGS_OK;
    REQUIRE(ctx, src && dst, "NULL argument");
    cudaSetDevice(ctx->device);
    return cast_bf16(ctx, src, dst, n, S(stream));
}

}  // extern "C"
