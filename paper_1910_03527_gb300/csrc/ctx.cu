// Context, error reporting, device workspace and the string tables (a3).
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

namespace mbe {

static thread_local char g_err[512] = "no error";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return MBE_ECUDA;
}

int workspace(mbe_ctx *ctx, size_t bytes, void **out)
{
    if (bytes > ctx->ws_size) {
        size_t want = bytes + bytes / 4 + (1 << 20);
        if (ctx->ws) MBE_CU(cudaFreeAsync(ctx->ws, ctx->stream));
        ctx->ws = nullptr;
        ctx->ws_size = 0;
        cudaError_t e = cudaMallocAsync(&ctx->ws, want, ctx->stream);
        if (e != cudaSuccess) {
            set_error("workspace allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? MBE_ENOMEM : MBE_ECUDA;
        }
        ctx->ws_size = want;
    }
    *out = ctx->ws;
    return MBE_OK;
}

// One thread per string I of class (n, k): the string's bit pattern by
// unranking in the combinatorial number system, then its replacement list
// E_pq |I> = sign |J>, q occupied (ascending), p empty or p == q (ascending).
__global__ void k_string_table(int n, int k, int64_t ns, int r, uint32_t *strings, int32_t *table)
{
    int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= ns) return;
    // Unrank: the largest c with C(c, i) <= rank, for i = k .. 1.
    uint32_t s = 0;
    int64_t rem = I;
    int c = n - 1;
    for (int i = k; i >= 1; --i) {
        while (binom(c, i) > rem) --c;
        s |= 1u << c;
        rem -= binom(c, i);
        --c;
    }
    strings[I] = s;
    if (!table) return;
    int32_t *row = table + I * r;
    int e = 0;
    for (int q = 0; q < n; ++q) {
        if (!((s >> q) & 1u)) continue;
        for (int p = 0; p < n; ++p) {
            if (p != q && ((s >> p) & 1u)) continue;
            uint32_t J = (s & ~(1u << q)) | (1u << p);
            int lo = p < q ? p : q, hi = p < q ? q : p;
            uint32_t between = (hi - lo > 1) ? (s & (((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u))) : 0u;
            int neg = __popc(between) & 1;
            row[e++] = (string_rank(J) << 9) | (pair_index(p, q) << 1) | neg;
        }
    }
}

int check_dev_err(mbe_ctx *ctx)
{
    int h = 0;
    MBE_CU(cudaMemcpyAsync(&h, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    if (h) {
        MBE_CU(cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), ctx->stream));
        set_error("a kernel's bounded wait on its tensor-core work ran out (results discarded)");
        return MBE_ECUDA;
    }
    return MBE_OK;
}

int get_table(mbe_ctx *ctx, int n, int k, const StringTable **out)
{
    MBE_CHECK(n >= 0 && n <= MBE_MAX_STRING_ORB && k >= 0 && k <= n, MBE_EUNSUPPORTED,
              "string class (%d, %d) outside 0 <= k <= n <= %d", n, k, MBE_MAX_STRING_ORB);
    StringTable &t = ctx->tables[n][k];
    if (!t.strings) {
        t.n = n;
        t.k = k;
        t.ns = binom(n, k);
        t.r = k * (n - k + 1);
        void *p = nullptr;
        MBE_CU(cudaMalloc(&p, t.ns * sizeof(uint32_t)));
        t.strings = (uint32_t *)p;
        p = nullptr;
        MBE_CU(cudaMalloc(&p, (size_t)(t.ns * (t.r > 0 ? t.r : 1)) * sizeof(int32_t)));
        t.table = (int32_t *)p;
        int threads = 128;
        int blocks = (int)((t.ns + threads - 1) / threads);
        k_string_table<<<blocks, threads, 0, ctx->stream>>>(n, k, t.ns, t.r, t.strings, t.table);
        MBE_CU(cudaGetLastError());
        ++ctx->launches;
        // Built once per class and context; later calls may run on other streams.
        MBE_CU(cudaStreamSynchronize(ctx->stream));
    }
    *out = &t;
    return MBE_OK;
}

}  // namespace mbe

using namespace mbe;

extern "C" {

void mbe_default_opts(mbe_opts *o)
{
    if (!o) return;
    o->precision = MBE_PREC_FP64;
    o->tol = 1e-7;
    o->tol_switch = 1e-5;
    o->max_iter = 2000;
    o->fp64_final_iters = 2;
    o->sectors = MBE_SECTORS_BOTH;
    o->s2_penalty = 0.0;
}

const char *mbe_last_error(void) { return g_err; }

int mbe_ctx_create(mbe_ctx **ctx, int device, void *cuda_stream)
{
    MBE_CHECK(ctx != nullptr, MBE_EINVAL, "mbe_ctx_create: ctx is NULL");
    *ctx = nullptr;
    int ndev = 0;
    MBE_CU(cudaGetDeviceCount(&ndev));
    MBE_CHECK(device >= 0 && device < ndev, MBE_EINVAL, "mbe_ctx_create: device %d of %d", device, ndev);
    MBE_CU(cudaSetDevice(device));
    mbe_ctx *c = new (std::nothrow) mbe_ctx();
    MBE_CHECK(c != nullptr, MBE_ENOMEM, "mbe_ctx_create: out of host memory");
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaGetDeviceProperties", __FILE__, __LINE__);
    }
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    for (auto &row : c->tune)
        for (auto &t : row) t = mbe_tuning{WARP_MAX_NDET, 4, 20};
    e = cudaMalloc(&c->dev_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->dev_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        if (c->dev_err) cudaFree(c->dev_err);
        delete c;
        return cuda_fail(e, "mbe_ctx_create: error flag", __FILE__, __LINE__);
    }
    *ctx = c;
    return MBE_OK;
}

int mbe_ctx_set_tuning(mbe_ctx *ctx, int precision, int n_cas, const mbe_tuning *t)
{
    MBE_CHECK(ctx && t, MBE_EINVAL, "mbe_ctx_set_tuning: NULL argument");
    MBE_CHECK(precision == MBE_PREC_FP64 || precision == MBE_PREC_MIXED, MBE_EINVAL,
              "mbe_ctx_set_tuning: precision %d", precision);
    MBE_CHECK(n_cas >= 0 && n_cas <= MBE_MAX_CAS, MBE_EINVAL, "mbe_ctx_set_tuning: n_cas %d", n_cas);
    MBE_CHECK(t->warp_max_ndet >= 1 && t->warp_max_ndet <= WARP_MAX_NDET && t->warp_warps >= 1 && t->warp_warps <= 4 &&
                  t->block_basis >= 4 && t->block_basis <= 20,
              MBE_EINVAL, "mbe_ctx_set_tuning: values out of range (%d, %d, %d)", t->warp_max_ndet, t->warp_warps,
              t->block_basis);
    const int p = precision == MBE_PREC_MIXED ? 1 : 0;
    for (int n = 0; n <= MBE_MAX_CAS; ++n)
        if (n_cas == 0 || n == n_cas) ctx->tune[p][n] = *t;
    return MBE_OK;
}

int mbe_ctx_get_tuning(const mbe_ctx *ctx, int precision, int n_cas, mbe_tuning *t)
{
    MBE_CHECK(ctx && t, MBE_EINVAL, "mbe_ctx_get_tuning: NULL argument");
    MBE_CHECK(precision == MBE_PREC_FP64 || precision == MBE_PREC_MIXED, MBE_EINVAL,
              "mbe_ctx_get_tuning: precision %d", precision);
    MBE_CHECK(n_cas >= 0 && n_cas <= MBE_MAX_CAS, MBE_EINVAL, "mbe_ctx_get_tuning: n_cas %d", n_cas);
    *t = ctx->tune[precision == MBE_PREC_MIXED ? 1 : 0][n_cas];
    return MBE_OK;
}

int mbe_ctx_set_stream(mbe_ctx *ctx, void *cuda_stream)
{
    MBE_CHECK(ctx != nullptr, MBE_EINVAL, "mbe_ctx_set_stream: ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    return MBE_OK;
}

int mbe_ctx_sync(mbe_ctx *ctx)
{
    MBE_CHECK(ctx != nullptr, MBE_EINVAL, "mbe_ctx_sync: ctx is NULL");
    MBE_CU(cudaSetDevice(ctx->device));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    MBE_CU(cudaGetLastError());
    return check_dev_err(ctx);
}

void mbe_ctx_destroy(mbe_ctx *ctx)
{
    if (!ctx) return;
    for (size_t i = 0; i < ctx->workers.size(); ++i) {
        mbe_ctx_destroy(ctx->workers[i]);
        cudaStreamDestroy(ctx->worker_streams[i]);
    }
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFreeAsync(ctx->ws, ctx->stream);
    for (auto &p : ctx->pending) {
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    for (int n = 0; n <= MBE_MAX_STRING_ORB; ++n)
        for (int k = 0; k <= MBE_MAX_STRING_ORB; ++k) {
            if (ctx->tables[n][k].strings) cudaFree(ctx->tables[n][k].strings);
            if (ctx->tables[n][k].table) cudaFree(ctx->tables[n][k].table);
        }
    cudaStreamSynchronize(ctx->stream);
    if (ctx->dev_err) cudaFree(ctx->dev_err);
    delete ctx;
}

int mbe_ctx_launches(const mbe_ctx *ctx, int64_t *count)
{
    MBE_CHECK(ctx != nullptr && count != nullptr, MBE_EINVAL, "mbe_ctx_launches: NULL argument");
    *count = ctx->launches;
    return MBE_OK;
}

int mbe_ctx_set_timing(mbe_ctx *ctx, int enable)
{
    MBE_CHECK(ctx != nullptr, MBE_EINVAL, "mbe_ctx_set_timing: ctx is NULL");
    ctx->timing = enable != 0;
    return MBE_OK;
}

int mbe_ctx_timings(mbe_ctx *ctx, int max, mbe_timing *out, int *count)
{
    MBE_CHECK(ctx != nullptr && count != nullptr && (max == 0 || out != nullptr), MBE_EINVAL,
              "mbe_ctx_timings: NULL argument");
    MBE_CU(cudaSetDevice(ctx->device));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    int n = 0;
    for (auto &p : ctx->pending) {
        float ms = 0.0f;
        MBE_CU(cudaEventElapsedTime(&ms, p.start, p.stop));
        if (n < max) {
            out[n] = p.rec;
            out[n].ms = ms;
        }
        ++n;
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
    }
    ctx->pending.clear();
    *count = n;
    return MBE_OK;
}

int mbe_string_table(mbe_ctx *ctx, int n_orb, int n_el, uint32_t *strings, int32_t *table)
{
    MBE_CHECK(ctx != nullptr && strings != nullptr, MBE_EINVAL, "mbe_string_table: NULL argument");
    MBE_CHECK(n_orb >= 0 && n_el >= 0 && n_el <= n_orb, MBE_EINVAL,
              "mbe_string_table: need 0 <= n_el <= n_orb (got %d, %d)", n_el, n_orb);
    MBE_CHECK(n_orb <= MBE_MAX_STRING_ORB, MBE_EUNSUPPORTED, "mbe_string_table: n_orb %d > %d",
              n_orb, MBE_MAX_STRING_ORB);
    MBE_CU(cudaSetDevice(ctx->device));
    const StringTable *t = nullptr;
    int rc = get_table(ctx, n_orb, n_el, &t);
    if (rc) return rc;
    MBE_CU(cudaMemcpyAsync(strings, t->strings, t->ns * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                           ctx->stream));
    if (table && t->r > 0)
        MBE_CU(cudaMemcpyAsync(table, t->table, (size_t)(t->ns * t->r) * sizeof(int32_t),
                               cudaMemcpyDeviceToDevice, ctx->stream));
    return MBE_OK;
}

}  // extern "C"
