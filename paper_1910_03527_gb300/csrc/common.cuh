// Internal declarations shared by the translation units of the MBE-FCI engine.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstddef>
#include <vector>

#include "mbe.h"

namespace mbe {

// ------------------------------------------------------------------ errors

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define MBE_CU(call)                                                     \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::mbe::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define MBE_CHECK(cond, code, ...)              \
    do {                                        \
        if (!(cond)) {                          \
            ::mbe::set_error(__VA_ARGS__);      \
            return (code);                      \
        }                                       \
    } while (0)

// Determinants one warp of the warp solver holds (13 per lane): the upper limit
// of mbe_tuning.warp_max_ndet and its default.
inline constexpr int WARP_MAX_NDET = 416;

// ------------------------------------------------------------------ combinatorics

__host__ __device__ inline int64_t binom(int n, int k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    int64_t c = 1;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}

// Packed index of the unordered orbital pair {p, q}.
__host__ __device__ inline int pair_index(int p, int q)
{
    int hi = p > q ? p : q, lo = p > q ? q : p;
    return hi * (hi + 1) / 2 + lo;
}

// Rank of a string (bit pattern) in ascending order among strings with the same
// number of set bits: sum over set bits c_1 < c_2 < ... of C(c_i, i).
__host__ __device__ inline int32_t string_rank(uint32_t s)
{
    int32_t r = 0;
    int i = 0;
    while (s) {
#ifdef __CUDA_ARCH__
        int c = __ffs((int)s) - 1;
#else
        int c = __builtin_ctz(s);
#endif
        ++i;
        r += (int32_t)binom(c, i);
        s &= s - 1;
    }
    return r;
}

// ------------------------------------------------------------------ string tables

struct StringTable {
    int n = 0, k = 0;
    int64_t ns = 0;   // number of strings C(n, k)
    int r = 0;        // replacement entries per string k (n - k + 1)
    uint32_t *strings = nullptr;  // device [ns]
    int32_t *table = nullptr;     // device [ns * r]
};

// Table entry packing: (J << 9) | (pair << 1) | negative
__host__ __device__ inline int entry_J(int32_t e) { return e >> 9; }
__host__ __device__ inline int entry_pair(int32_t e) { return (e >> 1) & 255; }
__host__ __device__ inline int entry_neg(int32_t e) { return e & 1; }

}  // namespace mbe

// ------------------------------------------------------------------ context

struct mbe_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    size_t smem_optin = 0;
    void *ws = nullptr;
    size_t ws_size = 0;
    mbe::StringTable tables[MBE_MAX_STRING_ORB + 1][MBE_MAX_STRING_ORB + 1];
    int *dev_err = nullptr;  // device flag set by a kernel whose bounded wait ran out
    // launch choices of casci_batch per precision (0 float64, 1 mixed) and active-space
    // size |R| + order (mbe_ctx_set_tuning, mbe_autotune)
    mbe_tuning tune[2][MBE_MAX_CAS + 1];
    int64_t launches = 0;  // kernels launched by this context
    bool timing = false;
    struct Pending {
        mbe_timing rec;
        cudaEvent_t start, stop;
    };
    std::vector<Pending> pending;
    // worker contexts of casci_batch_routed, each on its own non-blocking stream
    // (created on first use, destroyed with this context)
    std::vector<mbe_ctx *> workers;
    std::vector<cudaStream_t> worker_streams;
};

namespace mbe {

// Device workspace of at least `bytes` (stream-ordered growth).  The returned
// pointer stays valid until the next call that grows the workspace.
int workspace(mbe_ctx *ctx, size_t bytes, void **out);

// Cached device string table of class (n, k); builds it on first use.
int get_table(mbe_ctx *ctx, int n, int k, const StringTable **out);

// Reads and clears the context's device error flag (synchronous); MBE_ECUDA with a
// message when a kernel's bounded wait ran out.
int check_dev_err(mbe_ctx *ctx);

// Bump allocator over a workspace region.
struct Bump {
    char *base;
    size_t off = 0;
    explicit Bump(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base + off);
        off += count * sizeof(T);
        return p;
    }
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Position of the m-tuple `key` in a lexicographically sorted list, or -1.
__device__ inline int64_t find_tuple(const int32_t *list, int64_t len, int m, const int32_t *key)
{
    int64_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) >> 1;
        const int32_t *row = list + mid * m;
        int cmp = 0;
        for (int i = 0; i < m; ++i) {
            if (row[i] != key[i]) {
                cmp = row[i] < key[i] ? -1 : 1;
                break;
            }
        }
        if (cmp == 0) return mid;
        if (cmp < 0) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Exclusive scan of per-block counts into offsets[0..nblocks] (one block).
__global__ void k_scan_counts(const int32_t *counts, int64_t nblocks, int64_t *offsets);

// The opposite-spin term of one large active space's float32 sigma on the tensor
// cores (large_tc.cu): sigma[Ia][*] written for every alpha string Ia from the
// float32 coefficients c [Ns][Ns], the replacement lists tab [Ns][R] and the
// float32 packed-pair integrals V32 [P][P].  *err (device) is set to 1 if a
// bounded wait runs out.
int large_ab_tc(cudaStream_t st, int sm_count, size_t smem_optin, int P, int Ns, int R, const int32_t *tab,
                const float *V32, const float *c, double *sigma, int *err);

}  // namespace mbe
