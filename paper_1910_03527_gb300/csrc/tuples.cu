// a1: tuple enumeration on the device (Eq. 2's order-n tuples, skip rule after Eq. 3).
//
// Rank r in [0, C(M, n)) of the sorted expansion space -> lexicographic
// unranking into positions -> orbital indices -> skip filter -> order-preserving
// compaction (per-block counts, one scan, per-block scatter).
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace mbe {

constexpr int TB = 256;

struct TupleArgs {
    int M;                 // expansion-space size
    int order;
    int64_t total;         // C(M, order)
    int skip;              // apply the skip rule
    int ref_occ, ref_vir;  // reference space holds an occupied / virtual orbital
    int32_t exp[MBE_MAX_NORB];
    uint8_t exp_occ[MBE_MAX_NORB];
};

// Positions c_0 < c_1 < ... < c_{n-1} of the r-th n-subset of {0..M-1} in
// lexicographic order.
__device__ inline void lex_unrank(int64_t r, int M, int n, int *c)
{
    int x = 0;
    for (int i = 0; i < n; ++i) {
        for (;;) {
            int64_t cnt = binom(M - 1 - x, n - 1 - i);
            if (r < cnt) break;
            r -= cnt;
            ++x;
        }
        c[i] = x++;
    }
}

__device__ inline bool keep_rank(const TupleArgs &a, int64_t r, int *c)
{
    lex_unrank(r, a.M, a.order, c);
    if (!a.skip) return true;
    int nocc = 0;
    for (int i = 0; i < a.order; ++i) nocc += a.exp_occ[c[i]];
    bool has_occ = a.ref_occ || nocc > 0;
    bool has_vir = a.ref_vir || nocc < a.order;
    return has_occ && has_vir;
}

__global__ void k_tuple_count(TupleArgs a, int32_t *block_counts)
{
    __shared__ int warp_tot[TB / 32];
    int64_t r = (int64_t)blockIdx.x * TB + threadIdx.x;
    int c[MBE_MAX_ORDER];
    int keep = (r < a.total) ? (int)keep_rank(a, r, c) : 0;
    unsigned m = __ballot_sync(0xffffffffu, keep);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < TB / 32; ++w) s += warp_tot[w];
        block_counts[blockIdx.x] = s;
    }
}

// Exclusive scan of the block counts (one block; sequential over chunks).
__global__ void k_scan_counts(const int32_t *counts, int64_t nblocks, int64_t *offsets)
{
    __shared__ int64_t part[TB];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nblocks; base += TB) {
        int64_t i = base + threadIdx.x;
        int64_t v = (i < nblocks) ? counts[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < TB; off <<= 1) {
            int64_t add = (threadIdx.x >= (unsigned)off) ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nblocks) offsets[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == TB - 1) carry += part[TB - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[nblocks] = carry;
}

__global__ void k_tuple_write(TupleArgs a, const int64_t *offsets, int32_t *tuples)
{
    __shared__ int warp_base[TB / 32];
    int64_t r = (int64_t)blockIdx.x * TB + threadIdx.x;
    int c[MBE_MAX_ORDER];
    int keep = (r < a.total) ? (int)keep_rank(a, r, c) : 0;
    unsigned m = __ballot_sync(0xffffffffu, keep);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_base[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int i = 0; i < TB / 32; ++i) {
            int v = warp_base[i];
            warp_base[i] = s;
            s += v;
        }
    }
    __syncthreads();
    if (keep) {
        int64_t pos = offsets[blockIdx.x] + warp_base[w] + __popc(m & ((1u << lane) - 1u));
        int32_t *row = tuples + pos * a.order;
        for (int i = 0; i < a.order; ++i) row[i] = a.exp[c[i]];
    }
}

}  // namespace mbe

using namespace mbe;

extern "C" int mbe_tuples(mbe_ctx *ctx, int norb, const uint8_t *occ, int n_exp,
                          const int32_t *exp_orbs, int n_ref, const int32_t *ref_orbs, int order,
                          int flags, int64_t *n_tuples, int32_t *tuples)
{
    MBE_CHECK(n_tuples != nullptr && occ != nullptr && (n_exp == 0 || exp_orbs != nullptr) &&
                  (n_ref == 0 || ref_orbs != nullptr),
              MBE_EINVAL, "mbe_tuples: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "mbe_tuples: norb %d outside 1..%d",
              norb, MBE_MAX_NORB);
    MBE_CHECK(order >= 1 && order <= n_exp && order <= MBE_MAX_ORDER, MBE_EINVAL,
              "mbe_tuples: order %d outside 1..min(n_exp=%d, %d)", order, n_exp, MBE_MAX_ORDER);
    std::vector<int32_t> ex(exp_orbs, exp_orbs + n_exp);
    std::sort(ex.begin(), ex.end());
    std::vector<char> seen(norb, 0);
    for (int i = 0; i < n_exp; ++i) {
        MBE_CHECK(ex[i] >= 0 && ex[i] < norb && !seen[ex[i]], MBE_EINVAL,
                  "mbe_tuples: expansion orbital %d out of range or repeated", ex[i]);
        seen[ex[i]] = 1;
    }
    int ref_occ = 0, ref_vir = 0;
    for (int i = 0; i < n_ref; ++i) {
        MBE_CHECK(ref_orbs[i] >= 0 && ref_orbs[i] < norb && !seen[ref_orbs[i]], MBE_EINVAL,
                  "mbe_tuples: reference orbital %d out of range or in the expansion space",
                  ref_orbs[i]);
        if (occ[ref_orbs[i]]) ref_occ = 1; else ref_vir = 1;
    }
    int m_occ = 0;
    for (int i = 0; i < n_exp; ++i) m_occ += occ[ex[i]] ? 1 : 0;
    int m_vir = n_exp - m_occ;
    bool skip = (flags & MBE_SKIP_NO_OCC_OR_VIRT) != 0;
    int64_t total = binom(n_exp, order);
    int64_t count = total;
    if (skip) {
        if (!ref_occ) count -= binom(m_vir, order);
        if (!ref_vir) count -= binom(m_occ, order);
    }
    *n_tuples = count;
    if (!tuples || count == 0) return MBE_OK;
    MBE_CHECK(ctx != nullptr, MBE_EINVAL, "mbe_tuples: ctx is NULL");
    MBE_CU(cudaSetDevice(ctx->device));

    TupleArgs a;
    a.M = n_exp;
    a.order = order;
    a.total = total;
    a.skip = skip ? 1 : 0;
    a.ref_occ = ref_occ;
    a.ref_vir = ref_vir;
    for (int i = 0; i < n_exp; ++i) {
        a.exp[i] = ex[i];
        a.exp_occ[i] = occ[ex[i]] ? 1 : 0;
    }
    int64_t nblocks = (total + TB - 1) / TB;
    MBE_CHECK(nblocks < (1LL << 31), MBE_EUNSUPPORTED, "mbe_tuples: %lld candidate tuples",
              (long long)total);
    void *ws = nullptr;
    size_t bytes = align256(nblocks * sizeof(int32_t)) + align256((nblocks + 1) * sizeof(int64_t));
    int rc = workspace(ctx, bytes, &ws);
    if (rc) return rc;
    Bump b(ws);
    int32_t *counts = b.take<int32_t>(nblocks);
    int64_t *offsets = b.take<int64_t>(nblocks + 1);
    k_tuple_count<<<(unsigned)nblocks, TB, 0, ctx->stream>>>(a, counts);
    k_scan_counts<<<1, TB, 0, ctx->stream>>>(counts, nblocks, offsets);
    k_tuple_write<<<(unsigned)nblocks, TB, 0, ctx->stream>>>(a, offsets, tuples);
    MBE_CU(cudaGetLastError());
    ctx->launches += 3;
    return MBE_OK;
}
