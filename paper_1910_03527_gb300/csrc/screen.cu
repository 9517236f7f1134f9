// Screened expansion on the device: child spawning (Sec. 2) with the per-tuple
// thresholds of Eq. 4.
//
// An order-(k+1) tuple of the expansion space is spawned when the absolute
// increment of at least one of its order-k sub-tuples exceeds the child's
// threshold T_tup = T_init a^(M_tup - M_init) (zero below M_init), M_tup the
// larger of its occupied and virtual orbital counts; sub-tuples that were not
// computed count as zero, and the skip rule still applies to the child.
//
// Every spawned child has a computed sub-tuple (the one above threshold), so the
// candidates are (parent P, orbital c not in P). A child with several computed
// sub-tuples is emitted once: by the parent P = child \ {x*}, x* the largest
// orbital whose removal leaves a computed tuple. Per candidate this takes k + 1
// binary searches in the lexicographic parent list. Emitted children are written
// as their lexicographic rank among the (k+1)-subsets of the expansion space,
// sorted by an LSD radix sort (4-bit digits, stable per-block ranking) and
// unranked, so the output is lexicographic like mbe_tuples'.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace mbe {

constexpr int SP_TB = 256;

struct SpawnArgs {
    int M;      // expansion-space size
    int k;      // parent order; children have k + 1 orbitals
    int skip;
    int ref_occ, ref_vir;
    int32_t exp[MBE_MAX_NORB];         // sorted expansion orbitals
    int8_t pos[MBE_MAX_NORB];          // orbital -> position in exp, or -1
    uint8_t occ[MBE_MAX_NORB];         // orbital occupations
    double thr[MBE_MAX_ORDER + 2];     // child threshold by its occupied count
};

// Decides whether candidate t = parent * M + j is emitted; on success writes the
// child's positions (ascending) to cp.
__device__ inline bool spawn_candidate(const SpawnArgs &a, int64_t n_par, const int32_t *par,
                                       const double *inc, int64_t t, int *cp)
{
    const int k = a.k, n = k + 1;
    const int64_t p = t / a.M;
    const int j = (int)(t - p * a.M);
    const int c = a.exp[j];
    const int32_t *P = par + p * k;
    int child[MBE_MAX_ORDER + 1];
    int at = 0;
    bool placed = false;
    for (int i = 0; i < k; ++i) {
        const int o = P[i];
        if (o == c) return false;
        if (!placed && c < o) {
            child[at++] = c;
            placed = true;
        }
        child[at++] = o;
    }
    if (!placed) child[at++] = c;
    int nocc = 0;
    for (int i = 0; i < n; ++i) {
        const int o = child[i];
        if (o < 0 || o >= MBE_MAX_NORB || a.pos[o] < 0) return false;
        cp[i] = a.pos[o];
        nocc += a.occ[o];
    }
    if (a.skip) {
        const bool has_occ = a.ref_occ || nocc > 0, has_vir = a.ref_vir || nocc < n;
        if (!(has_occ && has_vir)) return false;
    }
    // the emitting parent: no computed sub-tuple may drop an orbital larger than c
    int32_t key[MBE_MAX_ORDER];
    double best = fabs(inc[p]);
    for (int r = n - 1; r >= 0; --r) {
        if (child[r] == c) continue;
        int m = 0;
        for (int i = 0; i < n; ++i)
            if (i != r) key[m++] = child[i];
        const int64_t f = find_tuple(par, n_par, k, key);
        if (f < 0) continue;
        if (child[r] > c) return false;
        best = fmax(best, fabs(inc[f]));
    }
    return best > a.thr[nocc];
}

// Lexicographic rank of the ascending positions cp[0..n) among the n-subsets of
// {0..M-1} (inverse of the unranking in tuples.cu).
__device__ inline int64_t lex_rank(const int *cp, int M, int n)
{
    int64_t r = 0;
    int x = 0;
    for (int i = 0; i < n; ++i) {
        for (; x < cp[i]; ++x) r += binom(M - 1 - x, n - 1 - i);
        x = cp[i] + 1;
    }
    return r;
}

__device__ inline void lex_unrank_pos(int64_t r, int M, int n, int *c)
{
    int x = 0;
    for (int i = 0; i < n; ++i) {
        for (;;) {
            const int64_t cnt = binom(M - 1 - x, n - 1 - i);
            if (r < cnt) break;
            r -= cnt;
            ++x;
        }
        c[i] = x++;
    }
}

__global__ void k_spawn_count(SpawnArgs a, int64_t n_par, const int32_t *par, const double *inc,
                              int32_t *block_counts)
{
    __shared__ int warp_tot[SP_TB / 32];
    const int64_t t = (int64_t)blockIdx.x * SP_TB + threadIdx.x;
    int cp[MBE_MAX_ORDER + 1];
    const int keep = (t < n_par * a.M) ? (int)spawn_candidate(a, n_par, par, inc, t, cp) : 0;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < SP_TB / 32; ++w) s += warp_tot[w];
        block_counts[blockIdx.x] = s;
    }
}

__global__ void k_spawn_write(SpawnArgs a, int64_t n_par, const int32_t *par, const double *inc,
                              const int64_t *offsets, uint64_t *keys)
{
    __shared__ int warp_base[SP_TB / 32];
    const int64_t t = (int64_t)blockIdx.x * SP_TB + threadIdx.x;
    int cp[MBE_MAX_ORDER + 1];
    const int keep = (t < n_par * a.M) ? (int)spawn_candidate(a, n_par, par, inc, t, cp) : 0;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_base[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int i = 0; i < SP_TB / 32; ++i) {
            const int v = warp_base[i];
            warp_base[i] = s;
            s += v;
        }
    }
    __syncthreads();
    if (keep) {
        const int64_t at = offsets[blockIdx.x] + warp_base[w] + __popc(m & ((1u << lane) - 1u));
        keys[at] = (uint64_t)lex_rank(cp, a.M, a.k + 1);
    }
}

// ---- LSD radix sort of 64-bit keys, 4-bit digits, tiles of RS_ITEMS x 256 keys

constexpr int RS_THREADS = 256, RS_ITEMS = 8, RS_TILE = RS_THREADS * RS_ITEMS, RS_BINS = 16;

__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const uint64_t *keys, int64_t n, int shift,
                                                           int64_t nblk, int32_t *hist)
{
    __shared__ int h[RS_BINS];
    if (threadIdx.x < RS_BINS) h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int64_t idx = base + i * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & (RS_BINS - 1)], 1);
    }
    __syncthreads();
    if (threadIdx.x < RS_BINS) hist[threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: keys of a tile are ranked in index order (rounds of 256 in
// thread order; within a warp by lane, across warps by warp).
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const uint64_t *in, uint64_t *out, int64_t n,
                                                              int shift, int64_t nblk, const int64_t *off)
{
    __shared__ int64_t run[RS_BINS];
    __shared__ int wcnt[RS_THREADS / 32][RS_BINS];
    __shared__ int wpre[RS_THREADS / 32][RS_BINS];
    __shared__ int tot[RS_BINS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < RS_BINS) run[threadIdx.x] = off[threadIdx.x * nblk + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = 0; i < RS_ITEMS; ++i) {
        if (threadIdx.x < (RS_THREADS / 32) * RS_BINS) (&wcnt[0][0])[threadIdx.x] = 0;
        __syncthreads();
        const int64_t idx = base + i * RS_THREADS + threadIdx.x;
        const bool valid = idx < n;
        const uint64_t key = valid ? in[idx] : 0;
        const int d = valid ? (int)((key >> shift) & (RS_BINS - 1)) : RS_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < RS_BINS) {
            int s = 0;
            for (int v = 0; v < RS_THREADS / 32; ++v) {
                wpre[v][threadIdx.x] = s;
                s += wcnt[v][threadIdx.x];
            }
            tot[threadIdx.x] = s;
        }
        __syncthreads();
        if (valid) out[run[d] + wpre[w][d] + rank] = key;
        __syncthreads();
        if (threadIdx.x < RS_BINS) run[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
}

__global__ void k_unrank_children(SpawnArgs a, const uint64_t *keys, int64_t n, int32_t *children)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[MBE_MAX_ORDER + 1];
    lex_unrank_pos((int64_t)keys[i], a.M, a.k + 1, c);
    int32_t *row = children + i * (a.k + 1);
    for (int j = 0; j <= a.k; ++j) row[j] = a.exp[c[j]];
}

}  // namespace mbe

using namespace mbe;

extern "C" int mbe_screen(mbe_ctx *ctx, int norb, const uint8_t *occ, int n_exp, const int32_t *exp_orbs,
                          int n_ref, const int32_t *ref_orbs, int order, int64_t n_parents,
                          const int32_t *parents, const double *parent_incs, double t_init, int m_init, double a,
                          int flags, int64_t capacity, int64_t *n_children, int32_t *children)
{
    MBE_CHECK(ctx != nullptr && n_children != nullptr && occ != nullptr && (n_exp == 0 || exp_orbs != nullptr) &&
                  (n_ref == 0 || ref_orbs != nullptr),
              MBE_EINVAL, "mbe_screen: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "mbe_screen: norb %d outside 1..%d", norb,
              MBE_MAX_NORB);
    MBE_CHECK(order >= 1 && order + 1 <= n_exp && order + 1 <= MBE_MAX_ORDER, MBE_EINVAL,
              "mbe_screen: child order %d outside 2..min(n_exp=%d, %d)", order + 1, n_exp, MBE_MAX_ORDER);
    MBE_CHECK(n_parents >= 0 && (n_parents == 0 || (parents != nullptr && parent_incs != nullptr)), MBE_EINVAL,
              "mbe_screen: %lld parents without tuples or increments", (long long)n_parents);
    MBE_CHECK(t_init >= 0.0 && a >= 0.0 && m_init >= 0, MBE_EINVAL,
              "mbe_screen: thresholds need T_init >= 0, a >= 0, M_init >= 0");
    std::vector<int32_t> ex(exp_orbs, exp_orbs + n_exp);
    std::sort(ex.begin(), ex.end());
    SpawnArgs sa;
    memset(&sa, 0, sizeof(sa));
    for (int o = 0; o < MBE_MAX_NORB; ++o) sa.pos[o] = -1;
    for (int i = 0; i < n_exp; ++i) {
        MBE_CHECK(ex[i] >= 0 && ex[i] < norb && sa.pos[ex[i]] < 0, MBE_EINVAL,
                  "mbe_screen: expansion orbital %d out of range or repeated", ex[i]);
        sa.pos[ex[i]] = (int8_t)i;
        sa.exp[i] = ex[i];
    }
    for (int i = 0; i < n_ref; ++i) {
        MBE_CHECK(ref_orbs[i] >= 0 && ref_orbs[i] < norb && sa.pos[ref_orbs[i]] < 0, MBE_EINVAL,
                  "mbe_screen: reference orbital %d out of range or in the expansion space", ref_orbs[i]);
        if (occ[ref_orbs[i]]) sa.ref_occ = 1; else sa.ref_vir = 1;
    }
    for (int o = 0; o < norb; ++o) sa.occ[o] = occ[o] ? 1 : 0;
    sa.M = n_exp;
    sa.k = order;
    sa.skip = (flags & MBE_SKIP_NO_OCC_OR_VIRT) ? 1 : 0;
    // Eq. 4 per occupied count of the child, by repeated products in this order
    const int n = order + 1;
    for (int no = 0; no <= n; ++no) {
        const int m_tup = std::max(no, n - no);
        double t = 0.0;
        if (m_tup >= m_init) {
            t = t_init;
            for (int e = 0; e < m_tup - m_init; ++e) t *= a;
        }
        sa.thr[no] = t;
    }
    *n_children = 0;
    if (n_parents == 0) return MBE_OK;
    MBE_CU(cudaSetDevice(ctx->device));
    const int64_t cand = n_parents * n_exp;
    const int64_t nblocks = (cand + SP_TB - 1) / SP_TB;
    MBE_CHECK(nblocks < (1LL << 31), MBE_EUNSUPPORTED, "mbe_screen: %lld candidates", (long long)cand);
    // an upper bound on the children: each candidate emits at most one
    const int64_t max_children = cand;
    const int64_t rs_blocks_max = (max_children + RS_TILE - 1) / RS_TILE;
    const size_t bytes = align256(nblocks * 4) + align256((nblocks + 1) * 8) + 2 * align256(max_children * 8) +
                         align256(RS_BINS * rs_blocks_max * 4) + align256((RS_BINS * rs_blocks_max + 1) * 8) + 4096;
    void *ws = nullptr;
    int rc = workspace(ctx, bytes, &ws);
    if (rc) return rc;
    Bump b(ws);
    int32_t *counts = b.take<int32_t>(nblocks);
    int64_t *offsets = b.take<int64_t>(nblocks + 1);
    uint64_t *keys = b.take<uint64_t>(max_children);
    uint64_t *keys2 = b.take<uint64_t>(max_children);
    int32_t *hist = b.take<int32_t>(RS_BINS * rs_blocks_max);
    int64_t *hoff = b.take<int64_t>(RS_BINS * rs_blocks_max + 1);
    k_spawn_count<<<(unsigned)nblocks, SP_TB, 0, ctx->stream>>>(sa, n_parents, parents, parent_incs, counts);
    k_scan_counts<<<1, 256, 0, ctx->stream>>>(counts, nblocks, offsets);
    int64_t total = 0;
    MBE_CU(cudaMemcpyAsync(&total, offsets + nblocks, 8, cudaMemcpyDeviceToHost, ctx->stream));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    ctx->launches += 2;
    *n_children = total;
    if (!children || total == 0) return MBE_OK;
    MBE_CHECK(total <= capacity, MBE_EINVAL, "mbe_screen: %lld children exceed the capacity %lld",
              (long long)total, (long long)capacity);
    k_spawn_write<<<(unsigned)nblocks, SP_TB, 0, ctx->stream>>>(sa, n_parents, parents, parent_incs, offsets, keys);
    // digits needed: bit length of C(M, k+1) - 1
    const uint64_t max_key = (uint64_t)binom(n_exp, n) - 1;
    int bits = 0;
    while (bits < 64 && (max_key >> bits) != 0) ++bits;
    const int64_t nblk = (total + RS_TILE - 1) / RS_TILE;
    uint64_t *src = keys, *dst = keys2;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 4, ++passes) {
        k_radix_hist<<<(unsigned)nblk, RS_THREADS, 0, ctx->stream>>>(src, total, shift, nblk, hist);
        k_scan_counts<<<1, 256, 0, ctx->stream>>>(hist, RS_BINS * nblk, hoff);
        k_radix_scatter<<<(unsigned)nblk, RS_THREADS, 0, ctx->stream>>>(src, dst, total, shift, nblk, hoff);
        std::swap(src, dst);
    }
    k_unrank_children<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(sa, src, total, children);
    MBE_CU(cudaGetLastError());
    ctx->launches += 2 + 3 * passes;
    return MBE_OK;
}
