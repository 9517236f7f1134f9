// a5, the dense part of the large-CAS sigma on the tensor cores (tcgen05, TF32).
//
// The opposite-spin term of sigma = H c for one large active space,
//     sigma[Ia][Ib] = sum_{x in list(Ia)} s_x sum_{y in list(Ib)} s_y V[p_x][p_y] c[J_x][J_y],
// is formed per alpha string Ia as a dense product followed by a scatter:
//     T[jb][p] = sum_x c[J_x][Jb0 + jb] * (s_x V[p_x][p])          (tensor cores)
//     sigma[Ia][K] += s T[jb][p]  for every entry E_p |Jb> = s |K> of Jb's list
// (e_p = E_pq + E_qp is symmetric, so the entries of Jb's list are exactly the
// (K, p, s) that sigma[Ia][K] gathers from).  M = 128 beta strings Jb of a tile,
// N = the pair count rounded up to 16, K = the alpha-list length rounded up to 8.
//
// Precision: the float32 inputs are split into TF32 pairs v = hi + lo (hi the
// round-to-nearest TF32 value, lo the TF32 rounding of the remainder) and the
// product is accumulated in float32 as hi*hi + hi*lo + lo*hi, three MMAs per
// K step ("3xTF32"), which keeps float32-class accuracy (the dropped lo*lo term
// is about 2^-22 of each product).
//
// Data path per CTA (persistent over Ia, one CTA per SM):
//   * the B operand (N pairs x K list entries, signed V columns) is built once per
//     Ia in shared memory, hi and lo;
//   * per tile of 128 beta strings: the A operand (128 x K, the gathered rows of c)
//     is written to shared memory, one thread issues the 3 x K/8 tcgen05.mma into
//     a TMEM accumulator and commits them to an mbarrier; after the wait, the warps
//     copy the accumulator (tcgen05.ld) over the A operand, and each beta string
//     scatters through its own list into a shared-memory sigma row (shared atomics);
//   * the row is written to sigma (float64) once per Ia.
// Operands use the K-major no-swizzle layout: 8-row x 16-byte core matrices,
// adjacent in K at LBO = 128 bytes, adjacent in M/N at SBO = 32 K bytes.
// Every wait is bounded: a wait that runs out sets *err, and the kernel still
// frees its TMEM before it returns.
#include <algorithm>

#include "common.cuh"

namespace mbe {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;          // beta strings per tile (MMA M, TMEM lanes)
constexpr int TC_TMEM_COLS = 256;  // accumulator columns allocated (>= N, power of two)
constexpr long long TC_SPIN = 1LL << 26;  // bounded mbarrier polls
constexpr int TC_MAXQ = 16;  // x-quads gathered per thread: K up to 4 * 2 * TC_MAXQ = 128 list entries

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) in a K-major no-swizzle operand with Kp columns.
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int Kp)
{
    return (uint32_t)((r >> 3) * (32 * Kp) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// Shared-memory matrix descriptor (tcgen05): start, LBO, SBO in 16-byte units,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::tf32: float32 accumulator, TF32 A and B, both
// K-major, dense; N >> 3 and M >> 4 in their fields.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_round(float v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return __uint_as_float(r);
}

__device__ __forceinline__ void split_tf32(float v, float &hi, float &lo)
{
    hi = tf32_round(v);
    lo = tf32_round(v - hi);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// Waits for the mbarrier phase `parity`; false when the bounded poll runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity)
{
    for (long long it = 0; it < TC_SPIN; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcArgs {
    int P, Ns, R, Np, Kp;
    const int32_t *tab;  // [Ns][R] replacement lists
    const float *V32;    // [P][P]
    const float *c;      // [Ns][Ns] float32 coefficients
    double *sigma;       // [Ns][Ns], written
    int *err;            // set to 1 when a wait runs out
};

struct TcSmem {
    uint32_t off_bhi, off_blo, off_ahi, off_alo, off_T, off_row, off_jx, off_bar, off_tmem, bytes;
    int Ts;  // row stride (floats) of the staged accumulator tile
};

__host__ __device__ inline TcSmem tc_smem(int Np, int Kp, int Ns, int R)
{
    TcSmem S;
    uint32_t o = 0;
    auto take = [&](uint32_t bytes, uint32_t align) {
        o = (o + align - 1) / align * align;
        const uint32_t at = o;
        o += bytes;
        return at;
    };
    S.off_bhi = take((uint32_t)Np * Kp * 4, 1024);
    S.off_blo = take((uint32_t)Np * Kp * 4, 1024);
    S.off_ahi = take((uint32_t)TC_M * Kp * 4, 1024);
    S.off_alo = take((uint32_t)TC_M * Kp * 4, 1024);
    // the accumulator tile [TC_M][Ts] lies over the A operand (2 x TC_M x Kp floats)
    // when it fits there; the odd stride Np + 1 avoids shared-memory bank conflicts
    S.Ts = (Np + 1 <= 2 * Kp || Np > 2 * Kp) ? Np + 1 : Np;
    S.off_T = (S.Ts <= 2 * Kp) ? S.off_ahi : take((uint32_t)TC_M * S.Ts * 4, 16);
    S.off_row = take((uint32_t)Ns * 4, 16);
    S.off_jx = take((uint32_t)R * 4, 16);
    S.off_bar = take(8, 8);
    S.off_tmem = take(4, 4);
    S.bytes = (o + 127) / 128 * 128;
    return S;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_large_ab_tc(TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcSmem S = tc_smem(a.Np, a.Kp, a.Ns, a.R);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.P, Ns = a.Ns, R = a.R, Np = a.Np, Kp = a.Kp;
    unsigned char *bhi = smem + S.off_bhi, *blo = smem + S.off_blo;
    unsigned char *ahi = smem + S.off_ahi, *alo = smem + S.off_alo;
    float *row = (float *)(smem + S.off_row);
    int *jx = (int *)(smem + S.off_jx);
    const uint32_t bar = smem_u32(smem + S.off_bar);
    uint32_t *tslot = (uint32_t *)(smem + S.off_tmem);
    __shared__ int s_ok;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tf32_idesc(TC_M, Np);
    const uint32_t lbo = 128, sbo = 32u * (uint32_t)Kp;
    uint32_t phase = 0;
    bool ok = true;

    for (int Ia = blockIdx.x; Ia < Ns && ok; Ia += gridDim.x) {
        const int32_t *ta = a.tab + (size_t)Ia * R;
        for (int x = tid; x < R; x += TC_THREADS) jx[x] = entry_J(ta[x]);
        for (int i = tid; i < Ns; i += TC_THREADS) row[i] = 0.f;
        // B operand: B[p][x] = s_x V[p_x][p] (zero beyond P and R), hi and lo
        for (int i = tid; i < Np * (Kp / 4); i += TC_THREADS) {
            const int p = i / (Kp / 4), x0 = (i - p * (Kp / 4)) * 4;
            float4 h, l;
            float *hv = &h.x, *lv = &l.x;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int x = x0 + j;
                float v = 0.f;
                if (p < P && x < R) {
                    const int e = ta[x];
                    v = a.V32[entry_pair(e) * P + p];
                    if (entry_neg(e)) v = -v;
                }
                split_tf32(v, hv[j], lv[j]);
            }
            *(float4 *)(bhi + kmajor_off(p, x0, Kp)) = h;
            *(float4 *)(blo + kmajor_off(p, x0, Kp)) = l;
        }
        __syncthreads();
        for (int Jb0 = 0; Jb0 < Ns; Jb0 += TC_M) {
            // A operand: A[jb][x] = c[J_x][Jb0 + jb] (zero beyond Ns and R), hi and lo.
            // Thread (jb, q) gathers the quads x = 4q, 4(q + 2), ...: every load of
            // the tile is issued before the first shared-memory store.
            {
                const int jb = tid & (TC_M - 1), q0 = tid >> 7, Jb = Jb0 + jb;
                float g[TC_MAXQ][4];
#pragma unroll
                for (int i = 0; i < TC_MAXQ; ++i) {
                    const int x0 = 4 * (q0 + 2 * i);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int x = x0 + j;
                        g[i][j] = (x0 < Kp && Jb < Ns && x < R) ? __ldg(a.c + (size_t)jx[x] * Ns + Jb) : 0.f;
                    }
                }
#pragma unroll
                for (int i = 0; i < TC_MAXQ; ++i) {
                    const int x0 = 4 * (q0 + 2 * i);
                    if (x0 < Kp) {
                        float4 h, l;
                        split_tf32(g[i][0], h.x, l.x);
                        split_tf32(g[i][1], h.y, l.y);
                        split_tf32(g[i][2], h.z, l.z);
                        split_tf32(g[i][3], h.w, l.w);
                        *(float4 *)(ahi + kmajor_off(jb, x0, Kp)) = h;
                        *(float4 *)(alo + kmajor_off(jb, x0, Kp)) = l;
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t ah = smem_u32(ahi), al = smem_u32(alo), bh = smem_u32(bhi), bl = smem_u32(blo);
                for (int s = 0; s < Kp / 8; ++s) {
                    const uint32_t ko = (uint32_t)s * 256u;
                    mma_tf32(tmem, smem_desc(ah + ko, lbo, sbo), smem_desc(bh + ko, lbo, sbo), idesc, s > 0);
                    mma_tf32(tmem, smem_desc(ah + ko, lbo, sbo), smem_desc(bl + ko, lbo, sbo), idesc, 1);
                    mma_tf32(tmem, smem_desc(al + ko, lbo, sbo), smem_desc(bh + ko, lbo, sbo), idesc, 1);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 bar)
                             : "memory");
                // one thread waits (bounded) and hands the outcome to the block
                s_ok = mbar_wait(bar, phase) ? 1 : 0;
                if (!s_ok) atomicExch(a.err, 1);
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            }
            __syncthreads();
            if (!s_ok) {
                ok = false;
                break;
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // epilogue 1: the accumulator tile T[jb][p] to shared memory, over the A
            // operand (free once the MMAs completed); warp w reads TMEM lanes
            // 32 (w % 4) .. + 31, half (w / 4) of the columns
            float *T = (float *)(smem + S.off_T);  // [TC_M][S.Ts]
            {
                const int jb = (warp & 3) * 32 + lane;
                const int half = Np / 16;  // column chunks of 8 in the first half
                const int c0 = (warp >> 2) ? half : 0, c1 = (warp >> 2) ? Np / 8 : half;
                const uint32_t tbase = tmem + ((uint32_t)((warp & 3) * 32) << 16);
                for (int ch = c0; ch < c1; ++ch) {
                    float v[8];
                    tmem_ld8(tbase + (uint32_t)(ch * 8), v);
#pragma unroll
                    for (int i = 0; i < 8; ++i) T[jb * S.Ts + ch * 8 + i] = v[i];
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            // epilogue 2: each beta string Jb of the tile walks its own list, E_pq|Jb> =
            // s|K>: sigma[Ia][K] += s T[Jb][pair(p,q)] (shared atomics); two threads per
            // string split the list
            {
                const int jb = tid & (TC_M - 1), part = tid >> 7, Jb = Jb0 + jb;
                if (Jb < Ns) {
                    const int32_t *tb = a.tab + (size_t)Jb * R;
                    const float *Trow = T + jb * S.Ts;
                    for (int y = part; y < R; y += 2) {
                        const int e = __ldg(tb + y);
                        const float v = Trow[entry_pair(e)];
                        atomicAdd(&row[entry_J(e)], entry_neg(e) ? -v : v);
                    }
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (ok)
            for (int K = tid; K < Ns; K += TC_THREADS) a.sigma[(size_t)Ia * Ns + K] = (double)row[K];
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

}  // namespace mbe

// Host side: shape checks, shared-memory size and the launch (one CTA per SM).
int mbe::large_ab_tc(cudaStream_t st, int sm_count, size_t smem_optin, int P, int Ns, int R, const int32_t *tab,
                     const float *V32, const float *c, double *sigma, int *err)
{
    TcArgs a;
    a.P = P;
    a.Ns = Ns;
    a.R = R;
    a.Np = (P + 15) / 16 * 16;
    a.Kp = R > 0 ? (R + 7) / 8 * 8 : 8;
    a.tab = tab;
    a.V32 = V32;
    a.c = c;
    a.sigma = sigma;
    a.err = err;
    // the gather holds up to 8 TC_MAXQ list entries per thread
    MBE_CHECK(a.Np >= 16 && a.Np <= TC_TMEM_COLS && a.Kp >= 8 && a.Kp <= 8 * TC_MAXQ, MBE_EUNSUPPORTED,
              "large CASCI: tensor-core sigma needs at most %d pairs and %d list entries (got %d, %d)", TC_TMEM_COLS,
              8 * TC_MAXQ, P, R);
    const TcSmem S = tc_smem(a.Np, a.Kp, Ns, R);
    MBE_CHECK(S.bytes + 1024 <= smem_optin, MBE_EUNSUPPORTED, "large CASCI: tensor-core sigma needs %u B shared memory",
              S.bytes);
    MBE_CU(cudaFuncSetAttribute(k_large_ab_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.bytes));
    const int grid = std::min(sm_count, Ns);
    k_large_ab_tc<<<grid, TC_THREADS, S.bytes, st>>>(a);
    MBE_CU(cudaGetLastError());
    return MBE_OK;
}
