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
// Data path per CTA (persistent over Ia, one CTA per SM, 16 warps):
//   * the B operand (N pairs x K list entries, signed V columns) is built once per
//     Ia in shared memory, hi and lo, by the whole CTA;
//   * the tiles of 128 beta strings are shared out to G groups of 16/G warps that
//     run independently (named barriers), each with its own A operand, TMEM
//     accumulator and mbarrier: with G = 2 one group gathers its next tile while
//     the other waits for its MMAs or scatters, so the gather latency, the tensor
//     pipe and the shared-memory scatter overlap.  G = 2 where two A operands fit
//     in shared memory (up to 14 orbitals), else G = 1;
//   * per tile: the A operand (128 x K, the gathered rows of c) is written to
//     shared memory, one thread issues the 3 x K/8 tcgen05.mma into the group's
//     TMEM accumulator and commits them to the group's mbarrier; after the wait the
//     group's warps copy the accumulator (tcgen05.ld) over its A operand (columns
//     XOR-swizzled by row so that the stores do not collide in one bank), and each
//     beta string scatters through its own list into the shared sigma row (shared
//     atomics);
//   * the row is written to sigma (float64) once per Ia.
// Operands use the K-major no-swizzle layout: 8-row x 16-byte core matrices,
// adjacent in K at LBO = 128 bytes, adjacent in M/N at SBO = 32 K bytes.
// Every wait is bounded: a wait that runs out sets *err, and the kernel still
// frees its TMEM before it returns.
#include <algorithm>

#include "common.cuh"

namespace mbe {

constexpr int TC_THREADS = 512;
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_M = 128;           // beta strings per tile (MMA M, TMEM lanes)
constexpr int TC_GROUP_COLS = 256;  // accumulator columns per group (>= N)
constexpr long long TC_SPIN = 1LL << 26;  // bounded mbarrier polls
constexpr int TC_MAXK = 128;        // list entries (K) the kernel accepts
constexpr int TC_CHUNK_Q = 8;       // x-quads a thread gathers before its stores

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

// One 16-column TMEM load of this warp's 32 lanes, then the wait.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Named barrier of one group (ids 1.. ; id 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g, int nthreads)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "r"(nthreads) : "memory");
}

struct TcArgs {
    int P, Ns, R, Np, Kp, G;
    const int32_t *tab;  // [Ns][R] replacement lists
    const float *V32;    // [P][P]
    const float *c;      // [Ns][Ns] float32 coefficients
    double *sigma;       // [Ns][Ns], written
    int *err;            // set to 1 when a wait runs out
};

struct TcSmem {
    uint32_t off_bhi, off_blo, off_a[2], off_T[2], off_row, off_jx, off_bar, off_tmem, off_flag, bytes;
    int Ts;    // row stride (floats) of the staged accumulator tile
    int swz;   // 15: columns XOR-swizzled by (row & 15) (even stride); 0: none (odd stride)
};

// G groups: B (hi, lo) shared; per group an A operand (hi, lo), over which the
// accumulator tile [TC_M][Ts] is staged when it fits there.
__host__ __device__ inline TcSmem tc_smem(int Np, int Kp, int Ns, int R, int G)
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
    // an odd stride Np + 1 spreads a warp's column stores over the banks; where only
    // Np fits over A, the XOR swizzle of the column (within its 16-column block,
    // Np being a multiple of 16) does it instead
    const bool over_a = Np <= 2 * Kp;
    S.Ts = (Np + 1 <= 2 * Kp || !over_a) ? Np + 1 : Np;
    S.swz = (S.Ts & 1) ? 0 : 15;
    for (int g = 0; g < 2; ++g) {
        S.off_a[g] = S.off_T[g] = 0;
        if (g >= G) continue;
        S.off_a[g] = take((uint32_t)2 * TC_M * Kp * 4, 1024);
        S.off_T[g] = over_a ? S.off_a[g] : take((uint32_t)TC_M * S.Ts * 4, 16);
    }
    S.off_row = take((uint32_t)Ns * 4, 16);
    S.off_jx = take((uint32_t)R * 4, 16);
    S.off_bar = take(16, 8);
    S.off_tmem = take(4, 4);
    S.off_flag = take(4 * 4, 4);
    S.bytes = (o + 127) / 128 * 128;
    return S;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_large_ab_tc(TcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int G = a.G;
    const TcSmem S = tc_smem(a.Np, a.Kp, a.Ns, a.R, G);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int P = a.P, Ns = a.Ns, R = a.R, Np = a.Np, Kp = a.Kp;
    const int W = TC_WARPS / G;                 // warps per group
    const int g = warp / W, wg = warp - g * W;  // group, warp within the group
    const int gthreads = 32 * W, tig = tid - g * gthreads;
    const int TPR = W / 4;                      // threads per beta string of a tile
    unsigned char *bhi = smem + S.off_bhi, *blo = smem + S.off_blo;
    unsigned char *ahi = smem + S.off_a[g], *alo = ahi + (size_t)TC_M * Kp * 4;
    float *T = (float *)(smem + S.off_T[g]);
    float *row = (float *)(smem + S.off_row);
    int *jx = (int *)(smem + S.off_jx);
    const uint32_t bar = smem_u32(smem + S.off_bar) + 8u * (uint32_t)g;
    uint32_t *tslot = (uint32_t *)(smem + S.off_tmem);
    int *flag = (int *)(smem + S.off_flag);  // [0]: a wait ran out; [1 + g]: group g's last wait succeeded
    const uint32_t ncols = (uint32_t)(TC_GROUP_COLS * G);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int i = 0; i < G; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(smem + S.off_bar) + 8u * i));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        flag[0] = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot + (uint32_t)(g * TC_GROUP_COLS);
    const uint32_t idesc = tf32_idesc(TC_M, Np);
    const uint32_t lbo = 128, sbo = 32u * (uint32_t)Kp;
    const int ntiles = (Ns + TC_M - 1) / TC_M, nq = Kp / 4;
    uint32_t phase = 0;

    for (int Ia = blockIdx.x; Ia < Ns; Ia += gridDim.x) {
        const int32_t *ta = a.tab + (size_t)Ia * R;
        for (int x = tid; x < R; x += TC_THREADS) jx[x] = entry_J(ta[x]);
        for (int i = tid; i < Ns; i += TC_THREADS) row[i] = 0.f;
        // B operand: B[p][x] = s_x V[p_x][p] (zero beyond P and R), hi and lo;
        // consecutive threads take consecutive pairs p (coalesced V loads, and
        // float4 stores that fill whole 128-byte rows of banks)
        for (int i = tid; i < Np * nq; i += TC_THREADS) {
            const int x0 = (i / Np) * 4, p = i - (i / Np) * Np;
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
        for (int tile = g; tile < ntiles; tile += G) {
            const int Jb0 = tile * TC_M;
            const int jb = tig & (TC_M - 1), q0 = tig >> 7, Jb = Jb0 + jb;
            // A operand: A[jb][x] = c[J_x][Jb0 + jb] (zero beyond Ns and R), hi and lo;
            // a thread issues the loads of TC_CHUNK_Q quads before their stores
            for (int qb = q0; qb < nq; qb += TC_CHUNK_Q * TPR) {
                float v[TC_CHUNK_Q][4];
#pragma unroll
                for (int i = 0; i < TC_CHUNK_Q; ++i) {
                    const int q = qb + i * TPR;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int x = 4 * q + j;
                        v[i][j] = (q < nq && Jb < Ns && x < R) ? __ldg(a.c + (size_t)jx[x] * Ns + Jb) : 0.f;
                    }
                }
#pragma unroll
                for (int i = 0; i < TC_CHUNK_Q; ++i) {
                    const int q = qb + i * TPR;
                    if (q < nq) {
                        float4 h, l;
                        split_tf32(v[i][0], h.x, l.x);
                        split_tf32(v[i][1], h.y, l.y);
                        split_tf32(v[i][2], h.z, l.z);
                        split_tf32(v[i][3], h.w, l.w);
                        *(float4 *)(ahi + kmajor_off(jb, 4 * q, Kp)) = h;
                        *(float4 *)(alo + kmajor_off(jb, 4 * q, Kp)) = l;
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            group_sync(g, gthreads);
            if (tig == 0) {
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
                // one thread waits (bounded) and hands the outcome to its group; after a
                // wait that ran out it waits once more (bounded) for the MMAs in flight
                // before the kernel goes on to free the accumulator
                bool ok = mbar_wait(bar, phase);
                if (!ok) {
                    atomicExch(a.err, 1);
                    atomicExch(&flag[0], 1);
                    mbar_wait(bar, phase);
                }
                flag[1 + g] = ok ? 1 : 0;
                phase ^= 1u;
                asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            }
            group_sync(g, gthreads);
            if (!flag[1 + g]) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // epilogue 1: the accumulator tile to T[jb][col ^ swz(jb)] over the A
            // operand (free once the MMAs completed); warp wg reads TMEM lanes
            // 32 (warp % 4) .. + 31 (the lanes its position in the warpgroup may
            // access), the columns split between the W / 4 warps that share them
            {
                const int jr = (warp & 3) * 32 + lane;
                const int sw = S.swz ? (jr & S.swz) : 0;
                const int nch = Np / 16, part = wg >> 2;
                const int c0 = part * nch / TPR, c1 = (part + 1) * nch / TPR;
                const uint32_t tbase = tmem + ((uint32_t)((warp & 3) * 32) << 16);
                float *Tr = T + jr * S.Ts;
                for (int ch = c0; ch < c1; ++ch) {
                    float v[16];
                    tmem_ld16(tbase + (uint32_t)(ch * 16), v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) Tr[ch * 16 + (i ^ sw)] = v[i];
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            group_sync(g, gthreads);
            // epilogue 2: each beta string Jb of the tile walks its own list, E_p|Jb> =
            // s|K>: sigma[Ia][K] += s T[Jb][p] (shared atomics); TPR threads per string
            if (Jb < Ns) {
                const int32_t *tb = a.tab + (size_t)Jb * R;
                const float *Trow = T + jb * S.Ts;
                const int sw = S.swz ? (jb & S.swz) : 0;
                for (int y = q0; y < R; y += TPR) {
                    const int e = __ldg(tb + y);
                    const float v = Trow[entry_pair(e) ^ sw];
                    atomicAdd(&row[entry_J(e)], entry_neg(e) ? -v : v);
                }
            }
            group_sync(g, gthreads);
        }
        __syncthreads();
        const bool failed = flag[0] != 0;
        if (!failed)
            for (int K = tid; K < Ns; K += TC_THREADS) a.sigma[(size_t)Ia * Ns + K] = (double)row[K];
        __syncthreads();
        if (failed) break;
    }
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(*tslot), "r"(ncols));
}

}  // namespace mbe

// Host side: shape checks, the group count, shared-memory size and the launch
// (one CTA per SM).
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
    MBE_CHECK(a.Np >= 16 && a.Np <= TC_GROUP_COLS && a.Kp >= 8 && a.Kp <= TC_MAXK, MBE_EUNSUPPORTED,
              "large CASCI: tensor-core sigma needs at most %d pairs and %d list entries (got %d, %d)", TC_GROUP_COLS,
              TC_MAXK, P, R);
    a.G = 2;
    TcSmem S = tc_smem(a.Np, a.Kp, Ns, R, a.G);
    if (S.bytes + 1024 > smem_optin) {
        a.G = 1;
        S = tc_smem(a.Np, a.Kp, Ns, R, a.G);
    }
    MBE_CHECK(S.bytes + 1024 <= smem_optin, MBE_EUNSUPPORTED, "large CASCI: tensor-core sigma needs %u B shared memory",
              S.bytes);
    MBE_CU(cudaFuncSetAttribute(k_large_ab_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.bytes));
    const int grid = std::min(sm_count, Ns);
    k_large_ab_tc<<<grid, TC_THREADS, S.bytes, st>>>(a);
    MBE_CU(cudaGetLastError());
    return MBE_OK;
}
