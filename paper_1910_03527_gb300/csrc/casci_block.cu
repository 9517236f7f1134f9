// a5-a6, the block solver: one tuple CASCI of more than the warp solver's
// determinants per thread block, vectors in a per-block slot of the workspace.
#include "casci_dev.cuh"

namespace mbe {

__global__ void __launch_bounds__(CTA_THREADS, 2) k_casci_block(BatchArgs a, int bucket)
{
    extern __shared__ __align__(16) char smem[];
    const int n = a.n, P = n * (n + 1) / 2;
    const BlockSmem S = block_smem(n, a.rdm == 2);
    int *A = (int *)(smem + S.off_A);
    double *red = (double *)(smem + S.off_red);
    __shared__ unsigned long long s_pos;
    char *slot = a.scratch + (size_t)blockIdx.x * a.slot_bytes;
    const int64_t begin = a.bucket_off[bucket];
    const int64_t cnt = a.bucket_off[bucket + 1] - begin;
    for (;;) {
        if (threadIdx.x == 0) s_pos = atomicAdd(&a.counters[bucket], 1ULL);
        __syncthreads();
        unsigned long long pos = s_pos;
        __syncthreads();
        if ((int64_t)pos >= cnt) break;
        const int64_t t = a.perm[begin + (int64_t)pos];
        if (threadIdx.x == 0) build_A(a, t, A);
        __syncthreads();
        int k = 0;
        for (int i = 0; i < n; ++i) k += a.occ[A[i]];
        const ClassInfo ci = a.cls[k];
        Problem pb;
        pb.n = n;
        pb.P = P;
        pb.k = k;
        pb.Ns = ci.ns;
        pb.N = ci.ns * ci.ns;
        pb.R = ci.r;
        pb.RS = ci.r;
        pb.HSS = odd_stride(ci.ns);
        pb.str = ci.strings;
        pb.tab = ci.table;
        pb.A = A;
        pb.pp = (const short *)(smem + S.off_pp);
        pb.h = (double *)(smem + S.off_h);
        pb.hp = (double *)(smem + S.off_hp);
        pb.V64 = (double *)(smem + S.off_V64);
        pb.V32 = (float *)(smem + S.off_V32);
        SlotLayout L = slot_layout(ci.ns, pb.N);
        pb.Hs64 = (double *)(slot + L.off_Hs64);
        pb.Hs32 = (float *)(slot + L.off_Hs32);
        pb.diag = (double *)(slot + L.off_diag);
        pb.c = nullptr;
        const bool mixed = a.precision == MBE_PREC_MIXED;
        pb.s2mu = a.s2mu;
        setup_problem<BlockGroup>(a, pb, mixed);
        uint32_t mphi = 0;
        for (int i = 0; i < n; ++i)
            if (a.occ[A[i]]) mphi |= 1u << i;
        int iphi = string_rank(mphi);
        double ephi = pb.diag[iphi * pb.Ns + iphi];
        if (pb.N == 1) {
            if (threadIdx.x == 0) store_result(a, t, pb.diag[0] - ephi - a.e_ref_corr, MBE_STATUS_OK, 0, 0);
            __syncthreads();
            continue;
        }
        // start vectors: the lowest diagonal element (ties -> lowest index), and for
        // the P = -1 sector the lowest one with Ia != Ib
        double best = 1e300, best_o = 1e300;
        int bi = 0x7fffffff, bj = 0x7fffffff;
        for (int d = threadIdx.x; d < pb.N; d += blockDim.x) {
            const double v = pb.diag[d];
            if (v < best || (v == best && d < bi)) {
                best = v;
                bi = d;
            }
            const int ia = d / pb.Ns;
            if (ia != d - ia * pb.Ns && (v < best_o || (v == best_o && d < bj))) {
                best_o = v;
                bj = d;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ov = __shfl_xor_sync(FULL, best, o);
            int oi = __shfl_xor_sync(FULL, bi, o);
            if (ov < best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
            ov = __shfl_xor_sync(FULL, best_o, o);
            oi = __shfl_xor_sync(FULL, bj, o);
            if (ov < best_o || (ov == best_o && oi < bj)) {
                best_o = ov;
                bj = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            red[threadIdx.x >> 5] = best;
            red[32 + (threadIdx.x >> 5)] = best_o;
            ((int *)(red + 64))[threadIdx.x >> 5] = bi;
            ((int *)(red + 64))[32 + (threadIdx.x >> 5)] = bj;
        }
        __syncthreads();
        best = red[0];
        best_o = red[32];
        bi = ((int *)(red + 64))[0];
        bj = ((int *)(red + 64))[32];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            double ov = red[w];
            int oi = ((int *)(red + 64))[w];
            if (ov < best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
            ov = red[32 + w];
            oi = ((int *)(red + 64))[32 + w];
            if (ov < best_o || (ov == best_o && oi < bj)) {
                best_o = ov;
                bj = oi;
            }
        }
        __syncthreads();
        double *x64 = (double *)(slot + L.off_x);
        double *x2 = (double *)(slot + L.off_x2);
        double lam = 0.0;
        int status = MBE_STATUS_OK, n64 = 0, n32 = 0;
        bool degen = false;
        // one copy of the sector's Davidson: two inlined copies, both hot on an SM,
        // overflow the instruction cache and slow every phase of every warp
#pragma unroll 1
        for (int sector = 0; sector < 2; ++sector) {
            if (sector == 1 && (pb.Ns < 2 || status != MBE_STATUS_OK || a.even_only)) break;
            const SectorGuess sg{sector == 0 ? bi : bj, sector == 0 ? 1 : -1};
            if (sector == 1 && a.rdm)
                for (int d = threadIdx.x; d < pb.N; d += blockDim.x) x2[d] = x64[d];
            pb.sector = sg.sgn;
            for (int d = threadIdx.x; d < pb.N; d += blockDim.x) x64[d] = sector_guess(d, pb.Ns, sg);
            __syncthreads();
            bool lose = false, refined = false;
            if (mixed) {
                float *x32 = (float *)(slot + L.off_x);
                // narrow x in place (float view of the same region), bottom up
                for (int base = 0; base < pb.N; base += blockDim.x) {
                    int d = base + threadIdx.x;
                    double v = (d < pb.N) ? x64[d] : 0.0;
                    __syncthreads();
                    if (d < pb.N) x32[d] = (float)v;
                    __syncthreads();
                }
                // the second sector: a pass to SECTOR_TOL, then one to tol_switch if undecided
                PhaseOut o32;
                for (int pass = 0; pass < 1 + sector; ++pass) {
                    const double tl = (sector == 0 || pass == 1) ? a.tol_switch : SECTOR_TOL;
                    o32 = davidson_block<float>(pb, (float *)(slot + L.off_V), (float *)(slot + L.off_W), L.vec / 4,
                                                x32, (float *)(slot + L.off_hx), (float *)(slot + L.off_t), smem, S,
                                                tl, 0, a.max_iter, BLOCK_STALL, 0.0, false, a.block_basis);
                    n32 += o32.nsig;
                    if (sector == 1)
                        lose = o32.status == MBE_STATUS_NONFINITE ||
                               sector_loses(o32.lambda, o32.rnorm, lam, a.tol_switch);
                    if (lose || o32.status == MBE_STATUS_NONFINITE) break;
                }
                const bool finite = o32.status != MBE_STATUS_NONFINITE;
                double *x0 = (double *)(slot + L.off_x0);
                if (!lose && finite) {
                    // Anchored refinement (struct Anchor): a float64 sigma of the float64
                    // anchor x0, then the float32 Davidson on H - theta0 with x0 as its
                    // first basis vector; x0 <- x0 + d after each pass, re-anchoring while
                    // the residual stays above tol.
                    for (int d = threadIdx.x; d < pb.N; d += blockDim.x) x0[d] = (double)x32[d];
                    __syncthreads();
                    float *V0 = (float *)(slot + L.off_V), *W0 = (float *)(slot + L.off_W);
                    double *s0 = (double *)(slot + L.off_hx);
                    bool done = false, bad = false;
                    double lam_s = 0.0;
                    for (int anc = 0; anc < BLOCK_ANCHORS && !done && !bad; ++anc) {
                        sigma_block<double>(pb, pb.V64, pb.Hs64, x0, s0);
                        ++n64;
                        double q[KRED];
                        q[0] = q[1] = 0.0;
                        for (int d = threadIdx.x; d < pb.N; d += blockDim.x) {
                            q[0] += x0[d] * s0[d];
                            q[1] += x0[d] * x0[d];
                        }
                        block_sum_n<double>(q, 2, red);
                        const double th = q[0] / q[1], inv = 1.0 / sqrt(q[1]);
                        for (int d = threadIdx.x; d < pb.N; d += blockDim.x) {
                            V0[d] = (float)(x0[d] * inv);
                            W0[d] = (float)((s0[d] - th * x0[d]) * inv);
                        }
                        __syncthreads();
                        PhaseOut o = davidson_block<float>(pb, V0, W0, L.vec / 4, x32, (float *)(slot + L.off_hx),
                                                           (float *)(slot + L.off_t), smem, S, a.tol, a.min_fp64,
                                                           a.max_iter, BLOCK_ANCHOR_STALL, th, true, a.block_basis);
                        n32 += o.nsig;
                        lam_s = th + o.lambda;
                        bad = o.status == MBE_STATUS_NONFINITE;
                        done = !bad && o.rnorm <= a.tol && o.dnorm <= MIX_DMAX;
                        if (!bad)
                            for (int d = threadIdx.x; d < pb.N; d += blockDim.x) x0[d] = x0[d] * inv + (double)x32[d];
                        __syncthreads();
                    }
                    // the refined vector (or the start of the float64 fallback) as x64
                    for (int d = threadIdx.x; d < pb.N; d += blockDim.x)
                        x64[d] = bad ? sector_guess(d, pb.Ns, sg) : x0[d];
                    __syncthreads();
                    if (done) {
                        refined = true;
                        if (sector == 1) degen = status == MBE_STATUS_OK && fabs(lam_s - lam) <= DEGEN_TOL;
                        if (sector == 0) {
                            lam = lam_s;
                            status = MBE_STATUS_OK;
                        } else if (lam_s < lam) {
                            lam = lam_s;
                            status = MBE_STATUS_OK;
                        } else {
                            lose = true;
                        }
                    }
                } else {
                    for (int d = threadIdx.x; d < pb.N; d += blockDim.x)
                        x64[d] = finite ? (double)x32[d] : sector_guess(d, pb.Ns, sg);
                    __syncthreads();
                }
            } else if (sector == 1) {
                PhaseOut o1 = davidson_block<double>(pb, (double *)(slot + L.off_V), (double *)(slot + L.off_W),
                                                     L.vec / 8, x64, (double *)(slot + L.off_hx),
                                                     (double *)(slot + L.off_t), smem, S, SECTOR_TOL, 0,
                                                     a.max_iter, BLOCK_STALL, 0.0, false, a.block_basis);
                n64 += o1.nsig;
                lose = o1.status == MBE_STATUS_NONFINITE || sector_loses(o1.lambda, o1.rnorm, lam, 0.0);
            }
            if (!lose && !refined) {
                PhaseOut o64 = davidson_block<double>(pb, (double *)(slot + L.off_V), (double *)(slot + L.off_W),
                                                      L.vec / 8, x64, (double *)(slot + L.off_hx),
                                                      (double *)(slot + L.off_t), smem, S, a.tol,
                                                      mixed ? a.min_fp64 : 0, a.max_iter, 0, 0.0, false, a.block_basis);
                n64 += o64.nsig;
                if (sector == 0) {
                    lam = o64.lambda;
                    status = o64.status;
                } else {
                    degen = o64.status == MBE_STATUS_OK && status == MBE_STATUS_OK && fabs(o64.lambda - lam) <= DEGEN_TOL;
                    lose = o64.status == MBE_STATUS_NONFINITE || !(o64.lambda < lam);
                    if (!lose) {
                        lam = o64.lambda;
                        status = o64.status;
                    }
                }
            }
            if (lose && a.rdm) {
                __syncthreads();
                for (int d = threadIdx.x; d < pb.N; d += blockDim.x) x64[d] = x2[d];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            double e = status == MBE_STATUS_NONFINITE ? __longlong_as_double(0x7ff8000000000000LL)
                                                      : lam - ephi - a.e_ref_corr;
            store_result(a, t, e, with_degeneracy(status, degen), n64, n32);
        }
        __syncthreads();
        if (a.rdm) {
            double *g1 = (double *)(smem + S.off_g1);
            double *g2 = (a.rdm == 2) ? (double *)(smem + S.off_g2) : nullptr;
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) g1[e] = 0.0;
            if (g2)
                for (int e = threadIdx.x; e < n * n * n * n; e += blockDim.x) g2[e] = 0.0;
            __syncthreads();
            rdm_accumulate<BlockGroup>(pb, x64, g1, g2);
            __syncthreads();
            rdm_flush<BlockGroup>(a, pb, g1, g2, a.weights ? a.weights[t] : 1.0);
            __syncthreads();
        }
    }
}

int block_grid(mbe_ctx *ctx, int n, bool two_body, int *grid, size_t *smem)
{
    BlockSmem S = block_smem(n, two_body);
    *smem = (size_t)S.bytes;
    MBE_CHECK(*smem <= ctx->smem_optin, MBE_EUNSUPPORTED, "casci_batch: block solver needs %zu B shared memory",
              *smem);
    MBE_CU(cudaFuncSetAttribute(k_casci_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem));
    int per_sm = 0;
    MBE_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_casci_block, CTA_THREADS, *smem));
    if (per_sm < 1) per_sm = 1;
    *grid = ctx->sm_count * per_sm;
    return MBE_OK;
}

int launch_block(mbe_ctx *ctx, const BatchArgs &a, int b, int grid, size_t smem)
{
    k_casci_block<<<grid, CTA_THREADS, smem, ctx->stream>>>(a, b);
    MBE_CU(cudaGetLastError());
    return MBE_OK;
}

}  // namespace mbe
