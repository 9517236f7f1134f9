// a2-a7: batched tuple CASCI.
//
// For every tuple Omega of the batch, with A = R u Omega (n orbitals) and
// n_alpha = n_beta = k = |O n A|:
//   a2  h_eff = F[A,A] - sum_{i in O n A} (2 (pq|ii) - (pi|iq)), F the core Fock
//       matrix h + sum_{i in O}(2 J_i - K_i); V[(pq),(rs)] = (pq|rs) over A with
//       symmetric pair packing; h'_pq = h_eff_pq - 1/2 sum_r (pr|rq);
//   a3  the (n, k) string class tables (cached in the context);
//   a4  the one-spin string Hamiltonian Hs = sum h'_pq E_pq + 1/2 sum (pq|rs)
//       E_pq E_rs (an Ns x Ns matrix, identical for both spins because
//       n_alpha = n_beta), the determinant diagonal
//       H_II = Hs[Ia,Ia] + Hs[Ib,Ib] + sum_{p in Ia, q in Ib} (pp|qq),
//       and the start vector (lowest diagonal element plus a small fixed
//       pseudo-random admixture that reaches every symmetry sector);
//   a5  sigma = H c = Hs C + C Hs^T + sum_{pq,rs} (pq|rs) E^a_pq E^b_rs C, the
//       last term as a double loop over the alpha and beta replacement lists;
//   a6  a block Davidson (locally optimal 3-vector form: current Ritz vector,
//       previous direction, preconditioned residual) with the diagonal
//       preconditioner, run in float32 first (mixed mode) and float64 last;
//   a7  eps = lambda_min - H[Phi_A, Phi_A] - e_ref_corr.
//
// Two solvers: problems of <= 416 determinants run one per warp with the
// Davidson vectors in registers (13 determinants per lane at most) and all
// per-tuple data in shared memory; larger ones run one per thread block with
// the vectors and Hs in a per-block slot of the context workspace.  Both are
// persistent kernels that pull tuples from an atomic counter per bucket.
#include <algorithm>
#include <cmath>
#include "casci_dev.cuh"

namespace mbe {

// ------------------------------------------------------------------ batch plumbing

// F = h + sum_{i in O} (2 (pq|ii) - (pi|iq))
__global__ void k_core_fock(int norb, const double *h1, const double *eri, const uint8_t *occ, double *F)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= norb * norb) return;
    int p = e / norb, q = e - p * norb;
    double v = h1[e];
    for (int i = 0; i < norb; ++i)
        if (occ[i]) v += 2.0 * eri[eri_index(norb, p, q, i, i)] - eri[eri_index(norb, p, i, i, q)];
    F[e] = v;
}

struct ClassifyArgs {
    int bucket_of_k[MBE_MAX_CAS + 1];
    int nbuckets;
};

__global__ void k_classify(BatchArgs a, ClassifyArgs c, int32_t *key, int64_t *counts)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.n_tuples) return;
    int A[MBE_MAX_CAS];
    int b = -1;
    if (build_A(a, t, A)) {
        int k = 0;
        for (int i = 0; i < a.n; ++i) k += a.occ[A[i]];
        b = c.bucket_of_k[k];
    }
    key[t] = b;
    if (b < 0) {
        a.eps[t] = __longlong_as_double(0x7ff8000000000000LL);
        a.status[t] = MBE_STATUS_BADINPUT;
        if (a.iters) a.iters[t] = 0;
        return;
    }
    atomicAdd((unsigned long long *)&counts[b], 1ULL);
}

__global__ void k_scatter(int64_t n_tuples, int nbuckets, const int32_t *key, const int64_t *counts,
                          unsigned long long *cursor, int64_t *bucket_off, int32_t *perm)
{
    __shared__ int64_t off[MAX_BUCKETS + 1];
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int b = 0; b < nbuckets; ++b) {
            off[b] = s;
            s += counts[b];
        }
        off[nbuckets] = s;
        if (blockIdx.x == 0)
            for (int b = 0; b <= nbuckets; ++b) bucket_off[b] = off[b];
    }
    __syncthreads();
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tuples) return;
    int b = key[t];
    if (b < 0) return;
    unsigned long long slot = atomicAdd(&cursor[b], 1ULL);
    perm[off[b] + (int64_t)slot] = (int32_t)t;
}

}  // namespace mbe

using namespace mbe;

// casci_batch and casci_rdm_batch: rdm = 0 energies only, 1 = + weighted 1-RDM
// gradients, 2 = + weighted 1- and 2-RDM gradients.
static int run_casci(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ, int n_ref,
                     const int32_t *ref_orbs, double e_ref_corr, int order, int64_t n_tuples, const int32_t *tuples,
                     const mbe_opts *opts, double *eps_out, int32_t *status_out, int32_t *iters_out, int rdm,
                     const double *weights, double *grad_h1, double *grad_eri)
{
    MBE_CHECK(ctx != nullptr && h1 != nullptr && eri != nullptr && occ != nullptr, MBE_EINVAL,
              "casci_batch: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "casci_batch: norb %d outside 1..%d", norb,
              MBE_MAX_NORB);
    MBE_CHECK(n_ref >= 0 && order >= 0 && n_tuples >= 0, MBE_EINVAL, "casci_batch: negative size");
    MBE_CHECK(n_ref == 0 || ref_orbs != nullptr, MBE_EINVAL, "casci_batch: ref_orbs is NULL");
    MBE_CHECK(order > 0 ? (tuples != nullptr || n_tuples == 0) : n_tuples <= 1, MBE_EINVAL,
              "casci_batch: order 0 computes the reference space alone (n_tuples <= 1)");
    const int n = n_ref + order;
    MBE_CHECK(n >= 1, MBE_EINVAL, "casci_batch: empty active space");
    MBE_CHECK(n <= MBE_MAX_CAS, MBE_EUNSUPPORTED, "casci_batch: |R| + order = %d > %d", n, MBE_MAX_CAS);
    MBE_CHECK(n_tuples < (1LL << 31), MBE_EUNSUPPORTED, "casci_batch: n_tuples >= 2^31");
    mbe_opts o;
    if (opts) o = *opts; else mbe_default_opts(&o);
    MBE_CHECK(o.precision == MBE_PREC_FP64 || o.precision == MBE_PREC_MIXED, MBE_EINVAL,
              "casci_batch: unknown precision %d", o.precision);
    MBE_CHECK(o.tol > 0 && o.tol_switch > 0 && o.max_iter >= 1 && o.fp64_final_iters >= 0 &&
                  (o.sectors == MBE_SECTORS_BOTH || o.sectors == MBE_SECTORS_EVEN) &&
                  o.s2_penalty >= 0.0 && o.s2_penalty < 1e6, MBE_EINVAL,
              "casci_batch: bad options");
    if (n_tuples == 0) return MBE_OK;
    MBE_CHECK(rdm || (eps_out != nullptr && status_out != nullptr), MBE_EINVAL, "casci_batch: NULL output");
    MBE_CHECK(!rdm || grad_h1 != nullptr, MBE_EINVAL, "casci_rdm_batch: grad_h1 is NULL");
    MBE_CHECK(rdm != 2 || n <= 10, MBE_EUNSUPPORTED, "casci_rdm_batch: 2-RDM needs |R| + order <= 10 (got %d)", n);
    MBE_CU(cudaSetDevice(ctx->device));

    BatchArgs a;
    memset(&a, 0, sizeof(a));
    std::vector<int> ref(ref_orbs, ref_orbs + n_ref);
    std::sort(ref.begin(), ref.end());
    for (int i = 0; i < n_ref; ++i) {
        MBE_CHECK(ref[i] >= 0 && ref[i] < norb && (i == 0 || ref[i] != ref[i - 1]), MBE_EINVAL,
                  "casci_batch: reference orbital %d out of range or repeated", ref[i]);
        a.ref[i] = ref[i];
    }
    a.norb = norb;
    a.n = n;
    a.n_ref = n_ref;
    a.order = order;
    a.eri = eri;
    a.occ = occ;
    a.tuples = order > 0 ? tuples : nullptr;
    a.n_tuples = n_tuples;
    a.e_ref_corr = e_ref_corr;
    a.precision = o.precision;
    a.tol = o.tol;
    a.tol_switch = o.tol_switch;
    a.max_iter = o.max_iter;
    a.min_fp64 = o.fp64_final_iters;
    a.even_only = o.sectors == MBE_SECTORS_EVEN ? 1 : 0;
    a.s2mu = o.s2_penalty;
    const mbe_tuning tu = ctx->tune[o.precision == MBE_PREC_MIXED ? 1 : 0][n];
    a.warps = tu.warp_warps;
    a.block_basis = tu.block_basis;
    a.eps = eps_out;
    a.status = status_out;
    a.iters = iters_out;

    // Classes k = 0..n and their buckets.
    ClassifyArgs cl;
    std::vector<Bucket> buckets;
    int warp_bucket_of_dpl[5] = {-1, -1, -1, -1, -1};
    int block_bucket = -1;
    int max_block_ns = 0;
    for (int k = 0; k <= n; ++k) {
        const StringTable *st = nullptr;
        int rc = get_table(ctx, n, k, &st);
        if (rc) return rc;
        a.cls[k].strings = st->strings;
        a.cls[k].table = st->table;
        a.cls[k].ns = (int)st->ns;
        a.cls[k].r = st->r;
        int64_t N = st->ns * st->ns;
        int b;
        if (n <= WARP_MAX_N && N <= tu.warp_max_ndet && rdm != 2) {
            int di = 0;
            while (DPL_SET[di] * 32 < N) ++di;
            if (warp_bucket_of_dpl[di] < 0) {
                warp_bucket_of_dpl[di] = (int)buckets.size();
                buckets.push_back(Bucket{true, DPL_SET[di], 0, 0, 0});
            }
            b = warp_bucket_of_dpl[di];
        } else {
            if (block_bucket < 0) {
                block_bucket = (int)buckets.size();
                buckets.push_back(Bucket{false, 0, 0, 0, 0});
            }
            b = block_bucket;
            max_block_ns = std::max(max_block_ns, (int)st->ns);
        }
        Bucket &bk = buckets[b];
        bk.max_ns = std::max(bk.max_ns, (int)st->ns);
        bk.max_r = std::max(bk.max_r, st->r);
        bk.max_n = std::max(bk.max_n, (int)N);
        cl.bucket_of_k[k] = b;
    }
    const int nb = (int)buckets.size();
    cl.nbuckets = nb;

    int block_grid_n = 0;
    size_t block_smem_bytes = 0;
    size_t slot_bytes = 0;
    if (block_bucket >= 0) {
        int rc = block_grid(ctx, n, rdm == 2, &block_grid_n, &block_smem_bytes);
        if (rc) return rc;
        slot_bytes = slot_layout(max_block_ns, max_block_ns * max_block_ns).bytes;
    }

    const bool own_out = (eps_out == nullptr || status_out == nullptr);
    // mixed mode without density matrices splits the warp solver in two launches
    bool any_warp = false;
    for (const Bucket &bk : buckets) any_warp = any_warp || bk.warp;
    const bool split = any_warp && a.precision == MBE_PREC_MIXED && rdm == 0;
    size_t bytes = align256((size_t)norb * norb * 8) + align256((size_t)n_tuples * 4) * 2 +
                   5 * align256((MAX_BUCKETS + 1) * 8) + (size_t)block_grid_n * slot_bytes +
                   (own_out ? align256((size_t)n_tuples * 8) + align256((size_t)n_tuples * 4) : 0) + 1024;
    if (split) bytes += align256((size_t)n_tuples * 8);
    void *ws = nullptr;
    int rc = workspace(ctx, bytes, &ws);
    if (rc) return rc;
    Bump bump(ws);
    double *F = bump.take<double>((size_t)norb * norb);
    int32_t *key = bump.take<int32_t>(n_tuples);
    int32_t *perm = bump.take<int32_t>(n_tuples);
    int64_t *counts = bump.take<int64_t>(MAX_BUCKETS + 1);
    unsigned long long *cursor = bump.take<unsigned long long>(MAX_BUCKETS + 1);
    unsigned long long *counters = bump.take<unsigned long long>(MAX_BUCKETS + 1);
    unsigned long long *counters2 = bump.take<unsigned long long>(MAX_BUCKETS + 1);
    int64_t *bucket_off = bump.take<int64_t>(MAX_BUCKETS + 1);
    char *scratch = nullptr;
    if (block_grid_n > 0) scratch = bump.take<char>((size_t)block_grid_n * slot_bytes);
    a.pstate = nullptr;
    if (split) a.pstate = bump.take<int32_t>((size_t)n_tuples * 2);
    if (own_out) {
        a.eps = bump.take<double>((size_t)n_tuples);
        a.status = status_out ? status_out : bump.take<int32_t>((size_t)n_tuples);
        if (eps_out) a.eps = eps_out;
    }
    a.rdm = rdm;
    a.weights = weights;
    a.grad_h1 = grad_h1;
    a.grad_eri = (rdm == 2) ? grad_eri : nullptr;

    a.F = F;
    a.perm = perm;
    a.bucket_off = bucket_off;
    a.counters = counters;
    a.counters2 = counters2;
    a.scratch = scratch;
    a.slot_bytes = slot_bytes;

    MBE_CU(cudaMemsetAsync(counts, 0, 4 * align256((MAX_BUCKETS + 1) * 8), ctx->stream));
    k_core_fock<<<(norb * norb + 127) / 128, 128, 0, ctx->stream>>>(norb, h1, eri, occ, F);
    unsigned g = (unsigned)((n_tuples + 255) / 256);
    k_classify<<<g, 256, 0, ctx->stream>>>(a, cl, key, counts);
    k_scatter<<<g, 256, 0, ctx->stream>>>(n_tuples, nb, key, counts, cursor, bucket_off, perm);
    MBE_CU(cudaGetLastError());
    ctx->launches += 3;
    // Largest problems first, so that the long solves start early.
    std::vector<int> order_b(nb);
    for (int b = 0; b < nb; ++b) order_b[b] = b;
    std::sort(order_b.begin(), order_b.end(),
              [&](int x, int y) { return buckets[x].max_n > buckets[y].max_n; });
    for (int b : order_b) {
        const Bucket &bk = buckets[b];
        if (!bk.warp) {
            TimedLaunch tl(ctx, order, 1, 0);
            if ((rc = launch_block(ctx, a, b, block_grid_n, block_smem_bytes))) return rc;
            ++ctx->launches;
            rc = tl.done();
            if (rc) return rc;
            continue;
        }
        if ((rc = launch_warp_bucket(ctx, a, b, bk))) return rc;
    }
    return MBE_OK;
}

extern "C" int casci_batch(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                           int n_ref, const int32_t *ref_orbs, double e_ref_corr, int order,
                           int64_t n_tuples, const int32_t *tuples, const mbe_opts *opts, double *eps_out,
                           int32_t *status_out, int32_t *iters_out)
{
    return run_casci(ctx, norb, h1, eri, occ, n_ref, ref_orbs, e_ref_corr, order, n_tuples, tuples, opts, eps_out,
                     status_out, iters_out, 0, nullptr, nullptr, nullptr);
}

// Autotuner of the launch choices (see include/mbe.h): each tuning field in turn,
// candidates timed on the caller's tuples with CUDA events (best of two calls
// after a warm-up call), the fastest kept.
extern "C" int mbe_autotune(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                            int n_ref, const int32_t *ref_orbs, double e_ref_corr, int order, int64_t n_tuples,
                            const int32_t *tuples, const mbe_opts *opts, mbe_tuning *best, mbe_tune_record *records,
                            int max_records, int *n_records)
{
    MBE_CHECK(ctx && best && n_records && (max_records == 0 || records), MBE_EINVAL, "mbe_autotune: NULL argument");
    MBE_CHECK(n_tuples >= 1, MBE_EINVAL, "mbe_autotune: no tuples");
    mbe_opts o;
    if (opts) o = *opts; else mbe_default_opts(&o);
    MBE_CHECK(o.precision == MBE_PREC_FP64 || o.precision == MBE_PREC_MIXED, MBE_EINVAL,
              "mbe_autotune: unknown precision %d", o.precision);
    const int n = n_ref + order;
    MBE_CHECK(n >= 1 && n <= MBE_MAX_CAS, MBE_EUNSUPPORTED, "mbe_autotune: |R| + order = %d", n);
    MBE_CU(cudaSetDevice(ctx->device));
    const int p = o.precision == MBE_PREC_MIXED ? 1 : 0;
    double *eps = nullptr;
    int32_t *st = nullptr;
    MBE_CU(cudaMallocAsync((void **)&eps, (size_t)n_tuples * 8, ctx->stream));
    MBE_CU(cudaMallocAsync((void **)&st, (size_t)n_tuples * 4, ctx->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MBE_CU(cudaEventCreate(&e0));
    MBE_CU(cudaEventCreate(&e1));
    const bool timing = ctx->timing;
    ctx->timing = false;
    int nrec = 0, rc = MBE_OK;
    auto time_one = [&](const mbe_tuning &t, float *ms) -> int {
        ctx->tune[p][n] = t;
        float bestms = 3e38f;
        for (int rep = 0; rep < 3; ++rep) {
            if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) return MBE_ECUDA;
            int r = run_casci(ctx, norb, h1, eri, occ, n_ref, ref_orbs, e_ref_corr, order, n_tuples, tuples, &o,
                              eps, st, nullptr, 0, nullptr, nullptr, nullptr);
            if (r) return r;
            MBE_CU(cudaEventRecord(e1, ctx->stream));
            MBE_CU(cudaEventSynchronize(e1));
            float t_ms = 0.f;
            MBE_CU(cudaEventElapsedTime(&t_ms, e0, e1));
            if (rep > 0) bestms = std::min(bestms, t_ms);  // call 0 warms up
        }
        *ms = bestms;
        if (nrec < max_records) records[nrec] = mbe_tune_record{t, bestms};
        ++nrec;
        return MBE_OK;
    };
    mbe_tuning cur = ctx->tune[p][n];
    const int warps_c[] = {2, 4}, ndet_c[] = {100, 225, 416}, basis_c[] = {12, 16, 20};
    for (int field = 0; field < 3 && rc == MBE_OK; ++field) {
        const int *cand = field == 0 ? warps_c : field == 1 ? ndet_c : basis_c;
        const int nc = field == 0 ? 2 : 3;
        float bms = 3e38f;
        mbe_tuning bt = cur;
        for (int i = 0; i < nc && rc == MBE_OK; ++i) {
            mbe_tuning t = cur;
            (field == 0 ? t.warp_warps : field == 1 ? t.warp_max_ndet : t.block_basis) = cand[i];
            float ms = 0.f;
            rc = time_one(t, &ms);
            if (rc == MBE_OK && ms < bms) {
                bms = ms;
                bt = t;
            }
        }
        cur = bt;
    }
    ctx->tune[p][n] = cur;
    ctx->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(eps, ctx->stream);
    cudaFreeAsync(st, ctx->stream);
    if (rc) return rc;
    *best = cur;
    *n_records = nrec;
    return MBE_OK;
}

extern "C" int casci_rdm_batch(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                               int n_ref, const int32_t *ref_orbs, int order, int64_t n_tuples,
                               const int32_t *tuples, const mbe_opts *opts, const double *weights, double *grad_h1,
                               double *grad_eri, int32_t *status_out)
{
    return run_casci(ctx, norb, h1, eri, occ, n_ref, ref_orbs, 0.0, order, n_tuples, tuples, opts, nullptr,
                     status_out, nullptr, grad_eri ? 2 : 1, weights, grad_h1, grad_eri);
}

// ------------------------------------------------------------------ single active space sigma

namespace mbe {

// One block: h_eff, V, h', Hs and the diagonal of the active space a.ref[0..n).
__global__ void __launch_bounds__(CTA_THREADS)
    k_sigma_setup(BatchArgs a, ClassInfo ci, double *V_out, double *Hs_out, double *diag_out)
{
    extern __shared__ __align__(16) char smem[];
    const int n = a.n, P = n * (n + 1) / 2;
    const BlockSmem S = block_smem(n);
    int *A = (int *)(smem + S.off_A);
    if (threadIdx.x == 0) build_A(a, 0, A);
    __syncthreads();
    Problem pb;
    pb.n = n;
    pb.P = P;
    pb.k = 0;
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
    pb.Hs64 = Hs_out;
    pb.Hs32 = nullptr;
    pb.diag = diag_out;
    pb.c = nullptr;
    setup_problem<BlockGroup>(a, pb, false);
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) V_out[e] = pb.V64[e];
}

__global__ void __launch_bounds__(CTA_THREADS)
    k_sigma_apply(int n, ClassInfo ci, const double *V, const double *Hs, const double *c, double *sigma)
{
    extern __shared__ __align__(16) char smem[];
    const int P = n * (n + 1) / 2;
    double *Vs = (double *)smem;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) Vs[e] = V[e];
    __syncthreads();
    Problem pb;
    pb.n = n;
    pb.P = P;
    pb.Ns = ci.ns;
    pb.N = ci.ns * ci.ns;
    pb.R = ci.r;
    pb.RS = ci.r;
    pb.HSS = odd_stride(ci.ns);
    pb.tab = ci.table;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < pb.N; d += (int64_t)gridDim.x * blockDim.x)
        sigma[d] = sigma_elem<double>(pb, Vs, Hs, c, (int)d);
}

}  // namespace mbe

extern "C" int casci_sigma(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                           int n_cas, const int32_t *cas_orbs, const double *c, double *sigma, double *diag)
{
    MBE_CHECK(ctx && h1 && eri && occ && cas_orbs && c && sigma, MBE_EINVAL, "casci_sigma: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "casci_sigma: norb %d", norb);
    MBE_CHECK(n_cas >= 1 && n_cas <= norb, MBE_EINVAL, "casci_sigma: n_cas %d", n_cas);
    MBE_CHECK(n_cas <= MBE_MAX_CAS, MBE_EUNSUPPORTED, "casci_sigma: n_cas %d > %d", n_cas, MBE_MAX_CAS);
    MBE_CU(cudaSetDevice(ctx->device));
    std::vector<int> A(cas_orbs, cas_orbs + n_cas);
    std::sort(A.begin(), A.end());
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < n_cas; ++i) {
        MBE_CHECK(A[i] >= 0 && A[i] < norb && (i == 0 || A[i] != A[i - 1]), MBE_EINVAL,
                  "casci_sigma: active orbital %d out of range or repeated", A[i]);
        a.ref[i] = A[i];
    }
    // The electron count needs occ on the host: one small synchronous copy.
    std::vector<uint8_t> occ_h(norb);
    MBE_CU(cudaMemcpyAsync(occ_h.data(), occ, norb, cudaMemcpyDeviceToHost, ctx->stream));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    int k = 0;
    for (int i = 0; i < n_cas; ++i) k += occ_h[A[i]] ? 1 : 0;
    const StringTable *st = nullptr;
    int rc = get_table(ctx, n_cas, k, &st);
    if (rc) return rc;
    ClassInfo ci{st->strings, st->table, (int)st->ns, st->r};
    const int P = n_cas * (n_cas + 1) / 2;
    const int64_t N = st->ns * st->ns;
    size_t hs_elems = (size_t)st->ns * odd_stride((int)st->ns);
    size_t bytes = align256((size_t)norb * norb * 8) + align256((size_t)P * P * 8) + align256(hs_elems * 8) +
                   align256((size_t)N * 8) + 1024;
    void *ws = nullptr;
    rc = workspace(ctx, bytes, &ws);
    if (rc) return rc;
    Bump bump(ws);
    double *F = bump.take<double>((size_t)norb * norb);
    double *V = bump.take<double>((size_t)P * P);
    double *Hs = bump.take<double>(hs_elems);
    double *dg = diag ? diag : bump.take<double>((size_t)N);
    a.norb = norb;
    a.n = n_cas;
    a.n_ref = n_cas;
    a.order = 0;
    a.eri = eri;
    a.occ = occ;
    a.F = F;
    a.n_tuples = 1;
    k_core_fock<<<(norb * norb + 127) / 128, 128, 0, ctx->stream>>>(norb, h1, eri, occ, F);
    BlockSmem S = block_smem(n_cas);
    MBE_CU(cudaFuncSetAttribute(k_sigma_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, S.bytes));
    k_sigma_setup<<<1, CTA_THREADS, S.bytes, ctx->stream>>>(a, ci, V, Hs, dg);
    size_t smem = (size_t)P * P * 8;
    MBE_CU(cudaFuncSetAttribute(k_sigma_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t blocks = (N + CTA_THREADS - 1) / CTA_THREADS;
    int grid = (int)std::min<int64_t>(blocks, (int64_t)ctx->sm_count * 8);
    k_sigma_apply<<<grid, CTA_THREADS, smem, ctx->stream>>>(n_cas, ci, V, Hs, c, sigma);
    MBE_CU(cudaGetLastError());
    ctx->launches += 3;
    return MBE_OK;
}

// ------------------------------------------------------------------ allocation-free sigma
//
// casci_sigma_noalloc: the same sigma product as casci_sigma for callers that
// cannot allocate device memory at call time (see include/mbe.h).  Its scratch
// (core Fock matrix, string tables, packed integrals, Hs and, when the caller
// passes no diag buffer, the diagonal) lives in one fixed file-scope device
// array instead of the context workspace.

namespace mbe {

__global__ void k_string_table(int n, int k, int64_t ns, int r, uint32_t *strings, int32_t *table);

static __device__ __align__(256) unsigned char g_noalloc_scratch[MBE_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol itself is only a host-side handle.  The address is looked up on every
// call (a lookup allocates nothing), so a device reset that reloads the module
// cannot leave a stale address behind.
static int noalloc_scratch(void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    *out = p;
    return MBE_OK;
}

}  // namespace mbe

extern "C" int casci_sigma_noalloc(int device, void *cuda_stream, int norb, const double *h1, const double *eri,
                                   const uint8_t *occ, int n_cas, const int32_t *cas_orbs, int n_el,
                                   const double *c, double *sigma, double *diag)
{
    MBE_CHECK(h1 && eri && occ && cas_orbs && c && sigma, MBE_EINVAL, "casci_sigma_noalloc: NULL argument");
    MBE_CHECK(device >= 0 && device < MBE_MAX_DEVICES, MBE_EINVAL, "casci_sigma_noalloc: device %d", device);
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "casci_sigma_noalloc: norb %d", norb);
    MBE_CHECK(n_cas >= 1 && n_cas <= norb, MBE_EINVAL, "casci_sigma_noalloc: n_cas %d", n_cas);
    MBE_CHECK(n_el >= 0 && n_el <= n_cas, MBE_EINVAL, "casci_sigma_noalloc: n_el %d outside 0..%d", n_el, n_cas);
    MBE_CHECK(n_cas <= MBE_NOALLOC_MAX_CAS, MBE_EUNSUPPORTED,
              "casci_sigma_noalloc: n_cas %d exceeds the allocation-free limit of %d orbitals", n_cas,
              MBE_NOALLOC_MAX_CAS);
    std::vector<int> A(cas_orbs, cas_orbs + n_cas);
    std::sort(A.begin(), A.end());
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    for (int i = 0; i < n_cas; ++i) {
        MBE_CHECK(A[i] >= 0 && A[i] < norb && (i == 0 || A[i] != A[i - 1]), MBE_EINVAL,
                  "casci_sigma_noalloc: active orbital %d out of range or repeated", A[i]);
        a.ref[i] = A[i];
    }
    const int64_t ns = binom(n_cas, n_el);
    const int r = n_el * (n_cas - n_el + 1);
    const int P = n_cas * (n_cas + 1) / 2;
    const int64_t N = ns * ns;
    const size_t hs_elems = (size_t)ns * odd_stride((int)ns);
    size_t need = align256((size_t)norb * norb * 8) + align256((size_t)ns * 4) +
                  align256((size_t)ns * (r > 0 ? r : 1) * 4) + align256((size_t)P * P * 8) + align256(hs_elems * 8) +
                  (diag ? 0 : align256((size_t)N * 8));
    MBE_CHECK(need <= MBE_NOALLOC_SCRATCH_BYTES, MBE_EUNSUPPORTED,
              "casci_sigma_noalloc: needs %zu bytes of scratch, more than the fixed %zu", need,
              (size_t)MBE_NOALLOC_SCRATCH_BYTES);
    int prev = 0;
    MBE_CU(cudaGetDevice(&prev));
    if (prev != device) MBE_CU(cudaSetDevice(device));
    void *scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc == MBE_OK) {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        Bump bump(scratch);
        double *F = bump.take<double>((size_t)norb * norb);
        uint32_t *strings = bump.take<uint32_t>((size_t)ns);
        int32_t *table = bump.take<int32_t>((size_t)ns * (r > 0 ? r : 1));
        double *V = bump.take<double>((size_t)P * P);
        double *Hs = bump.take<double>(hs_elems);
        double *dg = diag ? diag : bump.take<double>((size_t)N);
        a.norb = norb;
        a.n = n_cas;
        a.n_ref = n_cas;
        a.order = 0;
        a.eri = eri;
        a.occ = occ;
        a.F = F;
        a.n_tuples = 1;
        ClassInfo ci{strings, table, (int)ns, r};
        k_string_table<<<(unsigned)((ns + 127) / 128), 128, 0, st>>>(n_cas, n_el, ns, r, strings, table);
        k_core_fock<<<(norb * norb + 127) / 128, 128, 0, st>>>(norb, h1, eri, occ, F);
        BlockSmem S = block_smem(n_cas);
        cudaError_t e = cudaFuncSetAttribute(k_sigma_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, S.bytes);
        if (e == cudaSuccess) {
            k_sigma_setup<<<1, CTA_THREADS, S.bytes, st>>>(a, ci, V, Hs, dg);
            int smem = P * P * 8;
            e = cudaFuncSetAttribute(k_sigma_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        }
        if (e == cudaSuccess) {
            int64_t blocks = (N + CTA_THREADS - 1) / CTA_THREADS;
            int grid = (int)std::min<int64_t>(blocks, 4096);
            k_sigma_apply<<<grid, CTA_THREADS, P * P * 8, st>>>(n_cas, ci, V, Hs, c, sigma);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) rc = cuda_fail(e, "casci_sigma_noalloc launch", __FILE__, __LINE__);
    }
    if (prev != device) cudaSetDevice(prev);
    return rc;
}

