// Tuple CASCI for the large active spaces of Type-1 and Type-2 expansions
// (Sec. 1, Fig. 1): a reference space of every virtual (Type-1) or every
// occupied orbital (Type-2) makes R u Omega large at every order, up to the
// sizes of a single big CASCI.  The tuples of one order are split on the host:
// the ones the batched solvers take (at most MBE_MAX_CAS orbitals, at most
// `large_ndet` determinants) go to casci_batch in one call; each other tuple is
// solved by casci_solve with the whole GPU.  Both write eps = E_CAS(R u Omega) -
// E_Phi - E_ref,corr (Eq. 1), so the routed results are interchangeable.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace mbe {

// Scatters the results of the batched sub-call to their tuples' rows.
__global__ void k_route_scatter(int64_t n, const int64_t *rows, const double *eps, const int32_t *status,
                                const int32_t *iters, double *eps_out, int32_t *status_out, int32_t *iters_out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t r = rows[i];
    eps_out[r] = eps[i];
    status_out[r] = status[i];
    if (iters_out) iters_out[r] = iters[i];
}

// The one-determinant and malformed tuples of a call, in one launch: an active
// space whose only determinant is Phi_A has lambda = <Phi_A|H_A|Phi_A>, so
// eps = -E_ref,corr; a malformed tuple gets NaN and MBE_STATUS_BADINPUT.
__global__ void k_route_direct(int64_t n, const int64_t *rows, const int32_t *status, double e_ref_corr,
                               double *eps_out, int32_t *status_out, int32_t *iters_out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t r = rows[i];
    eps_out[r] = status[i] == MBE_STATUS_BADINPUT ? (double)NAN : -e_ref_corr;
    status_out[r] = status[i];
    if (iters_out) iters_out[r] = 0;
}

// Whole-GPU solves of up to ROUTE_CONCURRENT_NDET determinants run on up to
// ROUTE_WORKERS worker contexts at once, one host thread and one stream each: a
// solve of that size leaves most of the GPU idle while its host loop waits for
// the Davidson scalars of each iteration, and the other solves fill the gaps.
// Larger active spaces keep the GPU busy alone and run one at a time on the
// caller's context.
constexpr int ROUTE_WORKERS = 4;
constexpr int64_t ROUTE_CONCURRENT_NDET = 4000000;

// Makes sure the context has k worker contexts.
static int route_workers(mbe_ctx *ctx, int k)
{
    while ((int)ctx->workers.size() < k) {
        cudaStream_t s = nullptr;
        MBE_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        mbe_ctx *w = nullptr;
        const int rc = mbe_ctx_create(&w, ctx->device, s);
        if (rc) {
            cudaStreamDestroy(s);
            return rc;
        }
        ctx->workers.push_back(w);
        ctx->worker_streams.push_back(s);
    }
    return MBE_OK;
}

// Stream-ordered device buffers released when the call returns, on every path.
struct RouteBuffers {
    cudaStream_t stream;
    std::vector<void *> ptrs;
    explicit RouteBuffers(cudaStream_t s) : stream(s) {}
    ~RouteBuffers()
    {
        for (void *p : ptrs) cudaFreeAsync(p, stream);
    }
    cudaError_t get(size_t bytes, void **out)
    {
        cudaError_t e = cudaMallocAsync(out, std::max<size_t>(bytes, 256), stream);
        if (e == cudaSuccess) ptrs.push_back(*out);
        return e;
    }
};

}  // namespace mbe

using namespace mbe;

extern "C" int casci_batch_routed(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                                  int n_ref, const int32_t *ref_orbs, double e_ref_corr, int order,
                                  int64_t n_tuples, const int32_t *tuples, const mbe_opts *opts,
                                  int64_t large_ndet, double *eps_out, int32_t *status_out, int32_t *iters_out)
{
    MBE_CHECK(ctx && h1 && eri && occ && eps_out && status_out, MBE_EINVAL, "casci_batch_routed: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "casci_batch_routed: norb %d outside 1..%d", norb,
              MBE_MAX_NORB);
    MBE_CHECK(n_ref >= 0 && n_ref <= norb && (n_ref == 0 || ref_orbs != nullptr), MBE_EINVAL,
              "casci_batch_routed: bad reference space");
    MBE_CHECK(order >= 0 && order <= MBE_MAX_ORDER, MBE_EINVAL, "casci_batch_routed: order %d", order);
    MBE_CHECK(n_ref + order >= 1 && n_ref + order <= MBE_MAX_LARGE_CAS, MBE_EUNSUPPORTED,
              "casci_batch_routed: |R| + order = %d outside 1..%d", n_ref + order, MBE_MAX_LARGE_CAS);
    MBE_CHECK(order > 0 || n_tuples == 1, MBE_EINVAL, "casci_batch_routed: order 0 takes exactly one tuple");
    MBE_CHECK(n_tuples >= 0 && (order == 0 || n_tuples == 0 || tuples != nullptr), MBE_EINVAL,
              "casci_batch_routed: bad tuple list");
    MBE_CHECK(std::isfinite(e_ref_corr), MBE_EINVAL, "casci_batch_routed: e_ref_corr is not finite");
    for (int i = 0; i < n_ref; ++i)
        MBE_CHECK(ref_orbs[i] >= 0 && ref_orbs[i] < norb && (i == 0 || ref_orbs[i] > ref_orbs[i - 1]), MBE_EINVAL,
                  "casci_batch_routed: reference orbitals must be ascending and in 0..%d", norb - 1);
    const int n_cas = n_ref + order;
    if (n_tuples == 0) return MBE_OK;
    // Every tuple fits the batched solvers and no size limit was asked for: one call.
    if (n_cas <= MBE_MAX_CAS && large_ndet <= 0)
        return casci_batch(ctx, norb, h1, eri, occ, n_ref, ref_orbs, e_ref_corr, order, n_tuples, tuples, opts,
                           eps_out, status_out, iters_out);

    MBE_CU(cudaSetDevice(ctx->device));
    std::vector<uint8_t> occ_h(norb);
    std::vector<int32_t> tup_h((size_t)n_tuples * order);
    MBE_CU(cudaMemcpyAsync(occ_h.data(), occ, norb, cudaMemcpyDeviceToHost, ctx->stream));
    if (order > 0)
        MBE_CU(cudaMemcpyAsync(tup_h.data(), tuples, tup_h.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                               ctx->stream));
    MBE_CU(cudaStreamSynchronize(ctx->stream));

    // Classify: batched (B), one whole-GPU solve each (L), or a one-determinant
    // or malformed active space written directly (D).
    std::vector<int64_t> rows_b, rows_l, rows_d, ndet_l;
    std::vector<int32_t> tup_b;
    std::vector<uint8_t> in_ref(norb, 0);
    for (int i = 0; i < n_ref; ++i) in_ref[ref_orbs[i]] = 1;
    for (int64_t t = 0; t < n_tuples; ++t) {
        const int32_t *tp = tup_h.data() + (size_t)t * order;
        bool ok = true;
        int k = 0;
        for (int i = 0; i < order; ++i) {
            ok = ok && tp[i] >= 0 && tp[i] < norb && !in_ref[tp[i]] && (i == 0 || tp[i] > tp[i - 1]);
            if (ok) k += occ_h[tp[i]];
        }
        for (int i = 0; i < n_ref; ++i) k += occ_h[ref_orbs[i]];
        const int64_t ndet = ok ? binom(n_cas, k) * binom(n_cas, k) : 0;
        const bool batched = n_cas <= MBE_MAX_CAS && (large_ndet <= 0 || ndet <= large_ndet || !ok);
        if (batched) {
            rows_b.push_back(t);
            tup_b.insert(tup_b.end(), tp, tp + order);
        } else if (!ok || ndet == 1) {
            rows_d.push_back(t);
        } else {
            rows_l.push_back(t);
            ndet_l.push_back(ndet);
        }
    }

    RouteBuffers buf(ctx->stream);
    if (!rows_b.empty()) {
        const int64_t nb = (int64_t)rows_b.size();
        if (nb == n_tuples) {
            int rc = casci_batch(ctx, norb, h1, eri, occ, n_ref, ref_orbs, e_ref_corr, order, n_tuples, tuples,
                                 opts, eps_out, status_out, iters_out);
            if (rc) return rc;
        } else {
            void *d_tup = nullptr, *d_rows = nullptr, *d_eps = nullptr, *d_st = nullptr, *d_it = nullptr;
            MBE_CU(buf.get(tup_b.size() * sizeof(int32_t), &d_tup));
            MBE_CU(buf.get((size_t)nb * sizeof(int64_t), &d_rows));
            MBE_CU(buf.get((size_t)nb * sizeof(double), &d_eps));
            MBE_CU(buf.get((size_t)nb * sizeof(int32_t), &d_st));
            MBE_CU(buf.get((size_t)nb * sizeof(int32_t), &d_it));
            MBE_CU(cudaMemcpyAsync(d_tup, tup_b.data(), tup_b.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   ctx->stream));
            MBE_CU(cudaMemcpyAsync(d_rows, rows_b.data(), (size_t)nb * sizeof(int64_t), cudaMemcpyHostToDevice,
                                   ctx->stream));
            int rc = casci_batch(ctx, norb, h1, eri, occ, n_ref, ref_orbs, e_ref_corr, order, nb,
                                 order > 0 ? (const int32_t *)d_tup : nullptr, opts, (double *)d_eps,
                                 (int32_t *)d_st, (int32_t *)d_it);
            if (rc) return rc;
            k_route_scatter<<<(unsigned)((nb + 255) / 256), 256, 0, ctx->stream>>>(
                nb, (const int64_t *)d_rows, (const double *)d_eps, (const int32_t *)d_st, (const int32_t *)d_it,
                eps_out, status_out, iters_out);
            MBE_CU(cudaGetLastError());
            ctx->launches += 1;
        }
    }
    if (!rows_d.empty()) {
        const int64_t nd = (int64_t)rows_d.size();
        std::vector<int32_t> st_d(nd);
        for (int64_t i = 0; i < nd; ++i) {
            const int32_t *tp = tup_h.data() + (size_t)rows_d[i] * order;
            bool ok = true;
            for (int j = 0; j < order; ++j)
                ok = ok && tp[j] >= 0 && tp[j] < norb && !in_ref[tp[j]] && (j == 0 || tp[j] > tp[j - 1]);
            st_d[i] = ok ? MBE_STATUS_OK : MBE_STATUS_BADINPUT;
        }
        void *d_rows = nullptr, *d_st = nullptr;
        MBE_CU(buf.get((size_t)nd * sizeof(int64_t), &d_rows));
        MBE_CU(buf.get((size_t)nd * sizeof(int32_t), &d_st));
        MBE_CU(cudaMemcpyAsync(d_rows, rows_d.data(), (size_t)nd * sizeof(int64_t), cudaMemcpyHostToDevice,
                               ctx->stream));
        MBE_CU(cudaMemcpyAsync(d_st, st_d.data(), (size_t)nd * sizeof(int32_t), cudaMemcpyHostToDevice,
                               ctx->stream));
        k_route_direct<<<(unsigned)((nd + 255) / 256), 256, 0, ctx->stream>>>(
            nd, (const int64_t *)d_rows, (const int32_t *)d_st, e_ref_corr, eps_out, status_out, iters_out);
        MBE_CU(cudaGetLastError());
        ctx->launches += 1;
    }
    if (!rows_l.empty()) {
        // one whole-GPU solve per tuple (casci_solve is synchronous); the results
        // are scattered to their rows in one launch at the end
        const int64_t nl = (int64_t)rows_l.size();
        std::vector<double> eps_l(nl);
        std::vector<int32_t> st_l(nl), it_l(nl);
        auto solve = [&](mbe_ctx *c, int64_t i) -> int {
            std::vector<int32_t> A(n_cas);
            const int32_t *tp = tup_h.data() + (size_t)rows_l[i] * order;
            std::merge(ref_orbs, ref_orbs + n_ref, tp, tp + order, A.begin());
            double result[3] = {0.0, 0.0, 0.0};
            int32_t info[3] = {0, 0, 0};
            const int rc = casci_solve(c, norb, h1, eri, occ, n_cas, A.data(), opts, result, info, nullptr);
            if (rc) return rc;
            eps_l[i] = result[1] - e_ref_corr;
            st_l[i] = info[0];
            it_l[i] = (std::min(info[1], 65535) << 16) | std::min(info[2], 65535);
            return MBE_OK;
        };
        std::vector<int64_t> conc, alone;
        for (int64_t i = 0; i < nl; ++i) (ndet_l[i] <= ROUTE_CONCURRENT_NDET ? conc : alone).push_back(i);
        const int nw = (int)std::min<int64_t>(ROUTE_WORKERS, (int64_t)conc.size());
        if (nw >= 2) {
            int rc = route_workers(ctx, nw);
            if (rc) return rc;
            // the workers' streams start after the work queued so far on the caller's
            cudaEvent_t ready = nullptr;
            MBE_CU(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
            cudaError_t e = cudaEventRecord(ready, ctx->stream);
            for (int w = 0; w < nw && e == cudaSuccess; ++w) e = cudaStreamWaitEvent(ctx->worker_streams[w], ready, 0);
            cudaEventDestroy(ready);
            MBE_CU(e);
            std::vector<int64_t> launches0(nw);
            for (int w = 0; w < nw; ++w) launches0[w] = ctx->workers[w]->launches;
            std::atomic<int64_t> next{0};
            std::vector<int> rcs(nw, MBE_OK);
            std::vector<std::string> msgs(nw);
            auto work = [&](int w) {
                if (cudaSetDevice(ctx->device) != cudaSuccess) {
                    rcs[w] = MBE_ECUDA;
                    msgs[w] = "casci_batch_routed: cudaSetDevice failed in a worker thread";
                    next.store((int64_t)conc.size());
                    return;
                }
                for (;;) {
                    const int64_t j = next.fetch_add(1);
                    if (j >= (int64_t)conc.size()) break;
                    const int r = solve(ctx->workers[w], conc[j]);
                    if (r) {
                        rcs[w] = r;
                        msgs[w] = mbe_last_error();
                        next.store((int64_t)conc.size());
                        break;
                    }
                }
            };
            std::vector<std::thread> threads;
            for (int w = 1; w < nw; ++w) {
                try {
                    threads.emplace_back(work, w);
                } catch (...) {
                    break;  // fewer threads: the ones running take the rest of the list
                }
            }
            work(0);  // the calling thread drives worker 0
            for (auto &t : threads) t.join();
            for (int w = 0; w < nw; ++w) ctx->launches += ctx->workers[w]->launches - launches0[w];
            for (int w = 0; w < nw; ++w)
                if (rcs[w]) {
                    set_error("%s", msgs[w].c_str());
                    return rcs[w];
                }
        } else {
            alone.insert(alone.end(), conc.begin(), conc.end());
        }
        for (const int64_t i : alone) {
            const int rc = solve(ctx, i);
            if (rc) return rc;
        }
        void *d_rows = nullptr, *d_eps = nullptr, *d_st = nullptr, *d_it = nullptr;
        MBE_CU(buf.get((size_t)nl * sizeof(int64_t), &d_rows));
        MBE_CU(buf.get((size_t)nl * sizeof(double), &d_eps));
        MBE_CU(buf.get((size_t)nl * sizeof(int32_t), &d_st));
        MBE_CU(buf.get((size_t)nl * sizeof(int32_t), &d_it));
        MBE_CU(cudaMemcpyAsync(d_rows, rows_l.data(), (size_t)nl * sizeof(int64_t), cudaMemcpyHostToDevice,
                               ctx->stream));
        MBE_CU(cudaMemcpyAsync(d_eps, eps_l.data(), (size_t)nl * sizeof(double), cudaMemcpyHostToDevice,
                               ctx->stream));
        MBE_CU(cudaMemcpyAsync(d_st, st_l.data(), (size_t)nl * sizeof(int32_t), cudaMemcpyHostToDevice,
                               ctx->stream));
        MBE_CU(cudaMemcpyAsync(d_it, it_l.data(), (size_t)nl * sizeof(int32_t), cudaMemcpyHostToDevice,
                               ctx->stream));
        k_route_scatter<<<(unsigned)((nl + 255) / 256), 256, 0, ctx->stream>>>(
            nl, (const int64_t *)d_rows, (const double *)d_eps, (const int32_t *)d_st, (const int32_t *)d_it,
            eps_out, status_out, iters_out);
        MBE_CU(cudaGetLastError());
        ctx->launches += 1;
    }
    return MBE_OK;
}
