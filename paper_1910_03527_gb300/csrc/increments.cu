// a8: increment recursion (Eq. 2); a9: order sums and total (Eq. 1 / Eq. 3);
// the reference-determinant energy.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace mbe {

struct LowerLists {
    const int32_t *tuples[MBE_MAX_ORDER];
    const double *incs[MBE_MAX_ORDER];
    int64_t count[MBE_MAX_ORDER];
};

// One thread per tuple: Delta eps = eps - sum over the proper subsets (bit masks
// 1 .. 2^order - 2 of the tuple's positions, in that order) of their increments.
__global__ void k_increments(int order, int64_t n_tuples, const int32_t *tuples, const double *eps,
                             LowerLists L, double *inc_out)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tuples) return;
    int32_t tup[MBE_MAX_ORDER], sub[MBE_MAX_ORDER];
    for (int i = 0; i < order; ++i) tup[i] = tuples[t * order + i];
    double s = 0.0;
    const unsigned full = (1u << order) - 1u;
    for (unsigned mask = 1; mask < full; ++mask) {
        int m = 0;
        for (int i = 0; i < order; ++i)
            if (mask & (1u << i)) sub[m++] = tup[i];
        int64_t pos = find_tuple(L.tuples[m - 1], L.count[m - 1], m, sub);
        if (pos >= 0) s += L.incs[m - 1][pos];
    }
    inc_out[t] = eps[t] - s;
}

// Fixed-shape reduction: block m sums list m (strided partial sums, then a tree).
constexpr int RED_THREADS = 1024;

struct SumLists {
    const double *incs[MBE_MAX_ORDER];
    int64_t count[MBE_MAX_ORDER];
};

__global__ void __launch_bounds__(RED_THREADS) k_order_sums(SumLists S, double *e_order_out)
{
    __shared__ double part[RED_THREADS];
    const int m = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < S.count[m]; i += RED_THREADS) s += S.incs[m][i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) e_order_out[m] = part[0];
}

__global__ void k_total(int n_orders, const double *e_order, const double *e_phi, double e_ref_corr,
                        double *e_total)
{
    double s = (e_phi ? e_phi[0] : 0.0) + e_ref_corr;
    for (int m = 0; m < n_orders; ++m) s += e_order[m];
    e_total[0] = s;
}

// E_Phi = sum_{i in O} 2 h_ii + sum_{i,j in O} [2 (ii|jj) - (ij|ji)]
__global__ void k_phi_energy(int norb, const double *h1, const double *eri, const uint8_t *occ, double *out)
{
    __shared__ double part[256];
    double s = 0.0;
    for (int e = threadIdx.x; e < norb * norb; e += blockDim.x) {
        int i = e / norb, j = e - i * norb;
        if (!occ[i] || !occ[j]) continue;
        size_t iijj = (((size_t)i * norb + i) * norb + j) * norb + j;
        size_t ijji = (((size_t)i * norb + j) * norb + j) * norb + i;
        s += 2.0 * eri[iijj] - eri[ijji];
        if (i == j) s += 2.0 * h1[i * norb + i];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = part[0];
}

// ------------------------------------------------------------------ adjoint weights

struct WeightArgs {
    double scale;  // every weight is multiplied by this (the adjoint's upstream factor)
    int order;  // order m of the tuples whose weights this launch computes
    int n_max;  // highest order present
    int M;
    int32_t exp[MBE_MAX_NORB];
    const int32_t *tuples[MBE_MAX_ORDER];
    const double *w[MBE_MAX_ORDER];
    int64_t count[MBE_MAX_ORDER];
};

// One thread per order-m tuple S: w(S) = 1 - sum over computed proper supersets U
// of S of w(U), scaled: s w(S) = s - sum_U s w(U).  Supersets S u J, J a j-subset (j = 1 .. n_max - m) of the
// expansion orbitals outside S, are visited in lexicographic order of J.
__global__ void k_weights(WeightArgs a, double *w_out)
{
    const int m = a.order;
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.count[m - 1]) return;
    int32_t S[MBE_MAX_ORDER], U[MBE_MAX_ORDER], fr[MBE_MAX_NORB];
    int idx[MBE_MAX_ORDER];
    for (int i = 0; i < m; ++i) S[i] = a.tuples[m - 1][t * m + i];
    int nf = 0;
    for (int i = 0, k = 0; i < a.M; ++i) {
        while (k < m && S[k] < a.exp[i]) ++k;
        if (k < m && S[k] == a.exp[i]) continue;
        fr[nf++] = a.exp[i];
    }
    double acc = 0.0;
    for (int j = 1; j <= a.n_max - m && j <= nf; ++j) {
        const int mu = m + j;
        if (a.count[mu - 1] == 0) continue;
        for (int i = 0; i < j; ++i) idx[i] = i;
        for (;;) {
            int x = 0, y = 0, z = 0;  // merge S and fr[idx]
            while (x < m || y < j) {
                if (y >= j || (x < m && S[x] < fr[idx[y]])) U[z++] = S[x++];
                else U[z++] = fr[idx[y++]];
            }
            int64_t pos = find_tuple(a.tuples[mu - 1], a.count[mu - 1], mu, U);
            if (pos >= 0) acc += a.w[mu - 1][pos];
            int i = j - 1;  // next j-combination of nf
            while (i >= 0 && idx[i] == nf - j + i) --i;
            if (i < 0) break;
            ++idx[i];
            for (int l = i + 1; l < j; ++l) idx[l] = idx[l - 1] + 1;
        }
    }
    w_out[t] = a.scale - acc;
}

// Weight of the reference-space CASCI in E_MBE = E_CAS(R) + sum_S w(S) eps(S): its
// energy enters the total once directly and, through eps(S) = E_CAS(R u S) -
// E_Phi - E_ref,corr, once more with the weight -sum_S w(S) of every computed
// tuple, so w(R) = 1 - sum_S w(S).  One block; fixed-shape reduction (strided
// partial sums over the lists in order, then a tree), so the result is
// deterministic.  With scaled weights s w(S): s w(R) = s - sum_S s w(S).
__global__ void __launch_bounds__(RED_THREADS) k_ref_weight(SumLists S, int n_orders, double scale, double *out)
{
    __shared__ double part[RED_THREADS];
    double s = 0.0;
    for (int m = 0; m < n_orders; ++m)
        for (int64_t i = threadIdx.x; i < S.count[m]; i += RED_THREADS) s += S.incs[m][i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = scale - part[0];
}

// scale * dE_Phi/dtheta, one thread per ordered pair (i, j) of orbitals
__global__ void k_phi_gradient(int norb, const uint8_t *occ, double scale, double *gh, double *ge)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= norb * norb) return;
    int i = e / norb, j = e - i * norb;
    if (!occ[i] || !occ[j]) return;
    if (i == j) {
        gh[i * norb + i] += 2.0 * scale;
        if (ge) ge[(((size_t)i * norb + i) * norb + i) * norb + i] += scale;
    } else if (ge) {
        ge[(((size_t)i * norb + i) * norb + j) * norb + j] += 2.0 * scale;
        ge[(((size_t)i * norb + j) * norb + j) * norb + i] -= scale;
    }
}

}  // namespace mbe

using namespace mbe;

extern "C" {

int mbe_phi_energy(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                   double *e_phi)
{
    MBE_CHECK(ctx && h1 && eri && occ && e_phi, MBE_EINVAL, "mbe_phi_energy: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "mbe_phi_energy: norb %d", norb);
    MBE_CU(cudaSetDevice(ctx->device));
    k_phi_energy<<<1, 256, 0, ctx->stream>>>(norb, h1, eri, occ, e_phi);
    MBE_CU(cudaGetLastError());
    ++ctx->launches;
    return MBE_OK;
}

int mbe_increments(mbe_ctx *ctx, int order, int64_t n_tuples, const int32_t *tuples, const double *eps,
                   int n_lower, const int64_t *n_lower_tuples, const int32_t *const *lower_tuples,
                   const double *const *lower_incs, double *inc_out)
{
    MBE_CHECK(ctx != nullptr, MBE_EINVAL, "mbe_increments: ctx is NULL");
    MBE_CHECK(order >= 1 && order <= MBE_MAX_ORDER && order <= 31, MBE_EINVAL,
              "mbe_increments: order %d outside 1..%d", order, MBE_MAX_ORDER);
    MBE_CHECK(n_lower == order - 1, MBE_EINVAL, "mbe_increments: n_lower (%d) must be order - 1 (%d)", n_lower,
              order - 1);
    MBE_CHECK(n_tuples >= 0, MBE_EINVAL, "mbe_increments: n_tuples < 0");
    if (n_tuples == 0) return MBE_OK;
    MBE_CHECK(tuples && eps && inc_out, MBE_EINVAL, "mbe_increments: NULL argument");
    LowerLists L;
    for (int m = 0; m < MBE_MAX_ORDER; ++m) {
        L.tuples[m] = nullptr;
        L.incs[m] = nullptr;
        L.count[m] = 0;
    }
    for (int m = 0; m < n_lower; ++m) {
        MBE_CHECK(n_lower_tuples && n_lower_tuples[m] >= 0, MBE_EINVAL, "mbe_increments: bad lower count");
        L.count[m] = n_lower_tuples[m];
        if (L.count[m] > 0) {
            MBE_CHECK(lower_tuples && lower_incs && lower_tuples[m] && lower_incs[m], MBE_EINVAL,
                      "mbe_increments: NULL lower list of order %d", m + 1);
            L.tuples[m] = lower_tuples[m];
            L.incs[m] = lower_incs[m];
        }
    }
    MBE_CU(cudaSetDevice(ctx->device));
    unsigned g = (unsigned)((n_tuples + 127) / 128);
    k_increments<<<g, 128, 0, ctx->stream>>>(order, n_tuples, tuples, eps, L, inc_out);
    MBE_CU(cudaGetLastError());
    ++ctx->launches;
    return MBE_OK;
}

int mbe_weights(mbe_ctx *ctx, int n_orders, const int64_t *n_tuples, const int32_t *const *tuples, int n_exp,
                const int32_t *exp_orbs, double scale, double *const *weights, double *ref_weight)
{
    MBE_CHECK(ctx && n_tuples && tuples && weights && (n_exp == 0 || exp_orbs), MBE_EINVAL,
              "mbe_weights: NULL argument");
    MBE_CHECK(n_orders >= 1 && n_orders <= MBE_MAX_ORDER, MBE_EINVAL, "mbe_weights: n_orders %d", n_orders);
    MBE_CHECK(n_exp >= 0 && n_exp <= MBE_MAX_NORB, MBE_EINVAL, "mbe_weights: n_exp %d", n_exp);
    WeightArgs a;
    memset(&a, 0, sizeof(a));
    std::vector<int32_t> ex(exp_orbs, exp_orbs + n_exp);
    std::sort(ex.begin(), ex.end());
    for (int i = 0; i < n_exp; ++i) a.exp[i] = ex[i];
    a.M = n_exp;
    a.n_max = n_orders;
    a.scale = scale;
    for (int m = 0; m < n_orders; ++m) {
        MBE_CHECK(n_tuples[m] >= 0 && (n_tuples[m] == 0 || (tuples[m] && weights[m])), MBE_EINVAL,
                  "mbe_weights: bad list of order %d", m + 1);
        a.tuples[m] = tuples[m];
        a.w[m] = weights[m];
        a.count[m] = n_tuples[m];
    }
    MBE_CU(cudaSetDevice(ctx->device));
    for (int m = n_orders; m >= 1; --m) {
        if (a.count[m - 1] == 0) continue;
        a.order = m;
        unsigned g = (unsigned)((a.count[m - 1] + 127) / 128);
        k_weights<<<g, 128, 0, ctx->stream>>>(a, weights[m - 1]);
        MBE_CU(cudaGetLastError());
        ++ctx->launches;
    }
    if (ref_weight) {
        SumLists S;
        for (int m = 0; m < MBE_MAX_ORDER; ++m) {
            S.incs[m] = m < n_orders ? weights[m] : nullptr;
            S.count[m] = m < n_orders ? n_tuples[m] : 0;
        }
        k_ref_weight<<<1, RED_THREADS, 0, ctx->stream>>>(S, n_orders, scale, ref_weight);
        MBE_CU(cudaGetLastError());
        ++ctx->launches;
    }
    return MBE_OK;
}

int mbe_phi_gradient(mbe_ctx *ctx, int norb, const uint8_t *occ, double scale, double *grad_h1, double *grad_eri)
{
    MBE_CHECK(ctx && occ && grad_h1, MBE_EINVAL, "mbe_phi_gradient: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "mbe_phi_gradient: norb %d", norb);
    MBE_CU(cudaSetDevice(ctx->device));
    k_phi_gradient<<<(norb * norb + 127) / 128, 128, 0, ctx->stream>>>(norb, occ, scale, grad_h1, grad_eri);
    MBE_CU(cudaGetLastError());
    ++ctx->launches;
    return MBE_OK;
}

int mbe_total(mbe_ctx *ctx, int n_orders, const int64_t *n_tuples, const double *const *incs,
              const double *e_phi, double e_ref_corr, double *e_order_out, double *e_total_out)
{
    MBE_CHECK(ctx && e_order_out && e_total_out, MBE_EINVAL, "mbe_total: NULL argument");
    MBE_CHECK(n_orders >= 0 && n_orders <= MBE_MAX_ORDER, MBE_EINVAL, "mbe_total: n_orders %d", n_orders);
    SumLists S;
    for (int m = 0; m < MBE_MAX_ORDER; ++m) {
        S.incs[m] = nullptr;
        S.count[m] = 0;
    }
    for (int m = 0; m < n_orders; ++m) {
        MBE_CHECK(n_tuples && incs && n_tuples[m] >= 0 && (n_tuples[m] == 0 || incs[m]), MBE_EINVAL,
                  "mbe_total: bad list %d", m);
        S.incs[m] = incs[m];
        S.count[m] = n_tuples[m];
    }
    MBE_CU(cudaSetDevice(ctx->device));
    if (n_orders > 0) k_order_sums<<<n_orders, RED_THREADS, 0, ctx->stream>>>(S, e_order_out);
    k_total<<<1, 1, 0, ctx->stream>>>(n_orders, e_order_out, e_phi, e_ref_corr, e_total_out);
    MBE_CU(cudaGetLastError());
    ctx->launches += (n_orders > 0 ? 2 : 1);
    return MBE_OK;
}

}  // extern "C"
