#pragma once
// Device code shared by the tuple-CASCI translation units (casci.cu, casci_warp.cu,
// casci_mixed.cu, casci_block.cu, casci_large.cu): the per-tuple problem set-up,
// sigma, the warp and block Davidson solvers and their kernels as templates.
//
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
#include <vector>

#include "common.cuh"

namespace mbe {

constexpr unsigned FULL = 0xffffffffu;
constexpr int WARP_MAX_N = 8;
constexpr int WARPS_PER_BLOCK = 4;
constexpr int CTA_THREADS = 256;
constexpr int MAX_BUCKETS = 8;
constexpr int DPL_SET[5] = {1, 2, 4, 8, 13};
// The warp solvers keep their float32 V with both signs, V2[x][2y + s] =
// (-1)^s V[x][y]: the low 9 bits of a replacement-list entry (pair << 1 | neg)
// then index the signed value directly, which saves the pair decode and the
// sign flip in the innermost loop of the float32 sigma.
constexpr bool V32_SIGNED = true;

struct ClassInfo {
    const uint32_t *strings;
    const int32_t *table;
    int ns, r;
};

struct BatchArgs {
    int norb, n, n_ref, order;
    const double *eri;
    const double *F;
    const uint8_t *occ;
    int ref[MBE_MAX_CAS];
    const int32_t *tuples;
    int64_t n_tuples;
    const int32_t *perm;
    const int64_t *bucket_off;
    unsigned long long *counters;
    ClassInfo cls[MBE_MAX_CAS + 1];
    double e_ref_corr;
    int precision;
    double tol, tol_switch;
    int max_iter, min_fp64;
    int even_only;  // solve the even spin-flip sector only
    double s2mu;    // S^2 penalty: the solvers work on H + s2mu S^2 (0: off)
    double *eps;
    int32_t *status;
    int32_t *iters;
    char *scratch;
    size_t slot_bytes;
    // mixed mode of the warp solver: the mixed launch leaves each tuple's state
    // (pstate: [flag, float32 sigma count] per tuple) for the float64 redo launch
    unsigned long long *counters2;
    int32_t *pstate;
    // tuned launch choices (mbe_tuning): warps per warp-solver block, block-solver basis
    int warps, block_basis;
    // adjoint (casci_rdm_batch): 0 = energies only, 1 = + 1-RDM, 2 = + 1- and 2-RDM
    int rdm;
    const double *weights;
    double *grad_h1;
    double *grad_eri;
};

// ------------------------------------------------------------------ group primitives

struct WarpGroup {
    __device__ static int rank() { return threadIdx.x & 31; }
    __device__ static int size() { return 32; }
    __device__ static void sync() { __syncwarp(); }
};

struct BlockGroup {
    __device__ static int rank() { return threadIdx.x; }
    __device__ static int size() { return blockDim.x; }
    __device__ static void sync() { __syncthreads(); }
};

template <typename T>
__device__ inline T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Sum of K values over the block; every thread gets the totals.  red: >= 32*K.
template <typename T, int K>
__device__ inline void block_sum(T (&v)[K], T *red)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = warp_sum(v[i]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < K; ++i) red[w * K + i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < K; ++i) {
        T s = 0;
        for (int j = 0; j < nw; ++j) s += red[j * K + i];
        v[i] = s;
    }
    __syncthreads();
}

// ------------------------------------------------------------------ per-tuple problem

struct Problem {
    int n, P, k, Ns, N, R, RS, HSS;
    const uint32_t *str;  // [Ns]
    const int32_t *tab;   // [Ns * RS]
    const int *A;         // [n] global orbital indices
    const short *pp;      // [2P] pair -> (p, q)
    double *h;            // [n*n] h_eff, then scratch
    double *hp;           // [P] h' packed
    double *V64;          // [P*P]
    float *V32;           // [P*P]
    double *Hs64;         // [Ns*HSS]
    float *Hs32;          // [Ns*HSS]
    double *diag;         // [N]
    const float *diag32;  // [N] float32 copy of the diagonal (mixed warp solver), or NULL
    void *c;              // [N] vector sigma reads (T)
    void *sbuf;           // [N] sigma output staging (warp solver)
    int sector;           // spin-flip sector of the solver's vectors (+1 or -1)
    double s2mu = 0.0;    // S^2 penalty (state targeting): sigma of H + s2mu S^2
};

// Symmetric counterpart of determinant d = Ia * Ns + Ib under the exchange of the
// alpha and beta strings.
__device__ inline int flip_det(int d, int Ns)
{
    const int ia = d / Ns;
    return (d - ia * Ns) * Ns + ia;
}

// Advances (ia, ib) by `step` positions through the row-major upper triangle
// ia <= ib < Ns; past the end, ia reaches Ns.
__device__ inline void tri_advance(int &ia, int &ib, int step, int Ns)
{
    int r = ib - ia + step;
    while (ia < Ns && r >= Ns - ia) {
        r -= Ns - ia;
        ++ia;
    }
    ib = ia + r;
}

__host__ __device__ inline int odd_stride(int x) { return x | 1; }

__device__ inline size_t eri_index(int norb, int p, int q, int r, int s)
{
    return (((size_t)p * norb + q) * norb + r) * norb + s;
}

// A = ref u tuple_t (sorted merge).  Returns false for a malformed tuple.
__device__ inline bool build_A(const BatchArgs &a, int64_t t, int *A)
{
    const int32_t *row = a.tuples ? a.tuples + t * a.order : nullptr;
    int i = 0, j = 0, m = 0, prev = -1;
    while (i < a.n_ref || j < a.order) {
        int v;
        if (j >= a.order || (i < a.n_ref && a.ref[i] < row[j])) {
            v = a.ref[i++];
        } else {
            v = row[j++];
            if (v < 0 || v >= a.norb) return false;
        }
        if (v <= prev) return false;  // unsorted, repeated or overlapping R
        prev = v;
        A[m++] = v;
    }
    return true;
}

// a2 + a4 set-up shared by both solvers.  Fills h_eff, V, h', Hs and the diagonal.
template <class G>
__device__ void setup_problem(const BatchArgs &a, Problem &pb, bool want32, bool signed32 = false)
{
    const int tid = G::rank(), nt = G::size();
    const int n = pb.n, P = pb.P, norb = a.norb;
    // pair table
    for (int e = tid; e < P; e += nt) {
        int p = 0;
        while ((p + 1) * (p + 2) / 2 <= e) ++p;
        ((short *)pb.pp)[2 * e] = (short)p;
        ((short *)pb.pp)[2 * e + 1] = (short)(e - p * (p + 1) / 2);
    }
    // h_eff from the core Fock matrix minus the in-space occupied orbitals
    for (int e = tid; e < n * n; e += nt) {
        int x = e / n, y = e - x * n;
        int gp = pb.A[x], gq = pb.A[y];
        double v = a.F[gp * norb + gq];
        for (int c = 0; c < n; ++c) {
            int gi = pb.A[c];
            if (a.occ[gi])
                v -= 2.0 * a.eri[eri_index(norb, gp, gq, gi, gi)] - a.eri[eri_index(norb, gp, gi, gi, gq)];
        }
        pb.h[e] = v;
    }
    G::sync();
    // V over packed pairs
    for (int e = tid; e < P * P; e += nt) {
        int x = e / P, y = e - x * P;
        int p = pb.pp[2 * x], q = pb.pp[2 * x + 1], r = pb.pp[2 * y], s = pb.pp[2 * y + 1];
        double v = a.eri[eri_index(norb, pb.A[p], pb.A[q], pb.A[r], pb.A[s])];
        pb.V64[e] = v;
        if (want32 && signed32) {
            pb.V32[x * 2 * P + 2 * y] = (float)v;
            pb.V32[x * 2 * P + 2 * y + 1] = -(float)v;
        } else if (want32) {
            pb.V32[e] = (float)v;
        }
    }
    G::sync();
    // h'_pq = h_eff_pq - 1/2 sum_r (pr|rq)
    for (int e = tid; e < P; e += nt) {
        int p = pb.pp[2 * e], q = pb.pp[2 * e + 1];
        double v = pb.h[p * n + q];
        for (int r = 0; r < n; ++r) v -= 0.5 * pb.V64[pair_index(p, r) * P + pair_index(r, q)];
        pb.hp[e] = v;
    }
    G::sync();
    // Hs, one column J per thread:  <K|E_rs|J> = sb and <L|E_pq|K> = sa give
    // Hs[K,J] += h'_rs sb  and  Hs[L,J] += 1/2 (pq|rs) sa sb.
    for (int J = tid; J < pb.Ns; J += nt) {
        for (int I = 0; I < pb.Ns; ++I) pb.Hs64[I * pb.HSS + J] = 0.0;
        const int32_t *tj = pb.tab + J * pb.RS;
        for (int b = 0; b < pb.R; ++b) {
            int eb = tj[b];
            int K = entry_J(eb), rs = entry_pair(eb);
            double sb = entry_neg(eb) ? -1.0 : 1.0;
            pb.Hs64[K * pb.HSS + J] += sb * pb.hp[rs];
            const int32_t *tk = pb.tab + K * pb.RS;
            for (int q = 0; q < pb.R; ++q) {
                int ea = tk[q];
                double sa = entry_neg(ea) ? -1.0 : 1.0;
                pb.Hs64[entry_J(ea) * pb.HSS + J] += 0.5 * sa * sb * pb.V64[entry_pair(ea) * P + rs];
            }
        }
    }
    G::sync();
    if (want32)
        for (int e = tid; e < pb.Ns * pb.HSS; e += nt) pb.Hs32[e] = (float)pb.Hs64[e];
    // diagonal
    for (int d = tid; d < pb.N; d += nt) {
        int ia = d / pb.Ns, ib = d - ia * pb.Ns;
        double v = pb.Hs64[ia * pb.HSS + ia] + pb.Hs64[ib * pb.HSS + ib];
        uint32_t sa = pb.str[ia];
        while (sa) {
            int p = __ffs((int)sa) - 1;
            sa &= sa - 1;
            uint32_t sb = pb.str[ib];
            while (sb) {
                int q = __ffs((int)sb) - 1;
                sb &= sb - 1;
                v += pb.V64[pair_index(p, p) * P + pair_index(q, q)];
            }
        }
        // S^2 penalty: mu times the number of alpha-only orbitals
        v += pb.s2mu * __popc(pb.str[ia] & ~pb.str[ib]);
        pb.diag[d] = v;
    }
    G::sync();
}

// v with its sign bit flipped when neg is 1 (an integer operation, so that the
// signed product below stays one fused multiply-add).
__device__ inline double flip_if(double v, int neg)
{
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}
__device__ inline float flip_if(float v, int neg) { return __int_as_float(__float_as_int(v) ^ (neg << 31)); }

// a5: one element of sigma = H c, accumulated in T; the vector c may be stored
// in a narrower type TV (the float64 sigma of a float32 anchor vector).
// (S^2 c)[Ia][Ib] for n_alpha = n_beta = k.  With S^2 = S_- S_+ (S_z = 0) and the
// alpha and beta operators ordered apart, S^2 = k - sum_pq E^a_pq E^b_qp: the
// number of alpha-only orbitals times c[Ia][Ib], minus for every alpha-only p
// and beta-only q the spin exchange c[Ia - p + q][Ib - q + p], signed by the two
// single replacements.  Those are read from the strings' replacement lists: the
// entry that empties occupied orbital o and fills u sits at (number of occupied
// orbitals below o) * (n - k + 1) + (number of empty orbitals below u) + (o < u).
template <typename T, typename TV>
__device__ inline T s2_elem(const Problem &pb, const TV *__restrict__ c, int ia, int ib)
{
    const uint32_t sa = pb.str[ia], sb = pb.str[ib];
    const uint32_t ao = sa & ~sb, bo = sb & ~sa;
    const int Ns = pb.Ns, w = pb.n - pb.k + 1;
    const uint32_t full = (1u << pb.n) - 1u;
    const int32_t *ta = pb.tab + ia * pb.RS, *tb = pb.tab + ib * pb.RS;
    T acc = (T)__popc(ao) * (T)c[ia * Ns + ib];
    for (uint32_t pm = ao; pm; pm &= pm - 1u) {
        const int p = __ffs((int)pm) - 1;
        const uint32_t below_p = (1u << p) - 1u;
        const int xa = __popc(sa & below_p) * w, yb = __popc(~sb & full & below_p);
        for (uint32_t qm = bo; qm; qm &= qm - 1u) {
            const int q = __ffs((int)qm) - 1;
            const uint32_t below_q = (1u << q) - 1u;
            const int32_t ea = ta[xa + __popc(~sa & full & below_q) + (p < q ? 1 : 0)];
            const int32_t eb = tb[__popc(sb & below_q) * w + yb + (q < p ? 1 : 0)];
            acc -= flip_if((T)c[entry_J(ea) * Ns + entry_J(eb)], entry_neg(ea) ^ entry_neg(eb));
        }
    }
    return acc;
}

// Adds mu (S^2 c) to a sigma over the half space (the elements with Ia <= Ib,
// mirrored like the sigma itself).  A separate pass, out of line and taken only
// with the penalty on, keeps the sigma's inner loop and its register allocation
// as they are without it; each thread revisits the elements it computed in the
// sigma pass, so no synchronisation is needed in between.
template <typename T, typename TV>
__device__ __noinline__ void add_s2_half(const Problem &pb, const TV *__restrict__ c, T *sbuf, int first, int stride)
{
    const int Ns = pb.Ns, nh = Ns * (Ns + 1) / 2;
    int ia = 0, ib = 0;
    tri_advance(ia, ib, first, Ns);
#pragma unroll 1
    for (int h = first; h < nh; h += stride) {
        if (!(pb.sector < 0 && ia == ib)) {
            const int d = ia * Ns + ib, pd = ib * Ns + ia;
            const T v = (T)pb.s2mu * s2_elem<T, TV>(pb, c, ia, ib);
            sbuf[d] += v;
            if (pd != d) sbuf[pd] += pb.sector > 0 ? v : -v;
        }
        tri_advance(ia, ib, stride, Ns);
    }
}

// S2: V is the signed doubled table [P][2P] (V32_SIGNED), else the plain [P][P].
template <typename T, typename TV = T, bool S2 = false>
__device__ inline T sigma_elem(const Problem &pb, const T *__restrict__ V, const T *__restrict__ Hs,
                               const TV *__restrict__ c, int d)
{
    const int Ns = pb.Ns;
    int ia = d / Ns, ib = d - ia * Ns;
    const T *ha = Hs + ia * pb.HSS;
    const T *hb = Hs + ib * pb.HSS;
    const TV *crow = c + ia * Ns;
    // Two independent accumulators per sum keep two FMA chains in flight.
    T acc0 = 0, acc1 = 0;
    for (int J = 0; J < Ns; ++J) {
        acc0 = fma(ha[J], (T)c[J * Ns + ib], acc0);
        acc1 = fma(hb[J], (T)crow[J], acc1);
    }
    const int32_t *ta = pb.tab + ia * pb.RS;
    const int32_t *tb = pb.tab + ib * pb.RS;
    const int R = pb.R;
    for (int x = 0; x < R; ++x) {
        int ea = ta[x];
        const TV *cr = c + entry_J(ea) * Ns;
        T s0 = 0, s1 = 0;
        int y = 0;
        if constexpr (S2) {
            const T *vrow = V + entry_pair(ea) * (2 * pb.P);
            for (; y + 1 < R; y += 2) {
                int e0 = tb[y], e1 = tb[y + 1];
                s0 = fma(vrow[e0 & 0x1ff], (T)cr[entry_J(e0)], s0);
                s1 = fma(vrow[e1 & 0x1ff], (T)cr[entry_J(e1)], s1);
            }
            if (y < R) {
                int e0 = tb[y];
                s0 = fma(vrow[e0 & 0x1ff], (T)cr[entry_J(e0)], s0);
            }
        } else {
            const T *vrow = V + entry_pair(ea) * pb.P;
            for (; y + 1 < R; y += 2) {
                int e0 = tb[y], e1 = tb[y + 1];
                s0 = fma(flip_if(vrow[entry_pair(e0)], entry_neg(e0)), (T)cr[entry_J(e0)], s0);
                s1 = fma(flip_if(vrow[entry_pair(e1)], entry_neg(e1)), (T)cr[entry_J(e1)], s1);
            }
            if (y < R) {
                int e0 = tb[y];
                s0 = fma(flip_if(vrow[entry_pair(e0)], entry_neg(e0)), (T)cr[entry_J(e0)], s0);
            }
        }
        T s = s0 + s1;
        if (x & 1) acc1 += flip_if(s, entry_neg(ea)); else acc0 += flip_if(s, entry_neg(ea));
    }
    return acc0 + acc1;
}

// a5: one sigma element of the block solver's float32 phase, the same terms as
// sigma_elem in another loop order.  The block's neighbouring threads hold
// neighbouring beta strings of one alpha string, so the alpha string's
// replacement list runs innermost (one table entry for the whole warp per step,
// the vector read within one row of c), and the beta-beta term reads Hs[J][Ib]
// for Hs[Ib][J] (Hs is symmetric), so that neighbouring threads read
// neighbouring elements.  Measured on 9-orbital tuples: the float32 phase 10%
// faster than with sigma_elem; the float64 sigma, bound by the FP64 pipe,
// keeps sigma_elem (it was 2% slower in this order).
template <typename T>
__device__ inline T sigma_elem_ashared(const Problem &pb, const T *__restrict__ V, const T *__restrict__ Hs,
                                       const T *__restrict__ c, int ia, int ib)
{
    const int Ns = pb.Ns, HSS = pb.HSS, P = pb.P;
    const T *ha = Hs + ia * HSS;
    const T *crow = c + ia * Ns;
    T acc0 = 0, acc1 = 0;
    for (int J = 0; J < Ns; ++J) {
        acc0 = fma(ha[J], c[J * Ns + ib], acc0);
        acc1 = fma(Hs[J * HSS + ib], crow[J], acc1);
    }
    const int32_t *ta = pb.tab + ia * pb.RS;
    const int32_t *tb = pb.tab + ib * pb.RS;
    const int R = pb.R;
    for (int y = 0; y < R; ++y) {
        const int eb = tb[y];
        const T *vcol = V + entry_pair(eb);  // column pair(eb) of V, stride P
        const T *ccol = c + entry_J(eb);     // column J_b of c, stride Ns
        // four independent chains keep four gathers of c in flight
        T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        int x = 0;
        for (; x + 3 < R; x += 4) {
            const int e0 = ta[x], e1 = ta[x + 1], e2 = ta[x + 2], e3 = ta[x + 3];
            s0 = fma(flip_if(vcol[entry_pair(e0) * P], entry_neg(e0)), ccol[entry_J(e0) * Ns], s0);
            s1 = fma(flip_if(vcol[entry_pair(e1) * P], entry_neg(e1)), ccol[entry_J(e1) * Ns], s1);
            s2 = fma(flip_if(vcol[entry_pair(e2) * P], entry_neg(e2)), ccol[entry_J(e2) * Ns], s2);
            s3 = fma(flip_if(vcol[entry_pair(e3) * P], entry_neg(e3)), ccol[entry_J(e3) * Ns], s3);
        }
        for (; x < R; ++x) {
            const int e0 = ta[x];
            s0 = fma(flip_if(vcol[entry_pair(e0) * P], entry_neg(e0)), ccol[entry_J(e0) * Ns], s0);
        }
        const T s = (s0 + s1) + (s2 + s3);
        if (y & 1) acc1 += flip_if(s, entry_neg(eb)); else acc0 += flip_if(s, entry_neg(eb));
    }
    return acc0 + acc1;
}

// Lowest eigenpair of the symmetric 3x3 Rayleigh-Ritz matrix G (m = 2 or 3 active
// rows; with m = 2 the middle row/column is absent).  Float32 Jacobi on G shifted
// by G00, then (float64 phase) one inverse-iteration step in float64.
__device__ inline void rotate3(float (&A)[3][3], float (&Vv)[3][3], int p, int q)
{
    float apq = A[p][q];
    if (apq == 0.0f) return;
    float theta = (A[q][q] - A[p][p]) / (2.0f * apq);
    float t = 1.0f / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
    if (theta < 0.0f) t = -t;
    float c = rsqrtf(t * t + 1.0f), s = t * c;
    A[p][p] -= t * apq;
    A[q][q] += t * apq;
    A[p][q] = A[q][p] = 0.0f;
    int r = 3 - p - q;
    float arp = A[r][p], arq = A[r][q];
    A[r][p] = A[p][r] = c * arp - s * arq;
    A[r][q] = A[q][r] = s * arp + c * arq;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float vp = Vv[i][p], vq = Vv[i][q];
        Vv[i][p] = c * vp - s * vq;
        Vv[i][q] = s * vp + c * vq;
    }
}

template <typename T>
__device__ inline void eig3(const T (&G)[3][3], bool have_p, T (&y)[3])
{
    float A[3][3], Vv[3][3];
    const T s0 = G[0][0];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            A[i][j] = (float)(G[i][j] - (i == j ? s0 : (T)0));
            Vv[i][j] = (i == j) ? 1.0f : 0.0f;
        }
    if (!have_p) {
        // Only x and t span the subspace: a single rotation of the {0, 2} block.
        A[0][1] = A[1][0] = A[1][2] = A[2][1] = 0.0f;
        rotate3(A, Vv, 0, 2);
        A[1][1] = 3.0e38f;
    } else {
        for (int sweep = 0; sweep < 6; ++sweep) {
            float off = fabsf(A[0][1]) + fabsf(A[0][2]) + fabsf(A[1][2]);
            float dia = fabsf(A[0][0]) + fabsf(A[1][1]) + fabsf(A[2][2]);
            if (off <= 1e-10f * dia || off < 1e-36f) break;
            rotate3(A, Vv, 0, 1);
            rotate3(A, Vv, 0, 2);
            rotate3(A, Vv, 1, 2);
        }
    }
    int m = 0;
    if (A[1][1] < A[m][m]) m = 1;
    if (A[2][2] < A[m][m]) m = 2;
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] = (T)Vv[i][m];
    if (!have_p) y[1] = (T)0;
    if constexpr (sizeof(T) == 8) {
        // float64 phase: one inverse-iteration step z = adj(G - theta I) y with
        // theta = y^T G y / y^T y makes the float32 eigenvector float64-accurate.
        T nrm = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
        T Gm[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Gm[i][j] = G[i][j];
        if (!have_p) {
            Gm[0][1] = Gm[1][0] = Gm[1][2] = Gm[2][1] = (T)0;
            Gm[1][1] = G[0][0] + (T)1.0e30;
        }
        T th = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) th += y[i] * Gm[i][j] * y[j];
        th /= nrm;
        T M[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) M[i][j] = Gm[i][j] - (i == j ? th : (T)0);
        T adj[3][3];
        adj[0][0] = M[1][1] * M[2][2] - M[1][2] * M[2][1];
        adj[0][1] = M[0][2] * M[2][1] - M[0][1] * M[2][2];
        adj[0][2] = M[0][1] * M[1][2] - M[0][2] * M[1][1];
        adj[1][0] = M[1][2] * M[2][0] - M[1][0] * M[2][2];
        adj[1][1] = M[0][0] * M[2][2] - M[0][2] * M[2][0];
        adj[1][2] = M[0][2] * M[1][0] - M[0][0] * M[1][2];
        adj[2][0] = M[1][0] * M[2][1] - M[1][1] * M[2][0];
        adj[2][1] = M[0][1] * M[2][0] - M[0][0] * M[2][1];
        adj[2][2] = M[0][0] * M[1][1] - M[0][1] * M[1][0];
        T z[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) z[i] = adj[i][0] * y[0] + adj[i][1] * y[1] + adj[i][2] * y[2];
        T zz = z[0] * z[0] + z[1] * z[1] + z[2] * z[2];
        if (zz > (T)1e-280 && isfinite(zz)) {
            T inv = (T)1 / sqrt(zz);
            T sgn = (z[0] * y[0] + z[1] * y[1] + z[2] * y[2]) < (T)0 ? -inv : inv;
#pragma unroll
            for (int i = 0; i < 3; ++i) y[i] = z[i] * sgn;
        } else {
            T inv = (T)1 / sqrt(nrm);
#pragma unroll
            for (int i = 0; i < 3; ++i) y[i] *= inv;
        }
        if (!have_p) y[1] = (T)0;
    }
}

// Fixed pseudo-random admixture of the start vector, in [-1, 1].
__device__ inline double guess_noise(int d)
{
    uint32_t h = (uint32_t)d * 2654435761u + 0x9e3779b9u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    return (double)(h & 0xffffu) / 32768.0 - 1.0;
}

constexpr double GUESS_NOISE = 1e-4;

struct PhaseOut {
    double lambda, rnorm;
    int nsig, status;
    double dnorm;  // anchored refinements: |d| of the Ritz vector x0 + d
};

// ------------------------------------------------------------------ density matrices (adjoint)

// Oriented orbitals of the replacement entry e of string s: E_pq |s> = sign |s'>
// with p created and q annihilated (p = q for the diagonal entries).
__device__ inline void entry_orbitals(const Problem &pb, uint32_t s, int32_t e, int &p, int &q)
{
    uint32_t sk = pb.str[entry_J(e)];
    if (sk == s) {
        p = q = pb.pp[2 * entry_pair(e)];
    } else {
        q = __ffs((int)(s & ~sk)) - 1;
        p = __ffs((int)(sk & ~s)) - 1;
    }
}

// Accumulates, for the unit vector c of the (k, k) sector, the spin-free
//   g1[p n + q]           += <c| E_pq |c>
//   g2[((p n + q) n + r) n + s] += <c| E_pq E_rs |c>        (g2 may be NULL)
// with E = E^alpha + E^beta, walking the replacement lists: E_rs |J> = s1 |K>,
// E_pq |K> = s2 |L> contributes c_L s1 s2 c_J.  Shared- or global-memory atomics.
template <class G>
__device__ void rdm_accumulate(const Problem &pb, const double *c, double *g1, double *g2)
{
    const int tid = G::rank(), nt = G::size();
    const int n = pb.n, Ns = pb.Ns, R = pb.R, RS = pb.RS;
    for (int d = tid; d < pb.N; d += nt) {
        const double cd = c[d];
        if (cd == 0.0) continue;
        const int ja = d / Ns, jb = d - ja * Ns;
        const uint32_t sa = pb.str[ja], sb = pb.str[jb];
        const int32_t *ta = pb.tab + ja * RS;
        const int32_t *tb = pb.tab + jb * RS;
        for (int x = 0; x < R; ++x) {  // first operator on the alpha string
            const int e = ta[x], ka = entry_J(e);
            int p, q;
            entry_orbitals(pb, sa, e, p, q);
            atomicAdd(&g1[p * n + q], flip_if(c[ka * Ns + jb], entry_neg(e)) * cd);
            if (!g2) continue;
            const double s1cd = flip_if(cd, entry_neg(e));
            const uint32_t ska = pb.str[ka];
            const int32_t *tka = pb.tab + ka * RS;
            for (int x2 = 0; x2 < R; ++x2) {
                const int e2 = tka[x2];
                int p2, q2;
                entry_orbitals(pb, ska, e2, p2, q2);
                atomicAdd(&g2[((p2 * n + q2) * n + p) * n + q],
                          flip_if(c[entry_J(e2) * Ns + jb], entry_neg(e2)) * s1cd);
            }
            for (int y2 = 0; y2 < R; ++y2) {
                const int e2 = tb[y2];
                int p2, q2;
                entry_orbitals(pb, sb, e2, p2, q2);
                atomicAdd(&g2[((p2 * n + q2) * n + p) * n + q],
                          flip_if(c[ka * Ns + entry_J(e2)], entry_neg(e2)) * s1cd);
            }
        }
        for (int y = 0; y < R; ++y) {  // first operator on the beta string
            const int e = tb[y], kb = entry_J(e);
            int p, q;
            entry_orbitals(pb, sb, e, p, q);
            atomicAdd(&g1[p * n + q], flip_if(c[ja * Ns + kb], entry_neg(e)) * cd);
            if (!g2) continue;
            const double s1cd = flip_if(cd, entry_neg(e));
            const uint32_t skb = pb.str[kb];
            const int32_t *tkb = pb.tab + kb * RS;
            for (int x2 = 0; x2 < R; ++x2) {
                const int e2 = ta[x2];
                int p2, q2;
                entry_orbitals(pb, sa, e2, p2, q2);
                atomicAdd(&g2[((p2 * n + q2) * n + p) * n + q],
                          flip_if(c[entry_J(e2) * Ns + kb], entry_neg(e2)) * s1cd);
            }
            for (int y2 = 0; y2 < R; ++y2) {
                const int e2 = tkb[y2];
                int p2, q2;
                entry_orbitals(pb, skb, e2, p2, q2);
                atomicAdd(&g2[((p2 * n + q2) * n + p) * n + q],
                          flip_if(c[ja * Ns + entry_J(e2)], entry_neg(e2)) * s1cd);
            }
        }
    }
}

// Adds w * (dE_CAS(A)/dtheta - dE_Phi/dtheta) to the gradients from the active
// density matrices accumulated by rdm_accumulate (Gamma = <E_pq E_rs> - d_qr gamma_ps).
template <class G>
__device__ void rdm_flush(const BatchArgs &a, const Problem &pb, const double *g1, const double *g2, double w)
{
    const int tid = G::rank(), nt = G::size();
    const int n = pb.n, norb = a.norb;
    const int *A = pb.A;
    for (int e = tid; e < n * n; e += nt) {
        const int p = e / n, q = e - p * n;
        const double dg = g1[e] - ((p == q && a.occ[A[p]]) ? 2.0 : 0.0);
        atomicAdd(&a.grad_h1[A[p] * norb + A[q]], w * dg);
        if (!g2 || dg == 0.0) continue;
        const double gc = w * dg;
        for (int c = 0; c < norb; ++c) {
            if (!a.occ[c]) continue;
            bool in_a = false;
            for (int i = 0; i < n; ++i) in_a |= (A[i] == c);
            if (in_a) continue;
            atomicAdd(&a.grad_eri[eri_index(norb, c, c, A[p], A[q])], gc);
            atomicAdd(&a.grad_eri[eri_index(norb, A[p], A[q], c, c)], gc);
            atomicAdd(&a.grad_eri[eri_index(norb, c, A[q], A[p], c)], -0.5 * gc);
            atomicAdd(&a.grad_eri[eri_index(norb, A[p], c, c, A[q])], -0.5 * gc);
        }
    }
    if (!g2) return;
    for (int e = tid; e < n * n * n * n; e += nt) {
        const int s = e % n, r = (e / n) % n, q = (e / (n * n)) % n, p = e / (n * n * n);
        double Gv = g2[e] - (q == r ? g1[p * n + s] : 0.0);
        const bool op = a.occ[A[p]], oq = a.occ[A[q]], orr = a.occ[A[r]];
        double phi = 0.0;
        if (p == q && r == s && op && orr) phi += (p == r) ? 2.0 : 4.0;
        if (p == s && q == r && p != q && op && oq) phi -= 2.0;
        const double v = 0.5 * w * (Gv - phi);
        if (v != 0.0) atomicAdd(&a.grad_eri[eri_index(norb, A[p], A[q], A[r], A[s])], v);
    }
}

// ------------------------------------------------------------------ warp solver

template <typename T, int DPL, typename TV = T>
__device__ inline void sigma_warp(const Problem &pb, const T *V, const T *Hs, const TV *c, T *sbuf, T (&out)[DPL])
{
    const int lane = threadIdx.x & 31, Ns = pb.Ns;
    // c lies in one spin-flip sector (P c = sector * c) and H commutes with P, so
    // only the elements with Ia <= Ib are computed and the others mirrored,
    // sigma[P d] = sector * sigma[d]; the diagonal of the odd sector vanishes.
    // One compact loop (not unrolled) keeps the kernel small for the
    // instruction cache.
    const int nh = Ns * (Ns + 1) / 2;
    int ia = 0, ib = 0;
    tri_advance(ia, ib, lane, Ns);
#pragma unroll 1
    for (int h = lane; h < nh; h += 32) {
        const int d = ia * Ns + ib, pd = ib * Ns + ia;
        const T v = (pb.sector < 0 && ia == ib) ? (T)0
                                                   : sigma_elem<T, TV, V32_SIGNED && sizeof(T) == 4>(pb, V, Hs, c, d);
        sbuf[d] = v;
        if (pd != d) sbuf[pd] = pb.sector > 0 ? v : -v;
        tri_advance(ia, ib, 32, Ns);
    }
    if (pb.s2mu != 0.0) add_s2_half<T, TV>(pb, c, sbuf, lane, 32);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < DPL; ++j) {
        int d = lane + 32 * j;
        out[j] = (d < pb.N) ? sbuf[d] : (T)0;
    }
}

template <typename T>
__device__ inline T tiny_norm();
template <>
__device__ inline float tiny_norm<float>() { return 1e-6f; }
template <>
__device__ inline double tiny_norm<double>() { return 1e-13; }

// Anchor of a float32 refinement (mixed mode): a unit vector x0, exact in
// float32, whose image under A = H - theta0 was formed once in float64:
// theta0 = x0.Hx0 / x0.x0 and r0 = H x0 - theta0 x0, stored in float32 (r0 is
// small, so float32 keeps it to about 1e-7 of its own size).  The refinement
// iterates x = x0 + d on A; every quantity it forms (d, A d, r0, the Ritz value
// mu of A) is small, so float32 rounding is relative to those small numbers and
// lambda = theta0 + mu keeps float64 accuracy.  A d of a correction comes from a
// float32 sigma minus shift * d; its rounding (about u32 |H| |d|) enters the
// Ritz value only at second order in |d|, and the coupling x0.(A v) is always
// formed as v.r0 (A symmetric), never from the float32 image.
struct Anchor {
    const float *x0, *r0;  // shared [N]
    float shift, shift_lo; // theta0 = shift + shift_lo (the images A t = (H t - shift t) - shift_lo t
                           // of the corrections see the same theta0 as r0 to float64 accuracy)
    float x0x0;            // |x0|^2 (1 up to rounding)
};

// A refinement is accepted when its residual is below tol and its correction is
// small: the float32 images of the corrections carry an error of about
// u32 |H|, which enters the Ritz value as d^T E d, so |d| <= MIX_DMAX keeps it
// below ~1e-13 E_h; a larger converged correction re-anchors at x0 + d.
constexpr double MIX_DMAX = 3e-4;

// One Davidson phase in precision T (locally optimal 3-vector form: current
// Ritz vector x, previous direction p, preconditioned residual t).
// Plain (an == NULL): x is the start vector (any norm) in, the unit Ritz vector
// out, and the return value's lambda its Ritz value of H.
// Anchored (T = float): x is the correction d (zero in), the iterate is x0 + d,
// and lambda is the Ritz value mu of A = H - theta0; the formulas below are the
// plain ones with x -> x0 + d and H x -> r0 + A d (x0 = r0 = 0 when plain).
template <typename T, int DPL>
__device__ PhaseOut davidson_warp(const Problem &pb, T (&x)[DPL], double tol, int min_iter, int max_iter,
                                  bool steer, const Anchor *an = nullptr)
{
    const int lane = threadIdx.x & 31;
    const T *V = sizeof(T) == 8 ? (const T *)pb.V64 : (const T *)pb.V32;
    const T *Hs = sizeof(T) == 8 ? (const T *)pb.Hs64 : (const T *)pb.Hs32;
    T *c = (T *)pb.c;
    T *sbuf = (T *)pb.sbuf;
    const bool anch = sizeof(T) == 4 && an != nullptr;
    const float *x0s = anch ? an->x0 : nullptr;
    const float *r0s = anch ? an->r0 : nullptr;
    const T shift = anch ? (T)an->shift : (T)0;
    const T shift_lo = anch ? (T)an->shift_lo : (T)0;
    const T x0x0 = anch ? (T)an->x0x0 : (T)0;
    auto X0 = [&](int d) -> T { return anch ? (T)x0s[d] : (T)0; };
    auto R0 = [&](int d) -> T { return anch ? (T)r0s[d] : (T)0; };
    T hx[DPL], p[DPL], hp[DPL], ht[DPL];
    PhaseOut o;
    o.nsig = 0;
    o.status = MBE_STATUS_OK;
    o.dnorm = 0.0;

    T lam = 0;
    // The first pass (plain mode) forms H x through the same sigma call that later
    // forms each correction's image: one call site keeps the kernel's code small.
    bool first = !anch;
    if (!anch) {
        T s = 0;
#pragma unroll
        for (int j = 0; j < DPL; ++j) s += x[j] * x[j];
        s = warp_sum(s);
        T inv = (T)1 / sqrt(s);
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            x[j] *= inv;
            int d = lane + 32 * j;
            if (d < pb.N) c[d] = x[j];
        }
    } else {
#pragma unroll
        for (int j = 0; j < DPL; ++j) x[j] = hx[j] = 0;  // x = x0: A x = r0, mu = x0.r0 = 0
    }
#pragma unroll
    for (int j = 0; j < DPL; ++j) p[j] = hp[j] = 0;
    bool have_p = false;
    T best = (T)3e38;
    int stall = 0;
    T rn = 0;
    T xx = 1;  // |x|^2: 1 in plain mode (x normalised), |x0 + d|^2 when anchored
    for (int it = 0;;) {
      if (!first) {
        T rr = 0;
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            int d = lane + 32 * j;
            if (d < pb.N) {
                T r = (R0(d) + hx[j]) - lam * (X0(d) + x[j]);
                rr += r * r;
                const int pd = flip_det(d, pb.Ns);
                const int cd = d < pd ? d : pd;
                T den = (pb.diag32 ? (T)pb.diag32[cd] : (T)pb.diag[cd]) - shift - lam;
                if (fabs(den) < (T)1e-4) den = den >= (T)0 ? (T)1e-4 : (T)-1e-4;
                c[d] = r / den;
            }
        }
        rn = sqrt(warp_sum(rr));
        if (!isfinite(rn) || !isfinite(lam)) {
            o.status = MBE_STATUS_NONFINITE;
            break;
        }
        if (rn <= (T)tol && it >= min_iter) break;
        if (it >= max_iter) {
            o.status = MBE_STATUS_MAXITER;
            break;
        }
        if (steer) {
            if (rn < (T)0.9 * best) {
                best = rn;
                stall = 0;
            } else if (++stall >= 3) {
                break;
            }
        }
        // orthonormalise t against x and p (two passes)
        T t0n = 0;
        if (anch) {
#pragma unroll
            for (int j = 0; j < DPL; ++j) {
                int d = lane + 32 * j;
                if (d < pb.N) t0n += c[d] * c[d];
            }
            t0n = sqrt(warp_sum(t0n));
        }
        if (anch) {
            T s = 0;
#pragma unroll
            for (int j = 0; j < DPL; ++j) {
                int d = lane + 32 * j;
                if (d < pb.N) {
                    const T xj = X0(d) + x[j];
                    s += xj * xj;
                }
            }
            xx = warp_sum(s);
        }
        for (int pass = 0; pass < 2; ++pass) {
            T ax = 0, ap = 0;
#pragma unroll
            for (int j = 0; j < DPL; ++j) {
                int d = lane + 32 * j;
                if (d < pb.N) {
                    ax += (X0(d) + x[j]) * c[d];
                    ap += p[j] * c[d];
                }
            }
            ax = warp_sum(ax) / xx;
            ap = warp_sum(ap);
#pragma unroll
            for (int j = 0; j < DPL; ++j) {
                int d = lane + 32 * j;
                if (d < pb.N) c[d] -= ax * (X0(d) + x[j]) + ap * p[j];
            }
        }
        T tt = 0;
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            int d = lane + 32 * j;
            if (d < pb.N) tt += c[d] * c[d];
        }
        T tn = sqrt(warp_sum(tt));
        if (anch ? !(tn > (T)1e-4 * t0n) : !(tn > tiny_norm<T>())) {
            // The correction lies in span{x, p}: nothing left to add.
            if (!steer && rn > (T)tol) o.status = MBE_STATUS_MAXITER;
            break;
        }
        T tinv = (T)1 / tn;
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            int d = lane + 32 * j;
            if (d < pb.N) c[d] *= tinv;
        }
      }
        __syncwarp();
        sigma_warp<T, DPL>(pb, V, Hs, c, sbuf, ht);
        ++o.nsig;
        __syncwarp();
        if (first) {
            T xh = 0;
#pragma unroll
            for (int j = 0; j < DPL; ++j) {
                hx[j] = ht[j];
                xh += x[j] * ht[j];
            }
            lam = warp_sum(xh);
            first = false;
            continue;
        }
        ++it;
        // G = [x p t]^T A [x p t]; a coupling x.(A v) is formed as v.r0 + d.(A v)
        T g00 = 0, g01 = 0, g02 = 0, g11 = 0, g12 = 0, g22 = 0;
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            int d = lane + 32 * j;
            T tj = (d < pb.N) ? c[d] : (T)0;
            if (anch) ht[j] = (ht[j] - shift * tj) - shift_lo * tj;
            const T r0j = (d < pb.N) ? R0(d) : (T)0;
            g00 += x[j] * ((T)2 * r0j + hx[j]);
            g01 += p[j] * r0j + x[j] * hp[j];
            g02 += tj * r0j + x[j] * ht[j];
            g11 += p[j] * hp[j];
            g12 += p[j] * ht[j];
            g22 += tj * ht[j];
        }
        T G[3][3];
        const T sx = anch ? (T)1 / sqrt(xx) : (T)1;  // x of unit norm in the basis
        G[0][0] = warp_sum(g00) * sx * sx;
        G[0][1] = G[1][0] = warp_sum(g01) * sx;
        G[0][2] = G[2][0] = warp_sum(g02) * sx;
        G[1][1] = warp_sum(g11);
        G[1][2] = G[2][1] = warp_sum(g12);
        G[2][2] = warp_sum(g22);
        T y[3];
        eig3<T>(G, have_p, y);
        y[0] *= sx;  // back to the coefficient of x itself
        T w2 = y[1] * y[1] + y[2] * y[2];
        T q0 = -w2 * y[0], q1 = y[1] - w2 * y[1], q2 = y[2] - w2 * y[2];
        T zn = sqrt(q0 * q0 * xx + q1 * q1 + q2 * q2);
        bool np_ok = zn > (anch ? (T)1e-30 : tiny_norm<T>() * (T)1e-3);
        T zi = np_ok ? (T)1 / zn : (T)0;
        T y0 = y[0], y1 = y[1], y2 = y[2];
        q0 *= zi;
        q1 *= zi;
        q2 *= zi;
        // new x: plain y0 x + y1 p + y2 t, normalised; anchored scaled by 1/y0 so
        // that the coefficient of x0 stays 1 (d <- d + (y1 p + y2 t) / y0)
        T nxx = 0, nxh = 0, nxr = 0, nx0 = 0;
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            int d = lane + 32 * j;
            T tj = (d < pb.N) ? c[d] : (T)0;
            const T x0j = (d < pb.N) ? X0(d) : (T)0;
            const T r0j = (d < pb.N) ? R0(d) : (T)0;
            T nx = y0 * x[j] + y1 * p[j] + y2 * tj;
            T nhx = y0 * hx[j] + y1 * hp[j] + y2 * ht[j];
            T npv = q0 * (x0j + x[j]) + q1 * p[j] + q2 * tj;
            T nhp = q0 * (r0j + hx[j]) + q1 * hp[j] + q2 * ht[j];
            x[j] = nx;
            hx[j] = nhx;
            p[j] = npv;
            hp[j] = nhp;
            nxx += nx * nx;
            nxh += nx * nhx;
            nxr += nx * r0j;
            nx0 += nx * x0j;
        }
        have_p = np_ok;
        nxx = warp_sum(nxx);
        nxh = warp_sum(nxh);
        T sc;
        if (anch) {
            nxr = warp_sum(nxr);
            nx0 = warp_sum(nx0);
            sc = (T)1 / y0;
            // mu = (x.Ax) / (x.x), x = x0 + sc nx, A x = r0 + sc A nx, x0.r0 = 0
            lam = (sc * (T)2 * nxr + sc * sc * nxh) / (x0x0 + sc * (T)2 * nx0 + sc * sc * nxx);
            o.dnorm = (double)(fabs(sc) * sqrt(nxx));
        } else {
            sc = (T)1 / sqrt(nxx);
            lam = nxh / nxx;
        }
#pragma unroll
        for (int j = 0; j < DPL; ++j) {
            x[j] *= sc;
            hx[j] *= sc;
        }
        __syncwarp();
    }
    o.lambda = (double)lam;
    o.rnorm = (double)rn;
    return o;
}

struct WarpLayout {
    int off_A, off_pp, off_h, off_hp, off_V64, off_V32, off_Hs64, off_Hs32, off_diag, off_c, off_s, off_str,
        off_tab, off_g1, off_x2, bytes;
};

__host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

// vbytes: bytes per element of the Davidson's shared vectors c and sbuf (4 in
// the float32-only launch of mixed mode, else 8)
__host__ __device__ inline WarpLayout warp_layout(int n, int ns, int r, int N, bool keep_vector, int vbytes = 8)
{
    WarpLayout L;
    int P = n * (n + 1) / 2, HSS = odd_stride(ns), RS = odd_stride(r > 0 ? r : 1);
    int o = 0;
    L.off_A = o; o = al16(o + 4 * MBE_MAX_CAS);
    L.off_pp = o; o = al16(o + 4 * P);
    L.off_h = o; o = al16(o + 8 * n * n);
    L.off_hp = o; o = al16(o + 8 * P);
    L.off_V64 = o; o = al16(o + 8 * P * P);
    L.off_V32 = o; o = al16(o + (V32_SIGNED ? 8 : 4) * P * P);
    L.off_Hs64 = o; o = al16(o + 8 * ns * HSS);
    L.off_Hs32 = o; o = al16(o + 4 * ns * HSS);
    L.off_diag = o; o = al16(o + 8 * N);
    L.off_c = o; o = al16(o + vbytes * N);
    L.off_s = o; o = al16(o + vbytes * N);
    L.off_str = o; o = al16(o + 4 * ns);
    L.off_tab = o; o = al16(o + 4 * ns * RS);
    L.off_g1 = o; o = al16(o + 8 * n * n);
    L.off_x2 = o; o = al16(o + (keep_vector ? 8 * N : 0));
    L.bytes = o;
    return L;
}

// Spin-flip symmetry. Exchanging the alpha and beta strings, (P c)[Ia][Ib] =
// c[Ib][Ia], commutes with H (the sigma is symmetric in the two spins), so H is
// block-diagonal in the sectors P c = +c (holding the closed-shell determinants)
// and P c = -c. Each sector is solved from its own start vector, and the lower
// of the two lowest eigenvalues is the lowest of the determinant space.
struct SectorGuess {
    int g;    // determinant of the start vector
    int sgn;  // sector: +1 or -1
};

// Start-vector element d of a sector: e_g + sgn e_{P g}, plus a fixed admixture
// that has the sector's symmetry.
__device__ inline double sector_guess(int d, int Ns, SectorGuess sg)
{
    const int ia = d / Ns, ib = d - ia * Ns;
    const int pd = ib * Ns + ia, pg = (sg.g % Ns) * Ns + sg.g / Ns;
    double v = (d == sg.g ? 1.0 : 0.0) + (d == pg ? (double)sg.sgn : 0.0);
    const double z = GUESS_NOISE * guess_noise(d < pd ? d : pd);
    if (d == pd) return sg.sgn > 0 ? v + z : v;
    return v + (d < pd ? z : sg.sgn * z);
}

// The second sector is first converged to the residual SECTOR_TOL only. Its
// Ritz value theta then lies within the residual norm rn of an eigenvalue, so
// when theta - rn exceeds the first sector's eigenvalue by more than a float32
// rounding margin the sector holds no lower state near theta, and it is not
// refined further.  This bounds only the eigenvalue nearest theta: a Davidson
// that still sits near an excited state of the sector, its lowest state not yet
// found, would pass the test too.  The residual is therefore taken far down
// before the decision (1e-4 of a Hamiltonian of norm ~10-100): at 1e-2, the
// decision discarded odd-sector ground states of the synthetic molecule that lie
// 0.17 E_h below the even ones.
constexpr double SECTOR_TOL = 1e-4;
__host__ __device__ inline double sector_margin(double lam) { return 1e-5 * (1.0 + fabs(lam)); }

// Reading C3: a tuple whose two spin-flip sectors both converge to lowest
// eigenvalues within DEGEN_TOL of each other has a degenerate ground state; its
// energy is valid, its state (and density matrices) is not unique.
constexpr double DEGEN_TOL = 1e-8;
__host__ __device__ inline int with_degeneracy(int status, bool degen)
{
    return (status == MBE_STATUS_OK && degen) ? MBE_STATUS_DEGENERATE : status;
}
__host__ __device__ inline bool sector_loses(double theta, double rn, double lam, double tol_conv)
{
    const double m = sector_margin(lam);
    // near an eigenvalue: theta - rn bounds it from below; converged (rn <= tol_conv):
    // theta itself is within rn^2 / gap of the sector's eigenvalue
    return (rn <= SECTOR_TOL && theta - rn > lam + m) || (rn <= tol_conv && theta > lam + m);
}

__device__ inline void store_result(const BatchArgs &a, int64_t t, double eps, int status, int n64, int n32)
{
    a.eps[t] = eps;
    a.status[t] = status;
    if (a.iters) a.iters[t] = (n64 << 16) | (n32 & 0xffff);
}

// Warp-solver modes of k_casci_warp: WM_ALL solves in float64 (float64 mode, and
// the adjoint); WM_F64 redoes in float64 the tuples that the mixed solver
// (k_casci_warp_mixed) flagged PS_REDO and skips the others.
enum { WM_ALL = 0, WM_F64 = 2 };
// pstate flags written by the mixed solver: the tuple is done (0); redo it in
// float64 (3): a float32 phase was not finite, or a refinement did not converge
enum { PS_DONE = 0, PS_REDO = 3 };

template <int DPL, int MODE>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32)
    k_casci_warp(BatchArgs a, int bucket, WarpLayout L)
{
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    char *ws = smem + (size_t)wib * L.bytes;
    const int64_t begin = a.bucket_off[bucket];
    const int64_t cnt = a.bucket_off[bucket + 1] - begin;
    const int n = a.n, P = n * (n + 1) / 2;
    int *A = (int *)(ws + L.off_A);
    for (;;) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(&(MODE == WM_F64 ? a.counters2 : a.counters)[bucket], 1ULL);
        pos = __shfl_sync(FULL, pos, 0);
        if ((int64_t)pos >= cnt) break;
        const int64_t t = a.perm[begin + (int64_t)pos];
        if (MODE == WM_F64 && a.pstate[2 * t] != PS_REDO) continue;
        if (lane == 0) build_A(a, t, A);
        __syncwarp();
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
        pb.RS = odd_stride(ci.r > 0 ? ci.r : 1);
        pb.HSS = odd_stride(ci.ns);
        pb.diag32 = nullptr;
        uint32_t *str = (uint32_t *)(ws + L.off_str);
        int32_t *tab = (int32_t *)(ws + L.off_tab);
        for (int i = lane; i < ci.ns; i += 32) str[i] = ci.strings[i];
        for (int i = lane; i < ci.ns * ci.r; i += 32) {
            int row = i / ci.r, col = i - row * ci.r;
            tab[row * pb.RS + col] = ci.table[i];
        }
        pb.str = str;
        pb.tab = tab;
        pb.A = A;
        pb.pp = (const short *)(ws + L.off_pp);
        pb.h = (double *)(ws + L.off_h);
        pb.hp = (double *)(ws + L.off_hp);
        pb.V64 = (double *)(ws + L.off_V64);
        pb.V32 = (float *)(ws + L.off_V32);
        pb.Hs64 = (double *)(ws + L.off_Hs64);
        pb.Hs32 = (float *)(ws + L.off_Hs32);
        pb.diag = (double *)(ws + L.off_diag);
        pb.c = (void *)(ws + L.off_c);
        pb.sbuf = (void *)(ws + L.off_s);
        __syncwarp();
        const bool mixed = a.precision == MBE_PREC_MIXED;
        pb.s2mu = a.s2mu;
        setup_problem<WarpGroup>(a, pb, mixed, V32_SIGNED);
        // Phi_A: the in-space occupied orbitals
        uint32_t mphi = 0;
        for (int i = 0; i < n; ++i)
            if (a.occ[A[i]]) mphi |= 1u << i;
        int iphi = string_rank(mphi);
        double ephi = pb.diag[iphi * pb.Ns + iphi];
        if (pb.N == 1) {
            if (lane == 0) store_result(a, t, pb.diag[0] - ephi - a.e_ref_corr, MBE_STATUS_OK, 0, 0);
            __syncwarp();
            continue;
        }
        // start vectors: the lowest diagonal element (ties -> lowest index), and for
        // the P = -1 sector the lowest one with Ia != Ib
        double best = 1e300, best_o = 1e300;
        int bi = 0x7fffffff, bj = 0x7fffffff;
        for (int d = lane; d < pb.N; d += 32) {
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
        {
            double x64[DPL];
            double *x2 = (double *)(ws + L.off_x2);
            double lam = 0.0;
            int status = MBE_STATUS_OK, n64 = 0, n32 = 0;
            bool degen = false;
            if constexpr (MODE == WM_F64) n32 = a.pstate[2 * t + 1];  // the mixed solver's float32 work
            // one copy of the sector's Davidson: two inlined copies, both hot on an SM,
            // overflow the instruction cache and slow every phase of every warp
#pragma unroll 1
            for (int sector = 0; sector < 2; ++sector) {
                if (sector == 1 && (pb.Ns < 2 || status != MBE_STATUS_OK || a.even_only)) break;
                const SectorGuess sg{sector == 0 ? bi : bj, sector == 0 ? 1 : -1};
                if (sector == 1 && a.rdm) {
    #pragma unroll
                    for (int j = 0; j < DPL; ++j) {
                        const int d = lane + 32 * j;
                        if (d < pb.N) x2[d] = x64[j];
                    }
                }
                pb.sector = sg.sgn;
    #pragma unroll
                for (int j = 0; j < DPL; ++j) {
                    const int d = lane + 32 * j;
                    x64[j] = (d < pb.N) ? sector_guess(d, pb.Ns, sg) : 0.0;
                }
                // the second sector is refined in float64 only if its float32
                // eigenvalue may lie below the first sector's
                bool lose = false;
                if constexpr (MODE == WM_ALL) if (mixed) {
                    float x32[DPL];
    #pragma unroll
                    for (int j = 0; j < DPL; ++j) x32[j] = (float)x64[j];
                    // the second sector: a pass to SECTOR_TOL, then one to tol_switch if undecided
                    bool finite = true;
                    for (int pass = 0; pass < 1 + sector; ++pass) {
                        const double tl = (sector == 0 || pass == 1) ? a.tol_switch : SECTOR_TOL;
                        PhaseOut o32 = davidson_warp<float, DPL>(pb, x32, tl, 0, a.max_iter, true);
                        n32 += o32.nsig;
                        finite = o32.status != MBE_STATUS_NONFINITE;
                        if (sector == 1)
                            lose = !finite || sector_loses(o32.lambda, o32.rnorm, lam, a.tol_switch);
                        if (lose || !finite) break;
                    }
                    if (finite && !lose)
    #pragma unroll
                        for (int j = 0; j < DPL; ++j) x64[j] = (double)x32[j];
                }
                // float64: in float64 mode (and for a redo) the second sector's first
                // pass (to SECTOR_TOL) decides; one call site keeps the kernel within
                // the instruction cache
                const bool pure64 = !mixed || MODE == WM_F64;
                for (int pass = (sector == 1 && pure64) ? 0 : 1; pass < 2 && !lose; ++pass) {
                    const bool first = pass == 0;
                    PhaseOut o64 = davidson_warp<double, DPL>(pb, x64, first ? SECTOR_TOL : a.tol,
                                                              (first || pure64) ? 0 : a.min_fp64, a.max_iter, first);
                    n64 += o64.nsig;
                    if (first) {
                        lose = o64.status == MBE_STATUS_NONFINITE || sector_loses(o64.lambda, o64.rnorm, lam, 0.0);
                        continue;
                    }
                    if (sector == 0) {
                        lam = o64.lambda;
                        status = o64.status;
                    } else {
                        degen = o64.status == MBE_STATUS_OK && fabs(o64.lambda - lam) <= DEGEN_TOL;
                        lose = o64.status == MBE_STATUS_NONFINITE || !(o64.lambda < lam);
                        if (!lose) {
                            lam = o64.lambda;
                            status = o64.status;
                        }
                    }
                }
                if (lose && a.rdm) {
                    __syncwarp();
    #pragma unroll
                    for (int j = 0; j < DPL; ++j) {
                        const int d = lane + 32 * j;
                        x64[j] = (d < pb.N) ? x2[d] : 0.0;
                    }
                }
                __syncwarp();
            }
            if (lane == 0) {
                double e = status == MBE_STATUS_NONFINITE ? __longlong_as_double(0x7ff8000000000000LL)
                                                          : lam - ephi - a.e_ref_corr;
                store_result(a, t, e, with_degeneracy(status, degen), n64, n32);
            }
            __syncwarp();
            if (a.rdm) {
                double *cv = (double *)pb.c;
                double *g1 = (double *)(ws + L.off_g1);
    #pragma unroll
                for (int j = 0; j < DPL; ++j) {
                    int d = lane + 32 * j;
                    if (d < pb.N) cv[d] = x64[j];
                }
                for (int e = lane; e < n * n; e += 32) g1[e] = 0.0;
                __syncwarp();
                rdm_accumulate<WarpGroup>(pb, cv, g1, nullptr);
                __syncwarp();
                rdm_flush<WarpGroup>(a, pb, g1, nullptr, a.weights ? a.weights[t] : 1.0);
                __syncwarp();
            }
        }
    }
}

// ------------------------------------------------------------------ mixed warp solver
//
// Mixed precision in one launch.  Each spin-flip sector runs the float32
// Davidson to tol_switch (the second sector is decided there, as in the
// float64 solver), then an anchored refinement: one float64 sigma of the
// float32 Ritz vector x0 gives theta0 and r0 = (H - theta0) x0, and the float32
// Davidson continues on A = H - theta0 from x0 (struct Anchor) until the
// residual of x0 + d reaches tol; lambda = theta0 + mu.  A refinement that
// stalls short of tol re-anchors at x0 + d (up to MIX_ANCHORS anchors); a
// tuple whose refinement still fails, or whose float32 phase is not finite, is
// flagged PS_REDO and solved again in float64 by the WM_F64 launch.  The float64
// data of the anchor sigma (V, Hs) are kept as packed lower triangles, so that
// a warp's shared memory stays near that of a float32-only solver.

constexpr int MIX_ANCHORS = 6;

__host__ __device__ inline int tri_index(int a, int b)
{
    const int hi = a > b ? a : b, lo = a > b ? b : a;
    return hi * (hi + 1) / 2 + lo;
}

// One element of the float64 sigma of the vector c, from the packed lower
// triangles Vp (pair x pair) and Hsp (string x string).
__device__ inline double sigma_elem_anchor(const Problem &pb, const double *__restrict__ Vp,
                                           const double *__restrict__ Hsp, const double *__restrict__ c, int d)
{
    const int Ns = pb.Ns;
    const int ia = d / Ns, ib = d - ia * Ns;
    const double *crow = c + ia * Ns;
    double acc0 = 0.0, acc1 = 0.0;
    for (int J = 0; J < Ns; ++J) {
        acc0 = fma(Hsp[tri_index(ia, J)], c[J * Ns + ib], acc0);
        acc1 = fma(Hsp[tri_index(ib, J)], crow[J], acc1);
    }
    const int32_t *ta = pb.tab + ia * pb.RS;
    const int32_t *tb = pb.tab + ib * pb.RS;
    for (int x = 0; x < pb.R; ++x) {
        const int ea = ta[x], px = entry_pair(ea);
        const double *cr = c + entry_J(ea) * Ns;
        double s = 0.0;
        for (int y = 0; y < pb.R; ++y) {
            const int e = tb[y];
            s = fma(flip_if(Vp[tri_index(px, entry_pair(e))], entry_neg(e)), cr[entry_J(e)], s);
        }
        if (x & 1) acc1 += flip_if(s, entry_neg(ea)); else acc0 += flip_if(s, entry_neg(ea));
    }
    return acc0 + acc1;
}

// The anchor sigma over the half space of the vector's sector (see sigma_warp).
template <int DPL>
__device__ inline void sigma_warp_anchor(const Problem &pb, const double *Vp, const double *Hsp, const double *c,
                                         double *sbuf, double (&out)[DPL])
{
    const int lane = threadIdx.x & 31, Ns = pb.Ns;
    const int nh = Ns * (Ns + 1) / 2;
    int ia = 0, ib = 0;
    tri_advance(ia, ib, lane, Ns);
#pragma unroll 1
    for (int h = lane; h < nh; h += 32) {
        const int d = ia * Ns + ib, pd = ib * Ns + ia;
        const double v = (pb.sector < 0 && ia == ib) ? 0.0 : sigma_elem_anchor(pb, Vp, Hsp, c, d);
        sbuf[d] = v;
        if (pd != d) sbuf[pd] = pb.sector > 0 ? v : -v;
        tri_advance(ia, ib, 32, Ns);
    }
    if (pb.s2mu != 0.0) add_s2_half<double, double>(pb, c, sbuf, lane, 32);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < DPL; ++j) {
        const int d = lane + 32 * j;
        out[j] = (d < pb.N) ? sbuf[d] : 0.0;
    }
    __syncwarp();
}

// Shared memory of one warp of the mixed solver (n orbitals, ns strings, r list
// entries, N = ns^2 determinants at most).
struct MixLayout {
    int off_A, off_pp, off_Vp, off_V32, off_Hsp, off_Hs32, off_diag, off_c, off_s, off_x0, off_r0, off_str, off_tab,
        bytes;
};

__host__ __device__ inline MixLayout mix_layout(int n, int ns, int r, int N)
{
    MixLayout L;
    const int P = n * (n + 1) / 2, HSS = odd_stride(ns), RS = odd_stride(r > 0 ? r : 1);
    const int vec = al16(4 * N);
    int o = 0;
    L.off_A = o; o = al16(o + 4 * MBE_MAX_CAS);
    L.off_pp = o; o = al16(o + 4 * P);
    L.off_Vp = o; o = al16(o + 8 * (P * (P + 1) / 2));
    L.off_V32 = o; o = al16(o + (V32_SIGNED ? 8 : 4) * P * P);
    L.off_Hsp = o; o = al16(o + 8 * (ns * (ns + 1) / 2));
    L.off_Hs32 = o; o = al16(o + 4 * ns * HSS);
    L.off_diag = o; o = al16(o + 4 * N);
    // c and sbuf of the float32 Davidson, contiguous: the anchor sigma's float64
    // staging; during set-up the full float64 Hs, then the float64 diagonal
    L.off_c = o;
    L.off_s = o + vec;
    o += 2 * vec > 8 * N ? 2 * vec : al16(8 * N);
    // x0 and r0 of an anchor; during set-up h_eff and h' (float64)
    L.off_x0 = o;
    L.off_r0 = o + vec;
    const int su = al16(8 * n * n) + 8 * P;
    o += al16(2 * vec > su ? 2 * vec : su);
    L.off_str = o; o = al16(o + 4 * ns);
    L.off_tab = o; o = al16(o + 4 * ns * RS);
    L.bytes = o;
    return L;
}

// a2 + a4 for the mixed solver (one warp): h_eff and h' in float64 (scratch in
// the anchor region), V as a packed float64 triangle and a full float32 copy,
// Hs accumulated in float64 in the vector region and kept as a packed float64
// triangle and a float32 copy, and the diagonal in float64 (left in the vector
// region for the start vectors and Phi_A) and float32 (the preconditioner).
static __device__ void setup_mix(const BatchArgs &a, Problem &pb, char *ws, const MixLayout &L, double *Vp, double *Hsp,
                          double *diag64)
{
    const int lane = threadIdx.x & 31;
    const int n = pb.n, P = pb.P, norb = a.norb, Ns = pb.Ns;
    double *h = (double *)(ws + L.off_x0);
    double *hp = h + al16(8 * n * n) / 8;
    double *Hf = (double *)(ws + L.off_c);  // full float64 Hs [Ns][Ns]
    short *pp = (short *)pb.pp;
    for (int e = lane; e < P; e += 32) {
        int p = 0;
        while ((p + 1) * (p + 2) / 2 <= e) ++p;
        pp[2 * e] = (short)p;
        pp[2 * e + 1] = (short)(e - p * (p + 1) / 2);
    }
    for (int e = lane; e < n * n; e += 32) {
        const int x = e / n, y = e - x * n;
        const int gp = pb.A[x], gq = pb.A[y];
        double v = a.F[gp * norb + gq];
        for (int c = 0; c < n; ++c) {
            const int gi = pb.A[c];
            if (a.occ[gi])
                v -= 2.0 * a.eri[eri_index(norb, gp, gq, gi, gi)] - a.eri[eri_index(norb, gp, gi, gi, gq)];
        }
        h[e] = v;
    }
    __syncwarp();
    for (int e = lane; e < P * P; e += 32) {
        const int x = e / P, y = e - x * P;
        const int p = pp[2 * x], q = pp[2 * x + 1], r = pp[2 * y], s = pp[2 * y + 1];
        const double v = a.eri[eri_index(norb, pb.A[p], pb.A[q], pb.A[r], pb.A[s])];
        if (V32_SIGNED) {
            pb.V32[x * 2 * P + 2 * y] = (float)v;
            pb.V32[x * 2 * P + 2 * y + 1] = -(float)v;
        } else {
            pb.V32[e] = (float)v;
        }
        if (x >= y) Vp[tri_index(x, y)] = v;
    }
    __syncwarp();
    for (int e = lane; e < P; e += 32) {
        const int p = pp[2 * e], q = pp[2 * e + 1];
        double v = h[p * n + q];
        for (int r = 0; r < n; ++r) v -= 0.5 * Vp[tri_index(pair_index(p, r), pair_index(r, q))];
        hp[e] = v;
    }
    __syncwarp();
    // Hs, one column J per lane (as in setup_problem)
    for (int J = lane; J < Ns; J += 32) {
        for (int I = 0; I < Ns; ++I) Hf[I * Ns + J] = 0.0;
        const int32_t *tj = pb.tab + J * pb.RS;
        for (int b = 0; b < pb.R; ++b) {
            const int eb = tj[b];
            const int K = entry_J(eb), rs = entry_pair(eb);
            const double sb = entry_neg(eb) ? -1.0 : 1.0;
            Hf[K * Ns + J] += sb * hp[rs];
            const int32_t *tk = pb.tab + K * pb.RS;
            for (int q = 0; q < pb.R; ++q) {
                const int ea = tk[q];
                const double sa = entry_neg(ea) ? -1.0 : 1.0;
                Hf[entry_J(ea) * Ns + J] += 0.5 * sa * sb * Vp[tri_index(entry_pair(ea), rs)];
            }
        }
    }
    __syncwarp();
    for (int e = lane; e < Ns * Ns; e += 32) {
        const int I = e / Ns, J = e - I * Ns;
        const double v = Hf[e];
        pb.Hs32[I * pb.HSS + J] = (float)v;
        if (I >= J) Hsp[tri_index(I, J)] = v;
    }
    __syncwarp();
    float *d32 = (float *)pb.diag32;
    for (int d = lane; d < pb.N; d += 32) {
        const int ia = d / Ns, ib = d - ia * Ns;
        double v = Hsp[tri_index(ia, ia)] + Hsp[tri_index(ib, ib)];
        uint32_t sa = pb.str[ia];
        while (sa) {
            const int p = __ffs((int)sa) - 1;
            sa &= sa - 1;
            uint32_t sb = pb.str[ib];
            while (sb) {
                const int q = __ffs((int)sb) - 1;
                sb &= sb - 1;
                v += Vp[tri_index(pair_index(p, p), pair_index(q, q))];
            }
        }
        v += pb.s2mu * __popc(pb.str[ia] & ~pb.str[ib]);
        diag64[d] = v;
        d32[d] = (float)v;
    }
    __syncwarp();
}

// Up to 8 determinants per lane the kernel fits in 128 registers, so four 4-warp
// blocks share an SM (their shared memory allows it); at 13, three: 128
// registers there spill, and four blocks ran 19% slower.
template <int DPL>
__global__ void __launch_bounds__(WARPS_PER_BLOCK * 32, DPL <= 8 ? 4 : 3)
    k_casci_warp_mixed(BatchArgs a, int bucket, MixLayout L)
{
    extern __shared__ __align__(16) char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    char *ws = smem + (size_t)wib * L.bytes;
    const int64_t begin = a.bucket_off[bucket];
    const int64_t cnt = a.bucket_off[bucket + 1] - begin;
    const int n = a.n, P = n * (n + 1) / 2;
    int *A = (int *)(ws + L.off_A);
    double *Vp = (double *)(ws + L.off_Vp);
    double *Hsp = (double *)(ws + L.off_Hsp);
    double *diag64 = (double *)(ws + L.off_c);
    double *sb64 = (double *)(ws + L.off_c);
    float *x0s = (float *)(ws + L.off_x0);
    float *r0s = (float *)(ws + L.off_r0);
    for (;;) {
        unsigned long long pos = 0;
        if (lane == 0) pos = atomicAdd(&a.counters[bucket], 1ULL);
        pos = __shfl_sync(FULL, pos, 0);
        if ((int64_t)pos >= cnt) break;
        const int64_t t = a.perm[begin + (int64_t)pos];
        if (lane == 0) build_A(a, t, A);
        __syncwarp();
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
        pb.RS = odd_stride(ci.r > 0 ? ci.r : 1);
        pb.HSS = odd_stride(ci.ns);
        uint32_t *str = (uint32_t *)(ws + L.off_str);
        int32_t *tab = (int32_t *)(ws + L.off_tab);
        for (int i = lane; i < ci.ns; i += 32) str[i] = ci.strings[i];
        for (int i = lane; i < ci.ns * ci.r; i += 32) {
            const int row = i / ci.r, col = i - row * ci.r;
            tab[row * pb.RS + col] = ci.table[i];
        }
        pb.str = str;
        pb.tab = tab;
        pb.A = A;
        pb.pp = (const short *)(ws + L.off_pp);
        pb.h = nullptr;
        pb.hp = nullptr;
        pb.V64 = nullptr;
        pb.V32 = (float *)(ws + L.off_V32);
        pb.Hs64 = nullptr;
        pb.Hs32 = (float *)(ws + L.off_Hs32);
        pb.diag = nullptr;
        pb.diag32 = (const float *)(ws + L.off_diag);
        pb.c = (void *)(ws + L.off_c);
        pb.sbuf = (void *)(ws + L.off_s);
        __syncwarp();
        pb.s2mu = a.s2mu;
        setup_mix(a, pb, ws, L, Vp, Hsp, diag64);
        uint32_t mphi = 0;
        for (int i = 0; i < n; ++i)
            if (a.occ[A[i]]) mphi |= 1u << i;
        const int iphi = string_rank(mphi);
        const double ephi = diag64[iphi * pb.Ns + iphi];
        if (pb.N == 1) {
            if (lane == 0) {
                store_result(a, t, diag64[0] - ephi - a.e_ref_corr, MBE_STATUS_OK, 0, 0);
                a.pstate[2 * t] = PS_DONE;
            }
            __syncwarp();
            continue;
        }
        // start vectors: the lowest diagonal element (ties -> lowest index), and for
        // the P = -1 sector the lowest one with Ia != Ib
        double best = 1e300, best_o = 1e300;
        int bi = 0x7fffffff, bj = 0x7fffffff;
        for (int d = lane; d < pb.N; d += 32) {
            const double v = diag64[d];
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
        __syncwarp();  // the float64 diagonal is dead from here: its region holds c and sbuf
        int n32 = 0, n64 = 0;
        bool redo = false, degen = false;
        double lam = 0.0, lam32 = 0.0;
        // one copy of the sector's Davidson: two inlined copies, both hot on an SM,
        // overflow the instruction cache and slow every phase of every warp
#pragma unroll 1
        for (int sector = 0; sector < 2 && !redo; ++sector) {
            if (sector == 1 && (pb.Ns < 2 || a.even_only)) break;
            const SectorGuess sg{sector == 0 ? bi : bj, sector == 0 ? 1 : -1};
            pb.sector = sg.sgn;
            float xv[DPL];
#pragma unroll
            for (int j = 0; j < DPL; ++j) {
                const int d = lane + 32 * j;
                xv[j] = (d < pb.N) ? (float)sector_guess(d, pb.Ns, sg) : 0.f;
            }
            // plain float32 passes (the first sector one to tol_switch; the second one
            // to SECTOR_TOL, then tol_switch, decided against the first's float32
            // eigenvalue), then anchored refinements; one call site of the Davidson
            int passes = 0, anchors = 0;
            bool lose = false, fail = false, done = false;
            double th = 0.0, lam_s = 0.0;
            Anchor an{x0s, r0s, 0.f, 0.f, 1.f};
            for (;;) {
                const bool anchored = anchors > 0;
                const double tl = anchored ? a.tol : ((sector == 0 || passes == 1) ? a.tol_switch : SECTOR_TOL);
                PhaseOut o = davidson_warp<float, DPL>(pb, xv, tl, anchored ? a.min_fp64 : 0, a.max_iter, true,
                                                       anchored ? &an : nullptr);
                n32 += o.nsig;
                if (!anchored) {
                    const bool finite = o.status != MBE_STATUS_NONFINITE;
                    if (sector == 0) {
                        lam32 = o.lambda;
                        if (!finite) {
                            fail = true;
                            break;
                        }
                    } else {
                        lose = !finite || sector_loses(o.lambda, o.rnorm, lam32, a.tol_switch);
                        if (lose) break;
                    }
                    ++passes;
                    if (sector == 1 && passes < 2) continue;
                } else {
                    lam_s = th + o.lambda;
                    if (o.status == MBE_STATUS_NONFINITE) {
                        fail = true;
                        break;
                    }
                    if (o.rnorm <= a.tol && o.dnorm <= MIX_DMAX) {
                        done = true;
                        break;
                    }
                    if (anchors >= MIX_ANCHORS) {
                        fail = true;
                        break;
                    }
                    // stalled short of tol: re-anchor at x0 + d (rounded to float32)
#pragma unroll
                    for (int j = 0; j < DPL; ++j) {
                        const int d = lane + 32 * j;
                        xv[j] = (d < pb.N) ? x0s[d] + xv[j] : 0.f;
                    }
                    __syncwarp();
                }
                // anchor at xv: float64 sigma (the vector staged in float64 over the
                // anchor region, the result in the vector region), theta0, then x0 and
                // r0 = (H - theta0) x0 in float32 over the staged vector
                double *x64 = (double *)(ws + L.off_x0);
#pragma unroll
                for (int j = 0; j < DPL; ++j) {
                    const int d = lane + 32 * j;
                    if (d < pb.N) x64[d] = (double)xv[j];
                }
                __syncwarp();
                double s0[DPL];
                sigma_warp_anchor<DPL>(pb, Vp, Hsp, x64, sb64, s0);
                ++n64;
                double xs = 0.0, xx = 0.0;
#pragma unroll
                for (int j = 0; j < DPL; ++j) {
                    xs += (double)xv[j] * s0[j];
                    xx += (double)xv[j] * (double)xv[j];
                }
                xs = warp_sum(xs);
                xx = warp_sum(xx);
                th = xs / xx;
#pragma unroll
                for (int j = 0; j < DPL; ++j) {
                    const int d = lane + 32 * j;
                    if (d < pb.N) {
                        x0s[d] = xv[j];
                        r0s[d] = (float)(s0[j] - th * (double)xv[j]);
                    }
                }
                __syncwarp();
                an.shift = (float)th;
                an.shift_lo = (float)(th - (double)an.shift);
                an.x0x0 = (float)xx;
                ++anchors;
            }
            if (sector == 0) {
                if (fail || !done) redo = true;
                lam = lam_s;
            } else if (!lose) {
                if (fail || !done) redo = true;
                degen = fabs(lam_s - lam) <= DEGEN_TOL;
                if (lam_s < lam) lam = lam_s;
            }
            __syncwarp();
        }
        if (lane == 0) {
            if (redo) {
                a.pstate[2 * t] = PS_REDO;
                a.pstate[2 * t + 1] = n32;
            } else {
                a.pstate[2 * t] = PS_DONE;
                store_result(a, t, lam - ephi - a.e_ref_corr, with_degeneracy(MBE_STATUS_OK, degen), n64, n32);
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ block solver

constexpr int MMAX = 20;  // Davidson subspace of the block solver
constexpr int KRED = 24;  // values per block reduction (>= MMAX + 1)
// float32 iterations without a 10% residual drop that end the block solver's float32
// phase (a window of 10 moved work into float32 on the 40-orbital molecule but took
// longer: this solver's float32 sigma is not much cheaper than its float64 one)
constexpr int BLOCK_STALL = 3;
// anchored refinement of the block solver: iterations without a 10% residual drop
// before it re-anchors, and the number of anchors before the float64 fallback
constexpr int BLOCK_ANCHOR_STALL = 25;
constexpr int BLOCK_ANCHORS = 8;

// Per-block workspace slot: the Davidson basis V, its image W = H V, the Ritz
// vector x and H x, a spare correction vector, the diagonal and Hs.
struct SlotLayout {
    size_t off_V, off_W, off_x, off_hx, off_t, off_diag, off_Hs64, off_Hs32, off_x2, off_x0, vec, bytes;
};

__host__ __device__ inline SlotLayout slot_layout(int ns, int N)
{
    SlotLayout L;
    size_t o = 0;
    size_t vec = ((size_t)N * 8 + 255) & ~(size_t)255;
    int HSS = odd_stride(ns);
    L.vec = vec;
    L.off_V = o; o += vec * MMAX;
    L.off_W = o; o += vec * MMAX;
    L.off_x = o; o += vec;
    L.off_hx = o; o += vec;
    L.off_t = o; o += vec;
    L.off_diag = o; o += vec;
    L.off_Hs64 = o; o += ((size_t)ns * HSS * 8 + 255) & ~(size_t)255;
    L.off_Hs32 = o; o += ((size_t)ns * HSS * 4 + 255) & ~(size_t)255;
    L.off_x2 = o; o += vec;
    L.off_x0 = o; o += vec;  // float64 anchor of the mixed refinement
    L.bytes = o;
    return L;
}

struct BlockSmem {  // dynamic shared memory of the block solver
    int off_A, off_pp, off_h, off_hp, off_V64, off_V32, off_red, off_G, off_A32, off_E32, off_ev, off_y,
        off_yp, off_r, off_misc, off_g1, off_g2, bytes;
};

__host__ __device__ inline BlockSmem block_smem(int n, bool two_body = false)
{
    BlockSmem S;
    int P = n * (n + 1) / 2, o = 0;
    S.off_A = o; o = al16(o + 4 * MBE_MAX_CAS);
    S.off_pp = o; o = al16(o + 4 * P);
    S.off_h = o; o = al16(o + 8 * n * n);
    S.off_hp = o; o = al16(o + 8 * P);
    S.off_V64 = o; o = al16(o + 8 * P * P);
    S.off_V32 = o; o = al16(o + 4 * P * P);
    S.off_red = o; o = al16(o + 8 * 32 * KRED);
    S.off_G = o; o = al16(o + 8 * MMAX * MMAX);
    S.off_A32 = o; o = al16(o + 4 * MMAX * MMAX);
    S.off_E32 = o; o = al16(o + 4 * MMAX * MMAX);
    S.off_ev = o; o = al16(o + 4 * MMAX);
    S.off_y = o; o = al16(o + 8 * MMAX);
    S.off_yp = o; o = al16(o + 8 * MMAX);
    S.off_r = o; o = al16(o + 8 * MMAX);
    S.off_misc = o; o = al16(o + 8 * 4);
    S.off_g1 = o; o = al16(o + 8 * n * n);
    S.off_g2 = o; o = al16(o + (two_body ? 8 * n * n * n * n : 0));
    S.bytes = o;
    return S;
}

// Sums of the first k of the values v[0..KRED) over the block; every thread gets
// the totals.  red: >= 32 * KRED elements of T.
template <typename T>
__device__ inline void block_sum_n(T (&v)[KRED], int k, T *red)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < KRED; ++i)
        if (i < k) v[i] = warp_sum(v[i]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < KRED; ++i)
            if (i < k) red[w * KRED + i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < KRED; ++i)
        if (i < k) {
            T s = 0;
            for (int j = 0; j < nw; ++j) s += red[j * KRED + i];
            v[i] = s;
        }
    __syncthreads();
}

// Lowest eigenpair of the m x m symmetric Rayleigh matrix G (shared memory,
// float64, row stride MMAX), computed by one warp: a float32 cyclic Jacobi on
// G - G00 I gives all eigenpairs; in the float64 phase two Newton steps in that
// eigenbasis,  z = y - sum_{k != 0} e_k (e_k . r) / (theta_k - theta),
// r = G y - theta y,  theta = y.G y, make the lowest pair float64-accurate.
// Output: y[0..m) (shared, float64, unit norm) and misc[0] = theta.
template <bool REFINE>
__device__ void small_eig_warp(const double *G, int m, float *A, float *E, float *ev, double *y, double *y2,
                               double *r, double *misc)
{
    const int lane = threadIdx.x & 31;
    const double shift = G[0];
    for (int e = lane; e < m * m; e += 32) {
        int i = e / m, j = e - i * m;
        A[i * MMAX + j] = (float)(G[i * MMAX + j] - (i == j ? shift : 0.0));
        E[i * MMAX + j] = (i == j) ? 1.0f : 0.0f;
    }
    __syncwarp();
    for (int sweep = 0; sweep < 10; ++sweep) {
        float off = 0.0f, dia = 0.0f;
        if (lane < m)
            for (int j = 0; j < m; ++j) {
                float v = A[lane * MMAX + j];
                if (j == lane) dia += v * v; else off += v * v;
            }
        off = warp_sum(off);
        dia = warp_sum(dia);
        if (off <= 1e-14f * dia || off < 1e-36f) break;
        for (int p = 0; p < m - 1; ++p)
            for (int q = p + 1; q < m; ++q) {
                float apq = A[p * MMAX + q];
                if (fabsf(apq) < 1e-36f) continue;
                float app = A[p * MMAX + p], aqq = A[q * MMAX + q];
                float th = (aqq - app) / (2.0f * apq);
                float t = 1.0f / (fabsf(th) + sqrtf(th * th + 1.0f));
                if (th < 0.0f) t = -t;
                float c = rsqrtf(t * t + 1.0f), s = t * c;
                float ajp = 0.f, ajq = 0.f, ejp = 0.f, ejq = 0.f;
                if (lane < m) {
                    ajp = A[lane * MMAX + p];
                    ajq = A[lane * MMAX + q];
                    ejp = E[lane * MMAX + p];
                    ejq = E[lane * MMAX + q];
                }
                __syncwarp();
                if (lane < m) {
                    if (lane != p && lane != q) {
                        float np_ = c * ajp - s * ajq, nq = s * ajp + c * ajq;
                        A[lane * MMAX + p] = np_;
                        A[p * MMAX + lane] = np_;
                        A[lane * MMAX + q] = nq;
                        A[q * MMAX + lane] = nq;
                    } else if (lane == p) {
                        A[p * MMAX + p] = app - t * apq;
                        A[p * MMAX + q] = 0.0f;
                        A[q * MMAX + p] = 0.0f;
                    } else {
                        A[q * MMAX + q] = aqq + t * apq;
                    }
                    E[lane * MMAX + p] = c * ejp - s * ejq;
                    E[lane * MMAX + q] = s * ejp + c * ejq;
                }
                __syncwarp();
            }
    }
    float best = (lane < m) ? A[lane * MMAX + lane] : 3.0e38f;
    int bi = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(FULL, best, o);
        int oi = __shfl_xor_sync(FULL, bi, o);
        if (ov < best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    // second-lowest eigenvalue (its eigenvector seeds the thick restart)
    float best2 = (lane < m && lane != bi) ? A[lane * MMAX + lane] : 3.0e38f;
    int b2 = (lane < m && lane != bi) ? lane : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(FULL, best2, o);
        int oi = __shfl_xor_sync(FULL, b2, o);
        if (ov < best2 || (ov == best2 && oi < b2)) {
            best2 = ov;
            b2 = oi;
        }
    }
    if (lane < m) {
        ev[lane] = A[lane * MMAX + lane];
        y[lane] = (double)E[lane * MMAX + bi];
        y2[lane] = (b2 < m) ? (double)E[lane * MMAX + b2] : 0.0;
    }
    __syncwarp();
    double theta = shift + (double)best;
    if (REFINE) {
        for (int step = 0; step < 2; ++step) {
            double g = 0.0, yi = (lane < m) ? y[lane] : 0.0;
            if (lane < m)
                for (int j = 0; j < m; ++j) g += G[lane * MMAX + j] * y[j];
            double yy = warp_sum(yi * yi), ygy = warp_sum(yi * g);
            theta = ygy / yy;
            if (lane < m) r[lane] = g - theta * yi;
            __syncwarp();
            // coefficient of eigenvector k (lane k)
            double ck = 0.0;
            if (lane < m && lane != bi) {
                for (int i = 0; i < m; ++i) ck += (double)E[i * MMAX + lane] * r[i];
                double den = shift + (double)ev[lane] - theta;
                ck = (fabs(den) > 1e-300) ? ck / den : 0.0;
            }
            __syncwarp();
            if (lane < m) r[lane] = ck;  // reuse r for the coefficients
            __syncwarp();
            double z = yi;
            if (lane < m)
                for (int k = 0; k < m; ++k) z -= (double)E[lane * MMAX + k] * r[k];
            double zz = warp_sum(z * z);
            if (lane < m) y[lane] = z / sqrt(zz);
            __syncwarp();
        }
        double g = 0.0, yi = (lane < m) ? y[lane] : 0.0;
        if (lane < m)
            for (int j = 0; j < m; ++j) g += G[lane * MMAX + j] * y[j];
        theta = warp_sum(yi * g);
    }
    if (lane == 0) misc[0] = theta;
    __syncwarp();
}

// One Davidson phase in precision T (block solver).  x: start vector in, Ritz
// vector out.  V, W: MMAX vectors each, leading dimension ld (elements).
// Block-wide sigma of a vector of one spin-flip sector: the elements with
// Ia <= Ib are computed and mirrored (see sigma_warp); ends with a barrier.
template <typename T>
__device__ inline void sigma_block(const Problem &pb, const T *Vi, const T *Hs, const T *src, T *dst)
{
    const int Ns = pb.Ns, nh = Ns * (Ns + 1) / 2;
    int ia = 0, ib = 0;
    tri_advance(ia, ib, threadIdx.x, Ns);
    for (int h = threadIdx.x; h < nh; h += blockDim.x) {
        const int d = ia * Ns + ib, pd = ib * Ns + ia;
        T v = (T)0;
        if (!(pb.sector < 0 && ia == ib)) {
            if constexpr (sizeof(T) == 4) v = sigma_elem_ashared<T>(pb, Vi, Hs, src, ia, ib);
            else v = sigma_elem<T>(pb, Vi, Hs, src, d);
        }
        dst[d] = v;
        if (pd != d) dst[pd] = pb.sector > 0 ? v : -v;
        tri_advance(ia, ib, blockDim.x, Ns);
    }
    if (pb.s2mu != 0.0) add_s2_half<T, T>(pb, src, dst, threadIdx.x, blockDim.x);
    __syncthreads();
}

// Plain: x is the start vector in, the unit Ritz vector out.  Anchored (T =
// float, anch): V[0] = x0 and W[0] = r0 = (H - shift) x0 are given (see struct
// Anchor), every other basis vector is a correction whose image is the float32
// sigma minus shift times it, the Ritz value is that of H - shift, the coupling
// of x0 to a vector v is formed as v.r0, a thick restart keeps x0 and the
// corrections of the two lowest Ritz vectors, and x returns the correction d of
// the Ritz vector x0 + d.  steer: iterations without a 10% residual drop that end
// the phase (0: none).
template <typename T>
__device__ __noinline__ PhaseOut davidson_block(const Problem &pb, T *V, T *W, size_t ld, T *x, T *hx, T *tx, char *smem,
                                   const BlockSmem &S, double tol, int min_iter, int max_iter, int steer,
                                   double shift = 0.0, bool anch = false, int mmax = MMAX)
{
    const int tid = threadIdx.x, nt = blockDim.x, N = pb.N;
    const T *Vi = sizeof(T) == 8 ? (const T *)pb.V64 : (const T *)pb.V32;
    const T *Hs = sizeof(T) == 8 ? (const T *)pb.Hs64 : (const T *)pb.Hs32;
    T *red = (T *)(smem + S.off_red);
    double *G = (double *)(smem + S.off_G);
    float *A32 = (float *)(smem + S.off_A32);
    float *E32 = (float *)(smem + S.off_E32);
    float *ev = (float *)(smem + S.off_ev);
    double *ys = (double *)(smem + S.off_y);
    double *y2s = (double *)(smem + S.off_yp);
    double *rs = (double *)(smem + S.off_r);
    double *misc = (double *)(smem + S.off_misc);
    PhaseOut o;
    o.nsig = 0;
    o.status = MBE_STATUS_OK;
    o.dnorm = 0.0;
    const T shT = (T)shift, shT_lo = (T)(shift - (double)shT);
    T v[KRED];
    if (!anch) {
        v[0] = 0;
        for (int d = tid; d < N; d += nt) v[0] += x[d] * x[d];
        block_sum_n<T>(v, 1, red);
        T inv = (T)1 / sqrt(v[0]);
        for (int d = tid; d < N; d += nt) V[d] = x[d] * inv;
        __syncthreads();
        sigma_block<T>(pb, Vi, Hs, V, W);
        ++o.nsig;
        v[0] = 0;
        for (int d = tid; d < N; d += nt) v[0] += V[d] * W[d];
        block_sum_n<T>(v, 1, red);
        if (tid == 0) G[0] = (double)v[0];
    } else if (tid == 0) {
        G[0] = 0.0;  // x0.r0 = 0: shift is x0's Rayleigh quotient
    }
    __syncthreads();
    int m = 1;
    double theta = 0.0;
    T rn = 0;
    T best = (T)3e38;
    int stall = 0;
    for (int it = 0;; ++it) {
        if (tid < 32) small_eig_warp<sizeof(T) == 8>(G, m, A32, E32, ev, ys, y2s, rs, misc);
        __syncthreads();
        theta = misc[0];
        const T th = (T)theta;
        T *tdst = (m < mmax) ? V + (size_t)m * ld : tx;
        v[0] = 0;
        v[1] = 0;
        for (int d = tid; d < N; d += nt) {
            T xs = 0, hs = 0;
            for (int i = 0; i < m; ++i) {
                T yi = (T)ys[i];
                xs += yi * V[(size_t)i * ld + d];
                hs += yi * W[(size_t)i * ld + d];
            }
            x[d] = xs;
            hx[d] = hs;
            T r = hs - th * xs;
            v[0] += r * r;
            const int pd = flip_det(d, pb.Ns);
            T den = (T)(pb.diag[d < pd ? d : pd] - shift) - th;
            if (fabs(den) < (T)1e-4) den = den >= (T)0 ? (T)1e-4 : (T)-1e-4;
            const T td = r / den;
            tdst[d] = td;
            v[1] += td * td;
        }
        block_sum_n<T>(v, 2, red);
        rn = sqrt(v[0]);
        const T t0n = sqrt(v[1]);
        if (!isfinite(rn) || !isfinite(theta)) {
            o.status = MBE_STATUS_NONFINITE;
            break;
        }
        if (rn <= (T)tol && it >= min_iter) break;
        if (it >= max_iter) {
            o.status = MBE_STATUS_MAXITER;
            break;
        }
        if (steer) {
            if (rn < (T)0.9 * best) {
                best = rn;
                stall = 0;
            } else if (++stall >= steer) {
                break;
            }
        }
        if (m == mmax && anch) {
            // Thick restart that keeps the anchor: V[0] = x0, W[0] = r0 stay; V[1], V[2]
            // become the corrections of the two lowest Ritz vectors (both orthogonal
            // to x0), orthonormalised.
            for (int d = tid; d < N; d += nt) {
                T u1 = 0, w1 = 0, u2 = 0, w2 = 0;
                for (int i = 1; i < mmax; ++i) {
                    const T vi = V[(size_t)i * ld + d], wi = W[(size_t)i * ld + d];
                    u1 += (T)ys[i] * vi;
                    w1 += (T)ys[i] * wi;
                    u2 += (T)y2s[i] * vi;
                    w2 += (T)y2s[i] * wi;
                }
                V[ld + d] = u1;
                W[ld + d] = w1;
                V[2 * ld + d] = u2;
                W[2 * ld + d] = w2;
            }
            __syncthreads();
            v[0] = 0;
            for (int d = tid; d < N; d += nt) v[0] += V[ld + d] * V[ld + d];
            block_sum_n<T>(v, 1, red);
            const T i1 = (T)1 / sqrt(v[0]);
            for (int d = tid; d < N; d += nt) {
                V[ld + d] *= i1;
                W[ld + d] *= i1;
            }
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass) {
                v[0] = 0;
                for (int d = tid; d < N; d += nt) v[0] += V[ld + d] * V[2 * ld + d];
                block_sum_n<T>(v, 1, red);
                for (int d = tid; d < N; d += nt) {
                    V[2 * ld + d] -= v[0] * V[ld + d];
                    W[2 * ld + d] -= v[0] * W[ld + d];
                }
            }
            v[0] = 0;
            for (int d = tid; d < N; d += nt) v[0] += V[2 * ld + d] * V[2 * ld + d];
            block_sum_n<T>(v, 1, red);
            int mnew = 2;
            const T n2 = sqrt(v[0]);
            if (n2 > (T)1e-3) {
                const T i2 = (T)1 / n2;
                for (int d = tid; d < N; d += nt) {
                    V[2 * ld + d] *= i2;
                    W[2 * ld + d] *= i2;
                }
                mnew = 3;
            }
            __syncthreads();
            v[0] = v[1] = v[2] = v[3] = v[4] = 0;
            for (int d = tid; d < N; d += nt) {
                v[0] += W[d] * V[ld + d];  // x0.(A u1) as u1.r0
                v[1] += V[ld + d] * W[ld + d];
                if (mnew == 3) {
                    v[2] += W[d] * V[2 * ld + d];
                    v[3] += V[ld + d] * W[2 * ld + d];
                    v[4] += V[2 * ld + d] * W[2 * ld + d];
                }
            }
            block_sum_n<T>(v, 5, red);
            if (tid == 0) {
                G[1] = G[MMAX] = (double)v[0];
                G[MMAX + 1] = (double)v[1];
                if (mnew == 3) {
                    G[2] = G[2 * MMAX] = (double)v[2];
                    G[MMAX + 2] = G[2 * MMAX + 1] = (double)v[3];
                    G[2 * MMAX + 2] = (double)v[4];
                }
            }
            m = mnew;
        } else if (m == mmax) {
            // Thick restart on the two lowest Ritz vectors of the current basis
            // (orthogonal by construction, so W stays consistent with H V).
            for (int d = tid; d < N; d += nt) {
                T x2 = 0, hx2 = 0;
                for (int i = 0; i < mmax; ++i) {
                    T yi = (T)y2s[i];
                    x2 += yi * V[(size_t)i * ld + d];
                    hx2 += yi * W[(size_t)i * ld + d];
                }
                V[d] = x[d];
                W[d] = hx[d];
                V[ld + d] = x2;
                W[ld + d] = hx2;
            }
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass) {
                v[0] = 0;
                for (int d = tid; d < N; d += nt) v[0] += V[d] * V[ld + d];
                block_sum_n<T>(v, 1, red);
                for (int d = tid; d < N; d += nt) {
                    V[ld + d] -= v[0] * V[d];
                    W[ld + d] -= v[0] * W[d];
                }
            }
            v[0] = 0;
            for (int d = tid; d < N; d += nt) v[0] += V[ld + d] * V[ld + d];
            block_sum_n<T>(v, 1, red);
            int mnew = 1;
            T nn = sqrt(v[0]);
            if (nn > (T)0.5) {
                T inv = (T)1 / nn;
                for (int d = tid; d < N; d += nt) {
                    V[ld + d] *= inv;
                    W[ld + d] *= inv;
                }
                mnew = 2;
            }
            v[0] = v[1] = v[2] = 0;
            for (int d = tid; d < N; d += nt) {
                v[0] += V[d] * W[d];
                if (mnew == 2) {
                    v[1] += V[d] * W[ld + d];
                    v[2] += V[ld + d] * W[ld + d];
                }
            }
            block_sum_n<T>(v, 3, red);
            if (tid == 0) {
                G[0] = (double)v[0];
                if (mnew == 2) {
                    G[1] = G[MMAX] = (double)v[1];
                    G[MMAX + 1] = (double)v[2];
                }
            }
            m = mnew;
        }
        // Correction: orthogonalise against V[0..m) twice, into V[m].
        T *tv = V + (size_t)m * ld;
        const T *tsrc = (tdst == tx) ? tx : tv;
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
            for (int i = 0; i < KRED; ++i) v[i] = 0;
            for (int d = tid; d < N; d += nt) {
                T td = (pass == 0) ? tsrc[d] : tv[d];
#pragma unroll
                for (int i = 0; i < MMAX; ++i)
                    if (i < m) v[i] += V[(size_t)i * ld + d] * td;
            }
            block_sum_n<T>(v, m, red);
            for (int d = tid; d < N; d += nt) {
                T td = (pass == 0) ? tsrc[d] : tv[d];
#pragma unroll
                for (int i = 0; i < MMAX; ++i)
                    if (i < m) td -= v[i] * V[(size_t)i * ld + d];
                tv[d] = td;
            }
        }
        v[0] = 0;
        for (int d = tid; d < N; d += nt) v[0] += tv[d] * tv[d];
        block_sum_n<T>(v, 1, red);
        T tn = sqrt(v[0]);
        if (!(tn > (T)1e-12 * t0n) || !(tn > (T)0)) {
            // The correction lies in the current basis: nothing left to add.
            if (!steer && rn > (T)tol) o.status = MBE_STATUS_MAXITER;
            break;
        }
        T tinv = (T)1 / tn;
        for (int d = tid; d < N; d += nt) tv[d] *= tinv;
        __syncthreads();
        T *wv = W + (size_t)m * ld;
        sigma_block<T>(pb, Vi, Hs, tv, wv);
        ++o.nsig;
#pragma unroll
        for (int i = 0; i < KRED; ++i) v[i] = 0;
        for (int d = tid; d < N; d += nt) {
            T wd = wv[d];
            if (anch) {
                wd = (wd - shT * tv[d]) - shT_lo * tv[d];
                wv[d] = wd;
            }
#pragma unroll
            for (int i = 0; i < MMAX + 1; ++i)
                if (i <= m) v[i] += (anch && i == 0) ? W[d] * tv[d] : V[(size_t)i * ld + d] * wd;
        }
        block_sum_n<T>(v, m + 1, red);
        if (tid == 0)
            for (int i = 0; i <= m; ++i) G[i * MMAX + m] = G[m * MMAX + i] = (double)v[i];
        __syncthreads();
        ++m;
    }
    if (anch) {
        // the correction d of the Ritz vector, scaled so that x0 keeps coefficient 1
        const T inv0 = (T)(1.0 / ys[0]);
        v[0] = 0;
        for (int d = tid; d < N; d += nt) {
            T u = 0;
            for (int i = 1; i < MMAX; ++i)
                if (i < m) u += (T)ys[i] * V[(size_t)i * ld + d];
            x[d] = u * inv0;
            v[0] += x[d] * x[d];
        }
        block_sum_n<T>(v, 1, red);
        o.dnorm = (double)sqrt(v[0]);
    }
    o.lambda = theta;
    o.rnorm = (double)rn;
    return o;
}

// Optional event pair around one solver launch (mbe_ctx_set_timing).
struct TimedLaunch {
    mbe_ctx *ctx;
    mbe_ctx::Pending p;
    bool on;
    TimedLaunch(mbe_ctx *c, int order, int solver, int dpl) : ctx(c), on(c->timing)
    {
        if (!on) return;
        p.rec.order = order;
        p.rec.solver = solver;
        p.rec.dpl = dpl;
        p.rec.ms = 0.0f;
        if (cudaEventCreate(&p.start) != cudaSuccess || cudaEventCreate(&p.stop) != cudaSuccess) {
            on = false;
            return;
        }
        cudaEventRecord(p.start, ctx->stream);
    }
    int done()
    {
        if (!on) return MBE_OK;
        MBE_CU(cudaEventRecord(p.stop, ctx->stream));
        ctx->pending.push_back(p);
        return MBE_OK;
    }
};

struct Bucket {
    bool warp;
    int dpl;
    int max_ns, max_r, max_n;
};

// Launchers of the solver kernels, one translation unit each (compiled in parallel).
int launch_warp_bucket(mbe_ctx *ctx, const BatchArgs &a, int b, const Bucket &bk);       // casci_warp.cu
int launch_warp_mixed_dpl(mbe_ctx *ctx, const BatchArgs &a, int b, const MixLayout &L, int dpl);  // casci_mixed.cu
int block_grid(mbe_ctx *ctx, int n, bool two_body, int *grid, size_t *smem);             // casci_block.cu
int launch_block(mbe_ctx *ctx, const BatchArgs &a, int b, int grid, size_t smem);        // casci_block.cu
__global__ void k_core_fock(int norb, const double *h1, const double *eri, const uint8_t *occ, double *F);

}  // namespace mbe
