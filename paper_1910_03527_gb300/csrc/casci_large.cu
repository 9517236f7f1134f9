// ------------------------------------------------------------------ single large active space
//
// One CASCI over a large active space (up to 16 orbitals, 165.6M determinants
// at (16e,16o)), spread over the whole GPU:
//   * set-up: h_eff, packed V, h' (one block); the one-spin Hamiltonian Hs built
//     column-parallel over the grid as a dense Ns x Ns matrix, then compressed to
//     CSR (each row holds the strings connected by at most a double replacement);
//   * sigma = (Hs x 1) c + (1 x Hs) c + opposite-spin term.  The same-spin terms
//     are row-streamed sparse products C' = Hs C (coalesced over the second
//     index), the beta one applied to the transposed coefficient matrix and added
//     back transposed.  The opposite-spin term is, in float64, the direct double
//     loop over the alpha and beta replacement lists (one thread per determinant,
//     V in shared memory); in float32 it is, per alpha string, a dense product of
//     the signed V columns with the gathered rows of C followed by a scatter
//     through the beta lists into a shared-memory sigma row;
//   * inside the Davidson every vector lies in one spin-flip sector,
//     c[Ia][Ib] = sgn c[Ib][Ia], and so does its sigma: the float64 opposite-spin
//     term is computed for Ia <= Ib and mirrored, and the beta same-spin term is
//     sgn times the transpose of the alpha one (one sparse product and a
//     transposing add instead of two products and a transpose of c);
//   * Davidson: the tuple solvers' algorithm (MLARGE-vector basis, thick restart
//     on the two lowest Ritz vectors, float32 phase then float64 phase) with its
//     vector algebra in grid-wide kernels, the projected eigenproblem in one
//     warp on the device, and the host reading back one residual norm per
//     iteration to decide convergence.

#include "casci_dev.cuh"

using namespace mbe;


namespace mbe {

constexpr int MLARGE = 12;      // Davidson basis of the large solver (<= MMAX)
constexpr int LARGE_STALL = 20; // iterations without a 10% residual drop that end the sector-deciding pass
constexpr int LARGE_ANCHORS = 8;         // anchored refinements before the float64 fallback
constexpr int LARGE_ANCHOR_STALL = 30;   // iterations without a 10% drop before re-anchoring
constexpr int LRED = MLARGE + 2;  // values per grid reduction
constexpr int LARGE_THREADS = 256;
constexpr int SIGMA_THREADS = 512;

struct LargeCas {
    int n, P, k, Ns, R;
    int64_t N;
    const uint32_t *str;
    const int32_t *tab;
    double *V;      // [P*P]
    float *V32;     // [P*P]
    double *hp;     // [P]
    short *pp;      // [2P]
    double *Hd;     // dense Hs [Ns*Ns] (set-up only)
    int64_t *roff;  // CSR [Ns+1]
    int32_t *col;   // CSR [nnz]
    double *val;    // CSR [nnz]
    float *val32;   // CSR [nnz]
    double *diag;   // [N]
    int64_t nnz;
    const int32_t *tabT;  // beta lists transposed: tabT[y * Ns + J] = tab[J * R + y]
};


struct LargeSetupArgs {
    int norb;
    const double *eri;
    const double *F;
    const uint8_t *occ;
    int A[MBE_MAX_STRING_ORB];
};

// One block: pair table, h_eff, V over packed pairs (float64 and float32), h'.
__global__ void __launch_bounds__(CTA_THREADS) k_large_setup(LargeSetupArgs a, LargeCas L)
{
    __shared__ int A[MBE_MAX_STRING_ORB];
    __shared__ double h[MBE_MAX_STRING_ORB * MBE_MAX_STRING_ORB];
    const int n = L.n, P = L.P, norb = a.norb;
    if (threadIdx.x < n) A[threadIdx.x] = a.A[threadIdx.x];
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        int p = 0;
        while ((p + 1) * (p + 2) / 2 <= e) ++p;
        L.pp[2 * e] = (short)p;
        L.pp[2 * e + 1] = (short)(e - p * (p + 1) / 2);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int x = e / n, y = e - x * n;
        int gp = A[x], gq = A[y];
        double v = a.F[gp * norb + gq];
        for (int c = 0; c < n; ++c) {
            int gi = A[c];
            if (a.occ[gi])
                v -= 2.0 * a.eri[eri_index(norb, gp, gq, gi, gi)] - a.eri[eri_index(norb, gp, gi, gi, gq)];
        }
        h[e] = v;
    }
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int x = e / P, y = e - x * P;
        int p = L.pp[2 * x], q = L.pp[2 * x + 1], r = L.pp[2 * y], s = L.pp[2 * y + 1];
        double v = a.eri[eri_index(norb, A[p], A[q], A[r], A[s])];
        L.V[e] = v;
        L.V32[e] = (float)v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        int p = L.pp[2 * e], q = L.pp[2 * e + 1];
        double v = h[p * n + q];
        for (int r = 0; r < n; ++r) v -= 0.5 * L.V[pair_index(p, r) * P + pair_index(r, q)];
        L.hp[e] = v;
    }
}

// Dense Hs, one column J per thread (same recursion as the tuple set-up).
__global__ void k_large_hs_cols(LargeCas L)
{
    int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= L.Ns) return;
    const int Ns = L.Ns, R = L.R, P = L.P;
    for (int I = 0; I < Ns; ++I) L.Hd[(size_t)I * Ns + J] = 0.0;
    const int32_t *tj = L.tab + (size_t)J * R;
    for (int b = 0; b < R; ++b) {
        int eb = tj[b];
        int K = entry_J(eb), rs = entry_pair(eb);
        double sb = entry_neg(eb) ? -1.0 : 1.0;
        L.Hd[(size_t)K * Ns + J] += sb * L.hp[rs];
        const int32_t *tk = L.tab + (size_t)K * R;
        for (int q = 0; q < R; ++q) {
            int ea = tk[q];
            double sa = entry_neg(ea) ? -1.0 : 1.0;
            L.Hd[(size_t)entry_J(ea) * Ns + J] += 0.5 * sa * sb * L.V[entry_pair(ea) * P + rs];
        }
    }
}

// Non-zeros per row (one warp per row), for the CSR offsets.
__global__ void k_large_hs_count(LargeCas L, int32_t *cnt)
{
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= L.Ns) return;
    const double *hr = L.Hd + (size_t)row * L.Ns;
    int c = 0;
    for (int base = 0; base < L.Ns; base += 32) {
        int j = base + lane;
        bool nz = j < L.Ns && hr[j] != 0.0;
        c += __popc(__ballot_sync(FULL, nz));
    }
    if (lane == 0) cnt[row] = c;
}

__global__ void k_large_hs_fill(LargeCas L, const int64_t *off)
{
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= L.Ns) return;
    const double *hr = L.Hd + (size_t)row * L.Ns;
    int64_t pos = off[row];
    if (lane == 0) L.roff[row] = pos;
    if (row == L.Ns - 1 && lane == 0) L.roff[L.Ns] = off[L.Ns];
    for (int base = 0; base < L.Ns; base += 32) {
        int j = base + lane;
        double v = (j < L.Ns) ? hr[j] : 0.0;
        unsigned m = __ballot_sync(FULL, v != 0.0);
        if (v != 0.0) {
            int64_t at = pos + __popc(m & ((1u << lane) - 1u));
            L.col[at] = j;
            L.val[at] = v;
            L.val32[at] = (float)v;
        }
        pos += __popc(m);
    }
}

__global__ void k_large_diag(LargeCas L)
{
    const int Ns = L.Ns, P = L.P;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < L.N; d += (int64_t)gridDim.x * blockDim.x) {
        int ia = (int)(d / Ns), ib = (int)(d - (int64_t)ia * Ns);
        double v = L.Hd[(size_t)ia * Ns + ia] + L.Hd[(size_t)ib * Ns + ib];
        uint32_t sa = L.str[ia];
        while (sa) {
            int p = __ffs((int)sa) - 1;
            sa &= sa - 1;
            uint32_t sb = L.str[ib];
            while (sb) {
                int q = __ffs((int)sb) - 1;
                sb &= sb - 1;
                v += L.V[pair_index(p, p) * P + pair_index(q, q)];
            }
        }
        L.diag[d] = v;
    }
}

// Opposite-spin part of sigma in float64, one thread per determinant:
//     sigma[Ia][Ib] = sum_{x in list(Ia)} s_x sum_{y in list(Ib)} s_y V[p_x][p_y] c[J_x][J_y]
// (written, not accumulated). The beta lists are read through the transposed
// table, so a warp's 32 consecutive Ib load 32 consecutive words.
// SECTOR: c lies in the spin-flip sector sgn (c[Ia][Ib] = sgn c[Ib][Ia]), so only
// the elements with Ia <= Ib are computed, walking the upper triangle row by
// row, and each is mirrored, sigma[Ib][Ia] = sgn sigma[Ia][Ib] (the diagonal of
// the odd sector vanishes).  Otherwise every element, in row-major order.
template <bool SECTOR>
__global__ void __launch_bounds__(SIGMA_THREADS) k_large_ab64(LargeCas L, const double *__restrict__ c,
                                                               double *__restrict__ sigma, int sgn)
{
    extern __shared__ __align__(16) char smem[];
    double *Vs = (double *)smem;
    const int P = L.P, Ns = L.Ns, R = L.R;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) Vs[e] = L.V[e];
    __syncthreads();
    const int64_t count = SECTOR ? (int64_t)Ns * (Ns + 1) / 2 : L.N;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < count; h += (int64_t)gridDim.x * blockDim.x) {
        int ia, ib;
        if (SECTOR) {
            // row ia of the upper triangle starts at ia Ns - ia (ia - 1) / 2
            const double b2 = 2.0 * Ns + 1.0;
            ia = (int)((b2 - sqrt(b2 * b2 - 8.0 * (double)h)) * 0.5);
            auto start = [&](int64_t r) { return r * Ns - r * (r - 1) / 2; };
            while (ia > 0 && start(ia) > h) --ia;
            while (ia + 1 < Ns && start(ia + 1) <= h) ++ia;
            ib = ia + (int)(h - start(ia));
            if (sgn < 0 && ia == ib) {
                sigma[(int64_t)ia * Ns + ib] = 0.0;
                continue;
            }
        } else {
            ia = (int)(h / Ns);
            ib = (int)(h - (int64_t)ia * Ns);
        }
        double acc0 = 0.0, acc1 = 0.0;
        const int32_t *ta = L.tab + (size_t)ia * R;
        const int32_t *tb = L.tabT + ib;
        for (int x = 0; x < R; ++x) {
            const int ea = ta[x];
            const double *vrow = Vs + entry_pair(ea) * P;
            const double *cr = c + (int64_t)entry_J(ea) * Ns;
            double s0 = 0.0, s1 = 0.0;
            int y = 0;
            for (; y + 1 < R; y += 2) {
                const int e0 = tb[(size_t)y * Ns], e1 = tb[(size_t)(y + 1) * Ns];
                s0 = fma(flip_if(vrow[entry_pair(e0)], entry_neg(e0)), cr[entry_J(e0)], s0);
                s1 = fma(flip_if(vrow[entry_pair(e1)], entry_neg(e1)), cr[entry_J(e1)], s1);
            }
            if (y < R) {
                const int e0 = tb[(size_t)y * Ns];
                s0 = fma(flip_if(vrow[entry_pair(e0)], entry_neg(e0)), cr[entry_J(e0)], s0);
            }
            const double s = s0 + s1;
            if (x & 1) acc1 += flip_if(s, entry_neg(ea)); else acc0 += flip_if(s, entry_neg(ea));
        }
        const double v = acc0 + acc1;
        sigma[(int64_t)ia * Ns + ib] = v;
        if (SECTOR && ia < ib) sigma[(int64_t)ib * Ns + ia] = sgn > 0 ? v : -v;
    }
}

// Same-spin part, row-streamed: out[I][K] += sum_e val[e] X[col[e]][K] over the
// CSR row I of Hs, for a block of SS_ROWS rows and a tile of SS_TK columns per
// work item. Column tiles are the outer work index, so the CTAs in flight share
// one slab of X in L2. With TRANS the result is added at out[K][I] (X is the
// transposed coefficient matrix and the product is C Hs^T).
constexpr int SS_ROWS = 32, SS_TK = 256, SS_THREADS = 256;

// STORE: out[I][K] = (Hs X)[I][K] instead of adding it (TRANS false only).
template <typename T, bool TRANS, bool STORE = false>
__global__ void __launch_bounds__(SS_THREADS) k_large_ss(LargeCas L, const T *__restrict__ X,
                                                          double *__restrict__ sigma)
{
    extern __shared__ __align__(16) char smem[];
    T *out = (T *)smem;  // [SS_ROWS][SS_TK + 1]
    const int Ns = L.Ns, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const T *val = sizeof(T) == 8 ? (const T *)L.val : (const T *)L.val32;
    const int nrb = (Ns + SS_ROWS - 1) / SS_ROWS, nct = (Ns + SS_TK - 1) / SS_TK;
    for (int item = blockIdx.x; item < nrb * nct; item += gridDim.x) {
        const int ct = item / nrb, rb = item - ct * nrb;
        const int I0 = rb * SS_ROWS, K0 = ct * SS_TK;
        for (int r = w; r < SS_ROWS; r += SS_THREADS / 32) {
            const int I = I0 + r;
            T acc[SS_TK / 32];
#pragma unroll
            for (int j = 0; j < SS_TK / 32; ++j) acc[j] = 0;
            if (I < Ns) {
                const int64_t e1 = L.roff[I + 1];
                for (int64_t e = L.roff[I]; e < e1; ++e) {
                    const T v = val[e];
                    const T *xr = X + (size_t)L.col[e] * Ns + K0 + lane;
#pragma unroll
                    for (int j = 0; j < SS_TK / 32; ++j)
                        if (K0 + lane + 32 * j < Ns) acc[j] = fma(v, xr[32 * j], acc[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < SS_TK / 32; ++j) out[r * (SS_TK + 1) + lane + 32 * j] = acc[j];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < SS_ROWS * SS_TK; i += SS_THREADS) {
            const int r = TRANS ? (i & (SS_ROWS - 1)) : i / SS_TK;
            const int k = TRANS ? i / SS_ROWS : (i & (SS_TK - 1));
            const int I = I0 + r, K = K0 + k;
            if (I < Ns && K < Ns) {
                const size_t at = TRANS ? (size_t)K * Ns + I : (size_t)I * Ns + K;
                if (STORE)
                    sigma[at] = (double)out[r * (SS_TK + 1) + k];
                else
                    sigma[at] += (double)out[r * (SS_TK + 1) + k];
            }
        }
        __syncthreads();
    }
}

// sigma += A + sgn A^T for an Ns x Ns matrix A (32 x 32 tiles through shared
// memory): the same-spin terms of a vector in the spin-flip sector sgn, whose
// beta term is sgn times the transpose of the alpha term A = Hs C.
__global__ void k_sym_add(const double *__restrict__ A, int Ns, int sgn, double *__restrict__ sigma)
{
    __shared__ double tile[32][33];
    const int nt = (Ns + 31) / 32;
    for (int64_t t = blockIdx.x; t < (int64_t)nt * nt; t += gridDim.x) {
        const int bi = (int)(t / nt), bj = (int)(t - (int64_t)bi * nt);
        // tile[x][r] = A[bj*32 + r][bi*32 + x], read row-wise (coalesced)
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int i = bj * 32 + r, j = bi * 32 + threadIdx.x;
            tile[threadIdx.x][r] = (i < Ns && j < Ns) ? A[(size_t)i * Ns + j] : 0.0;
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int i = bi * 32 + r, j = bj * 32 + threadIdx.x;
            if (i < Ns && j < Ns) {
                const size_t at = (size_t)i * Ns + j;
                const double at_t = tile[r][threadIdx.x];  // A[j][i]
                sigma[at] += A[at] + (sgn > 0 ? at_t : -at_t);
            }
        }
        __syncthreads();
    }
}

// out = in^T for an Ns x Ns matrix, 32 x 32 tiles through shared memory.
template <typename T>
__global__ void k_large_transpose(const T *__restrict__ in, int Ns, T *__restrict__ out)
{
    __shared__ T tile[32][33];
    const int nt = (Ns + 31) / 32;
    for (int64_t t = blockIdx.x; t < (int64_t)nt * nt; t += gridDim.x) {
        const int bi = (int)(t / nt), bj = (int)(t - (int64_t)bi * nt);
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int i = bi * 32 + r, j = bj * 32 + threadIdx.x;
            if (i < Ns && j < Ns) tile[r][threadIdx.x] = in[(size_t)i * Ns + j];
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += blockDim.y) {
            const int j = bj * 32 + r, i = bi * 32 + threadIdx.x;
            if (i < Ns && j < Ns) out[(size_t)j * Ns + i] = tile[threadIdx.x][r];
        }
        __syncthreads();
    }
}

// tabT[y * Ns + J] = tab[J * R + y] (the beta lists of the float64 opposite-spin term)
__global__ void k_large_tables(LargeCas L, int32_t *tabT)
{
    for (int J = blockIdx.x * blockDim.x + threadIdx.x; J < L.Ns; J += gridDim.x * blockDim.x)
        for (int y = 0; y < L.R; ++y) tabT[(size_t)y * L.Ns + J] = L.tab[(size_t)J * L.R + y];
}

// ---- grid-wide vector algebra of the large Davidson (all float64)

// partial[b*K + i] = block b's share of sum_d A_i[d] * u[d], i < K; A_i = A + i*ld.
__global__ void __launch_bounds__(LARGE_THREADS) k_multidot(const double *A, size_t ld, int K, const double *u,
                                                            int64_t N, double *partial)
{
    __shared__ double red[32 * LRED];
    double v[LRED];
#pragma unroll
    for (int i = 0; i < LRED; ++i) v[i] = 0.0;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x) {
        const double ud = u[d];
#pragma unroll
        for (int i = 0; i < LRED; ++i)
            if (i < K) v[i] += A[i * ld + d] * ud;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < LRED; ++i)
        if (i < K) v[i] = warp_sum(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < LRED; ++i)
            if (i < K) red[w * LRED + i] = v[i];
    __syncthreads();
    if (threadIdx.x < K) {
        double s = 0.0;
        for (int j = 0; j < nw; ++j) s += red[j * LRED + threadIdx.x];
        partial[(size_t)blockIdx.x * K + threadIdx.x] = s;
    }
}

// out[i] = sum over blocks of partial (fixed order); one warp per value.
__global__ void k_multidot_final(const double *partial, int nblocks, int K, double *out)
{
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (i >= K) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(size_t)b * K + i];
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
}

// x = V y, hx = W y, r = hx - theta x, t = r / clamp(diag - theta); partial sums of
// |r|^2 and |t|^2 (two values per block).
__global__ void __launch_bounds__(LARGE_THREADS) k_ritz(const double *V, const double *W, size_t ld, int m,
                                                        const double *ys, const double *misc, const double *diag,
                                                        double shift, int64_t N, double *x, double *hx, double *t,
                                                        double *partial)
{
    __shared__ double red[64];
    const double th = misc[0];
    double y[MLARGE];
#pragma unroll
    for (int i = 0; i < MLARGE; ++i) y[i] = (i < m) ? ys[i] : 0.0;
    double rr = 0.0, tt = 0.0;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x) {
        double xs = 0.0, hs = 0.0;
#pragma unroll
        for (int i = 0; i < MLARGE; ++i)
            if (i < m) {
                xs += y[i] * V[i * ld + d];
                hs += y[i] * W[i * ld + d];
            }
        x[d] = xs;
        hx[d] = hs;
        double r = hs - th * xs;
        double den = (diag[d] - shift) - th;
        if (fabs(den) < 1e-4) den = den >= 0.0 ? 1e-4 : -1e-4;
        double td = r / den;
        t[d] = td;
        rr += r * r;
        tt += td * td;
    }
    rr = warp_sum(rr);
    tt = warp_sum(tt);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[w] = rr;
        red[32 + w] = tt;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int j = 0; j < nw; ++j) s += red[threadIdx.x * 32 + j];
        partial[(size_t)blockIdx.x * 2 + threadIdx.x] = s;
    }
}

// u -= sum_{i<K} coef[i] A_i  (and the same on a second pair when B is not NULL:
// ub -= sum coef[i] B_i), coefficients read on the device.
__global__ void k_subtract(const double *A, const double *B, size_t ld, int K, const double *coef, int64_t N,
                           double *u, double *ub)
{
    double cf[LRED];
#pragma unroll
    for (int i = 0; i < LRED; ++i) cf[i] = (i < K) ? coef[i] : 0.0;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x) {
        double s = u[d], sb = ub ? ub[d] : 0.0;
#pragma unroll
        for (int i = 0; i < LRED; ++i)
            if (i < K) {
                s -= cf[i] * A[i * ld + d];
                if (ub) sb -= cf[i] * B[i * ld + d];
            }
        u[d] = s;
        if (ub) ub[d] = sb;
    }
}

// u = src * scale(norm2), scale = 1/sqrt(norm2[0]); optional second vector.
__global__ void k_scale_copy(const double *src, const double *src2, const double *norm2, int64_t N, double *u,
                             double *u2, float *u32)
{
    const double s = 1.0 / sqrt(norm2[0]);
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x) {
        double v = src[d] * s;
        u[d] = v;
        if (u2) u2[d] = src2[d] * s;
        if (u32) u32[d] = (float)v;
    }
}

__global__ void k_to_float(const double *src, int64_t N, float *dst)
{
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x)
        dst[d] = (float)src[d];
}

__global__ void k_copy2(const double *a, const double *b, int64_t N, double *ca, double *cb)
{
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x) {
        ca[d] = a[d];
        cb[d] = b[d];
    }
}

// start vector: lowest diagonal element (index given) + fixed admixture
__global__ void k_large_guess(const int64_t *best, int Ns, int sgn, int64_t N, double *x)
{
    const SectorGuess sg{(int)best[0], sgn};
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x)
        x[d] = sector_guess((int)d, Ns, sg);
}

// index of the smallest diagonal element (ties -> lowest index), optionally
// among the determinants with Ia != Ib only; one block
__global__ void k_argmin(const double *diag, int64_t N, int Ns, int open_only, int64_t *out)
{
    __shared__ double bv[32];
    __shared__ int64_t bix[32];
    double best = 1e300;
    int64_t bi = INT64_MAX;
    for (int64_t d = threadIdx.x; d < N; d += blockDim.x) {
        if (open_only && d / Ns == d % Ns) continue;
        double v = diag[d];
        if (v < best || (v == best && d < bi)) {
            best = v;
            bi = d;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(FULL, best, o);
        int64_t oi = __shfl_xor_sync(FULL, bi, o);
        if (ov < best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        bv[w] = best;
        bix[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j)
            if (bv[j] < best || (bv[j] == best && bix[j] < bi)) {
                best = bv[j];
                bi = bix[j];
            }
        out[0] = bi;
    }
}

// Projected eigenproblem (one warp) and bookkeeping of G on the device.
__global__ void k_large_small_eig(const double *Gd, int m, double *ys, double *y2s, double *misc)
{
    __shared__ double G[MMAX * MMAX];
    __shared__ float A[MMAX * MMAX], E[MMAX * MMAX], ev[MMAX];
    __shared__ double r[MMAX];
    for (int e = threadIdx.x; e < MMAX * MMAX; e += 32) G[e] = Gd[e];
    __syncwarp();
    small_eig_warp<true>(G, m, A, E, ev, ys, y2s, r, misc);
}

// G column m (and row m) from the dots in `dots` (m + 1 values)
__global__ void k_set_gcol(double *Gd, int m, const double *dots)
{
    int i = threadIdx.x;
    if (i <= m) {
        Gd[i * MMAX + m] = dots[i];
        Gd[m * MMAX + i] = dots[i];
    }
}

__global__ void k_set_g2(double *Gd, const double *dots, int two)
{
    if (threadIdx.x == 0) {
        Gd[0] = dots[0];
        if (two) {
            Gd[1] = Gd[MMAX] = dots[1];
            Gd[MMAX + 1] = dots[2];
        }
    }
}

}  // namespace mbe

namespace mbe {

struct LargePlan {
    LargeCas L;
    int grid_ab64, grid_ss64, grid_ss32, grid_vec, grid_tr;
    size_t smem_ab64, smem_ss64, smem_ss32;
    void *cT;      // transposed coefficients (room for N float64)
};


// Sets up one large CAS; the dense Hs may live in `dense_at` (e.g. the Davidson
// basis region, unused during set-up). `fp32` adds the float32 sigma's tables.
static int large_setup(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ, int n_cas,
                       const int32_t *cas_orbs, Bump &bump, double *dense_at, bool fp32, LargePlan *plan, int *k_out,
                       int64_t *dphi_out)
{
    MBE_CHECK(n_cas >= 1 && n_cas <= MBE_MAX_STRING_ORB && n_cas <= norb, MBE_EUNSUPPORTED,
              "large CASCI: n_cas %d outside 1..%d", n_cas, MBE_MAX_STRING_ORB);
    std::vector<int> A(cas_orbs, cas_orbs + n_cas);
    std::sort(A.begin(), A.end());
    for (int i = 0; i < n_cas; ++i)
        MBE_CHECK(A[i] >= 0 && A[i] < norb && (i == 0 || A[i] != A[i - 1]), MBE_EINVAL,
                  "large CASCI: active orbital %d out of range or repeated", A[i]);
    std::vector<uint8_t> occ_h(norb);
    MBE_CU(cudaMemcpyAsync(occ_h.data(), occ, norb, cudaMemcpyDeviceToHost, ctx->stream));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    int k = 0;
    uint32_t mphi = 0;
    for (int i = 0; i < n_cas; ++i)
        if (occ_h[A[i]]) {
            ++k;
            mphi |= 1u << i;
        }
    const StringTable *st = nullptr;
    int rc = get_table(ctx, n_cas, k, &st);
    if (rc) return rc;
    LargeCas &L = plan->L;
    L.n = n_cas;
    L.P = n_cas * (n_cas + 1) / 2;
    L.k = k;
    L.Ns = (int)st->ns;
    L.R = st->r;
    L.N = st->ns * st->ns;
    L.str = st->strings;
    L.tab = st->table;
    const int P = L.P;
    const int64_t conn = 1 + (int64_t)k * (n_cas - k) + binom(k, 2) * binom(n_cas - k, 2);
    double *F = bump.take<double>((size_t)norb * norb);
    L.V = bump.take<double>((size_t)P * P);
    L.V32 = bump.take<float>((size_t)P * P);
    L.hp = bump.take<double>(P);
    L.pp = bump.take<short>(2 * P);
    L.roff = bump.take<int64_t>((size_t)L.Ns + 1);
    L.col = bump.take<int32_t>((size_t)L.Ns * conn);
    L.val = bump.take<double>((size_t)L.Ns * conn);
    L.val32 = bump.take<float>((size_t)L.Ns * conn);
    L.diag = bump.take<double>((size_t)L.N);
    int32_t *cnt = bump.take<int32_t>((size_t)L.Ns);
    int64_t *off = bump.take<int64_t>((size_t)L.Ns + 1);
    int32_t *tabT = bump.take<int32_t>((size_t)L.R * L.Ns);
    L.tabT = tabT;
    plan->cT = bump.take<double>((size_t)L.N);  // float32 or float64 use
    L.Hd = dense_at ? dense_at : bump.take<double>((size_t)L.Ns * L.Ns);
    // (all of the above fits: the caller sized the workspace with large_bytes)
    k_core_fock<<<(norb * norb + 127) / 128, 128, 0, ctx->stream>>>(norb, h1, eri, occ, F);
    LargeSetupArgs sa;
    memset(&sa, 0, sizeof(sa));
    for (int i = 0; i < n_cas; ++i) sa.A[i] = A[i];
    sa.norb = norb;
    sa.eri = eri;
    sa.occ = occ;
    sa.F = F;
    k_large_setup<<<1, CTA_THREADS, 0, ctx->stream>>>(sa, L);
    k_large_hs_cols<<<(L.Ns + 127) / 128, 128, 0, ctx->stream>>>(L);
    const unsigned wgrid = (unsigned)(((int64_t)L.Ns * 32 + 255) / 256);
    k_large_hs_count<<<wgrid, 256, 0, ctx->stream>>>(L, cnt);
    k_scan_counts<<<1, 256, 0, ctx->stream>>>(cnt, L.Ns, off);
    k_large_hs_fill<<<wgrid, 256, 0, ctx->stream>>>(L, off);
    k_large_diag<<<ctx->sm_count * 8, 256, 0, ctx->stream>>>(L);
    k_large_tables<<<(L.Ns + 255) / 256, 256, 0, ctx->stream>>>(L, tabT);
    MBE_CU(cudaGetLastError());
    ctx->launches += 8;
    *k_out = k;
    int iphi = string_rank(mphi);
    *dphi_out = (int64_t)iphi * L.Ns + iphi;
    // launch shapes
    plan->smem_ab64 = (size_t)P * P * 8;
    MBE_CHECK(plan->smem_ab64 <= ctx->smem_optin, MBE_EUNSUPPORTED, "large CASCI: V needs %zu B shared memory",
              plan->smem_ab64);
    MBE_CU(cudaFuncSetAttribute(k_large_ab64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem_ab64));
    MBE_CU(cudaFuncSetAttribute(k_large_ab64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem_ab64));
    int b = 0;
    MBE_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_large_ab64<false>, SIGMA_THREADS, plan->smem_ab64));
    plan->grid_ab64 = ctx->sm_count * (b > 0 ? b : 1);
    plan->smem_ss64 = (size_t)SS_ROWS * (SS_TK + 1) * 8;
    plan->smem_ss32 = (size_t)SS_ROWS * (SS_TK + 1) * 4;
    MBE_CU(cudaFuncSetAttribute(k_large_ss<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)plan->smem_ss64));
    MBE_CU(cudaFuncSetAttribute(k_large_ss<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)plan->smem_ss64));
    MBE_CU(cudaFuncSetAttribute(k_large_ss<double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)plan->smem_ss64));
    MBE_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_large_ss<double, false>, SS_THREADS, plan->smem_ss64));
    plan->grid_ss64 = ctx->sm_count * (b > 0 ? b : 1);
    MBE_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_large_ss<float, false>, SS_THREADS, plan->smem_ss32));
    plan->grid_ss32 = ctx->sm_count * (b > 0 ? b : 1);
    plan->grid_tr = ctx->sm_count * 8;
    plan->grid_vec = ctx->sm_count * 4;
    return MBE_OK;
}

// Workspace bytes of large_setup (and the dense Hs unless aliased).
static size_t large_bytes(int norb, int n, int k, bool dense_separate, bool fp32)
{
    const int64_t ns = binom(n, k), N = ns * ns;
    const int P = n * (n + 1) / 2;
    const int64_t conn = 1 + (int64_t)k * (n - k) + binom(k, 2) * binom(n - k, 2);
    size_t b = align256((size_t)norb * norb * 8) + align256((size_t)P * P * 8) + align256((size_t)P * P * 4) +
               align256(P * 8) + align256(2 * P * 2) + align256((ns + 1) * 8) + align256(ns * conn * 4) +
               align256(ns * conn * 8) + align256(ns * conn * 4) + align256(N * 8) + align256(ns * 4) +
               align256((ns + 1) * 8) + 4096;
    b += align256((size_t)k * (n - k + 1) * ns * 4) + align256((size_t)N * 8);
    if (dense_separate) b += align256((size_t)ns * ns * 8);
    return b;
}

// sigma = H c: the opposite-spin term written first, then Hs C added, then C Hs^T
// added through the transposed copy of c.
template <typename T>
static int large_sigma_launch(mbe_ctx *ctx, const LargePlan &pl, const T *c, double *sigma, int order_tag,
                              int sgn = 0)
{
    TimedLaunch tl(ctx, order_tag, 2, sizeof(T) == 8 ? 64 : 32);
    const int Ns = pl.L.Ns;
    if (sizeof(T) == 8) {
        if (sgn == 0)
            k_large_ab64<false><<<pl.grid_ab64, SIGMA_THREADS, pl.smem_ab64, ctx->stream>>>(pl.L, (const double *)c,
                                                                                          sigma, 0);
        else
            k_large_ab64<true><<<pl.grid_ab64, SIGMA_THREADS, pl.smem_ab64, ctx->stream>>>(pl.L, (const double *)c,
                                                                                         sigma, sgn);
    } else {
        // the dense product on the tensor cores (large_tc.cu)
        const int rc = large_ab_tc(ctx->stream, ctx->sm_count, ctx->smem_optin, pl.L.P, pl.L.Ns, pl.L.R, pl.L.tab,
                                   pl.L.V32, (const float *)c, sigma, ctx->dev_err);
        if (rc) return rc;
    }
    const int grid_ss = sizeof(T) == 8 ? pl.grid_ss64 : pl.grid_ss32;
    const size_t smem_ss = sizeof(T) == 8 ? pl.smem_ss64 : pl.smem_ss32;
    if (sgn == 0) {
        T *cT = (T *)pl.cT;
        k_large_ss<T, false><<<grid_ss, SS_THREADS, smem_ss, ctx->stream>>>(pl.L, c, sigma);
        k_large_transpose<T><<<pl.grid_tr, dim3(32, 8), 0, ctx->stream>>>(c, Ns, cT);
        k_large_ss<T, true><<<grid_ss, SS_THREADS, smem_ss, ctx->stream>>>(pl.L, cT, sigma);
    } else {
        // c in the sector sgn: the beta same-spin term is sgn times the transpose
        // of the alpha one, so one product (into the spare buffer) and a
        // transposing add replace the second product and the transpose of c
        double *A = (double *)pl.cT;
        k_large_ss<T, false, true><<<grid_ss, SS_THREADS, smem_ss, ctx->stream>>>(pl.L, c, A);
        k_sym_add<<<pl.grid_tr, dim3(32, 8), 0, ctx->stream>>>(A, Ns, sgn, sigma);
    }
    MBE_CU(cudaGetLastError());
    ctx->launches += sgn == 0 ? 4 : 3;
    return tl.done();
}

}  // namespace mbe

extern "C" int casci_sigma_large(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                                 int n_cas, const int32_t *cas_orbs, int precision, const double *c,
                                 double *sigma, double *diag)
{
    MBE_CHECK(ctx && h1 && eri && occ && cas_orbs && c && sigma, MBE_EINVAL, "casci_sigma_large: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "casci_sigma_large: norb %d", norb);
    MBE_CHECK(precision == MBE_PREC_FP64 || precision == MBE_PREC_MIXED, MBE_EINVAL,
              "casci_sigma_large: precision %d", precision);
    MBE_CU(cudaSetDevice(ctx->device));
    // occupation count first (sizes depend on it)
    std::vector<uint8_t> occ_h(norb);
    MBE_CU(cudaMemcpyAsync(occ_h.data(), occ, norb, cudaMemcpyDeviceToHost, ctx->stream));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    MBE_CHECK(n_cas >= 1 && n_cas <= MBE_MAX_STRING_ORB && n_cas <= norb, MBE_EUNSUPPORTED,
              "casci_sigma_large: n_cas %d outside 1..%d", n_cas, MBE_MAX_STRING_ORB);
    int k0 = 0;
    for (int i = 0; i < n_cas; ++i) k0 += (cas_orbs[i] >= 0 && cas_orbs[i] < norb && occ_h[cas_orbs[i]]) ? 1 : 0;
    const int64_t N = binom(n_cas, k0) * binom(n_cas, k0);
    const bool fp32 = precision == MBE_PREC_MIXED;
    size_t bytes = large_bytes(norb, n_cas, k0, true, fp32) + (fp32 ? align256(N * 4) : 0);
    void *ws = nullptr;
    int rc = workspace(ctx, bytes, &ws);
    if (rc) return rc;
    Bump bump(ws);
    LargePlan pl;
    int k = 0;
    int64_t dphi = 0;
    rc = large_setup(ctx, norb, h1, eri, occ, n_cas, cas_orbs, bump, nullptr, fp32, &pl, &k, &dphi);
    if (rc) return rc;
    if (diag) MBE_CU(cudaMemcpyAsync(diag, pl.L.diag, N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (precision == MBE_PREC_FP64) return large_sigma_launch<double>(ctx, pl, c, sigma, n_cas);
    float *c32 = bump.take<float>((size_t)N);
    k_to_float<<<pl.grid_vec, 256, 0, ctx->stream>>>(c, N, c32);
    ++ctx->launches;
    rc = large_sigma_launch<float>(ctx, pl, c32, sigma, n_cas);
    if (rc) return rc;
    return check_dev_err(ctx);  // the tensor-core product reports a wait that ran out
}

namespace mbe {

// x2 = V y2, hx2 = W y2 over the first m basis vectors
__global__ void k_lincomb2(const double *V, const double *W, size_t ld, int m, const double *ys, int64_t N,
                           double *x2, double *hx2)
{
    double y[MLARGE];
#pragma unroll
    for (int i = 0; i < MLARGE; ++i) y[i] = (i < m) ? ys[i] : 0.0;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x) {
        double xs = 0.0, hs = 0.0;
#pragma unroll
        for (int i = 0; i < MLARGE; ++i)
            if (i < m) {
                xs += y[i] * V[i * ld + d];
                hs += y[i] * W[i * ld + d];
            }
        x2[d] = xs;
        hx2[d] = hs;
    }
}

// Projects v onto the spin-flip sector sgn (v[Ia][Ib] = sgn v[Ib][Ia]), pairs
// (d, P d) averaged: the large solver's sigma is not formed over a half space,
// so its rounding would otherwise let the other sector's lower states leak in.
__global__ void k_project_sector(double *v, int Ns, int sgn, int64_t N)
{
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x) {
        const int ia = (int)(d / Ns), ib = (int)(d - (int64_t)ia * Ns);
        if (ia == ib) {
            if (sgn < 0) v[d] = 0.0;
        } else if (ia < ib) {
            const int64_t pd = (int64_t)ib * Ns + ia;
            const double m = 0.5 * (v[d] + sgn * v[pd]);
            v[d] = m;
            v[pd] = sgn * m;
        }
    }
}

// w -= shift * v  (the image of a correction under H - theta0)
__global__ void k_shift_image(const double *v, double shift, int64_t N, double *w)
{
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x)
        w[d] -= shift * v[d];
}

// Thick restart that keeps the anchor V[0], W[0]: u1 = sum_{i>=1} y_i V_i and
// u2 = sum_{i>=1} y2_i V_i (the corrections of the two lowest Ritz vectors) and
// their images.
__global__ void k_anchor_restart(const double *V, const double *W, size_t ld, int m, const double *ys,
                                 const double *y2s, int64_t N, double *u1, double *w1, double *u2, double *w2)
{
    double y[MLARGE], y2[MLARGE];
#pragma unroll
    for (int i = 0; i < MLARGE; ++i) {
        y[i] = (i >= 1 && i < m) ? ys[i] : 0.0;
        y2[i] = (i >= 1 && i < m) ? y2s[i] : 0.0;
    }
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < N; d += (int64_t)gridDim.x * blockDim.x) {
        double a = 0.0, b = 0.0, c = 0.0, e = 0.0;
#pragma unroll
        for (int i = 1; i < MLARGE; ++i) {
            const double v = V[i * ld + d], w = W[i * ld + d];
            a += y[i] * v;
            b += y[i] * w;
            c += y2[i] * v;
            e += y2[i] * w;
        }
        u1[d] = a;
        w1[d] = b;
        u2[d] = c;
        w2[d] = e;
    }
}

// G entries of the anchored restart basis {V0, V1, V2} from dots = [W0.V1, V1.W1,
// W0.V2, V1.W2, V2.W2] (G00 kept); two = 0 when V2 was dropped.
__global__ void k_set_g3(double *Gd, const double *dots, int two)
{
    if (threadIdx.x == 0) {
        Gd[1] = Gd[MMAX] = dots[0];
        Gd[MMAX + 1] = dots[1];
        if (two) {
            Gd[2] = Gd[2 * MMAX] = dots[2];
            Gd[MMAX + 2] = Gd[2 * MMAX + 1] = dots[3];
            Gd[2 * MMAX + 2] = dots[4];
        }
    }
}

struct LargeDav {
    double *V, *W, *x, *hx, *t, *x2, *hx2, *xs, *partial, *dots, *Gd, *ys, *y2s, *misc;
    float *c32;
    int64_t *best;
    size_t ld;
    int nblk;
};

static void dot_to(mbe_ctx *ctx, const LargePlan &pl, const LargeDav &D, const double *A, int K, const double *u,
                   double *out)
{
    k_multidot<<<D.nblk, LARGE_THREADS, 0, ctx->stream>>>(A, D.ld, K, u, pl.L.N, D.partial);
    k_multidot_final<<<1, 32 * K, 0, ctx->stream>>>(D.partial, D.nblk, K, out);
    ctx->launches += 2;
}

template <typename T>
static int large_apply(mbe_ctx *ctx, const LargePlan &pl, const LargeDav &D, const double *vin, double *wout,
                       int sgn)
{
    if (sizeof(T) == 8) return large_sigma_launch<double>(ctx, pl, vin, wout, pl.L.n, sgn);
    k_to_float<<<pl.grid_vec, 256, 0, ctx->stream>>>(vin, pl.L.N, D.c32);
    ++ctx->launches;
    return large_sigma_launch<float>(ctx, pl, D.c32, wout, pl.L.n, sgn);
}

// One Davidson phase on the large space (T = sigma arithmetic).  D.x: start
// vector in, Ritz vector out.
// Anchored (anchor != NULL, T = float; see struct Anchor): D.x is the anchor x0;
// one float64 sigma gives theta0 = x0.Hx0 and the exact image W0 = (H - theta0) x0
// of V0 = x0; every later basis vector is a correction whose image is the float32
// sigma minus theta0 times it; the coupling of x0 to V_m is formed as W0.V_m; a
// thick restart keeps V0; *lambda returns theta0 + mu, *anchor_y0 the coefficient
// of x0 in the Ritz vector (which is left in D.x, float64).
template <typename T>
static int large_phase(mbe_ctx *ctx, const LargePlan &pl, const LargeDav &D, int sgn, double tol, int min_iter,
                       int max_iter, int steer, double *lambda, double *rnorm, int *nsig, int *status,
                       int *nsig64 = nullptr, double *anchor_y0 = nullptr)
{
    const int64_t N = pl.L.N;
    const size_t ld = D.ld;
    cudaStream_t st = ctx->stream;
    const int g = pl.grid_vec;
    const bool anch = sizeof(T) == 4 && anchor_y0 != nullptr;
    double h3[4];
    *nsig = 0;
    *status = MBE_STATUS_OK;
    int rc;
    double shift = 0.0;
    const int Ns = pl.L.Ns;
    k_project_sector<<<g, 256, 0, st>>>(D.x, Ns, sgn, N);
    dot_to(ctx, pl, D, D.x, 1, D.x, D.dots);
    k_scale_copy<<<g, 256, 0, st>>>(D.x, nullptr, D.dots, N, D.V, nullptr, nullptr);
    ctx->launches += 2;
    if (anch) {
        if ((rc = large_sigma_launch<double>(ctx, pl, D.V, D.W, pl.L.n, sgn))) return rc;
        ++*nsig64;
        k_project_sector<<<g, 256, 0, st>>>(D.W, Ns, sgn, N);
        ++ctx->launches;
        dot_to(ctx, pl, D, D.W, 1, D.V, D.dots);
        MBE_CU(cudaMemcpyAsync(&shift, D.dots, 8, cudaMemcpyDeviceToHost, st));
        MBE_CU(cudaStreamSynchronize(st));
        k_shift_image<<<g, 256, 0, st>>>(D.V, shift, N, D.W);
        ++ctx->launches;
    } else {
        if ((rc = large_apply<T>(ctx, pl, D, D.V, D.W, sgn))) return rc;
        ++*nsig;
    }
    k_project_sector<<<g, 256, 0, st>>>(D.W, Ns, sgn, N);
    ++ctx->launches;
    dot_to(ctx, pl, D, D.W, 1, D.V, D.dots);
    k_set_g2<<<1, 32, 0, st>>>(D.Gd, D.dots, 0);
    ++ctx->launches;
    int m = 1;
    double best = 3e38;
    int stall = 0;
    for (int it = 0;; ++it) {
        k_large_small_eig<<<1, 32, 0, st>>>(D.Gd, m, D.ys, D.y2s, D.misc);
        double *tdst = (m < MLARGE) ? D.V + (size_t)m * ld : D.t;
        k_ritz<<<D.nblk, LARGE_THREADS, 0, st>>>(D.V, D.W, ld, m, D.ys, D.misc, pl.L.diag, shift, N, D.x, D.hx,
                                                 tdst, D.partial);
        k_multidot_final<<<1, 64, 0, st>>>(D.partial, D.nblk, 2, D.dots);
        ctx->launches += 3;
        int herr = 0;
        MBE_CU(cudaMemcpyAsync(h3, D.dots, 16, cudaMemcpyDeviceToHost, st));
        MBE_CU(cudaMemcpyAsync(h3 + 2, D.misc, 8, cudaMemcpyDeviceToHost, st));
        MBE_CU(cudaMemcpyAsync(h3 + 3, D.ys, 8, cudaMemcpyDeviceToHost, st));
        MBE_CU(cudaMemcpyAsync(&herr, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        MBE_CU(cudaStreamSynchronize(st));
        if (herr) return check_dev_err(ctx);
        const double rn = sqrt(h3[0]), t0n = sqrt(h3[1]);
        *lambda = shift + h3[2];
        *rnorm = rn;
        if (anch) *anchor_y0 = h3[3];
        if (!std::isfinite(rn) || !std::isfinite(h3[2])) {
            *status = MBE_STATUS_NONFINITE;
            break;
        }
        if (rn <= tol && it >= min_iter) break;
        if (it >= max_iter) {
            *status = MBE_STATUS_MAXITER;
            break;
        }
        if (steer) {
            if (rn < 0.9 * best) {
                best = rn;
                stall = 0;
            } else if (++stall >= steer) {
                break;
            }
        }
        double *u = D.V + (size_t)m * ld;
        if (m == MLARGE && anch) {
            // keep V0 = x0, W0 = r0; V1, V2: corrections of the two lowest Ritz vectors
            // (D.t holds the new correction; D.x, D.hx are recomputed by the next k_ritz)
            k_anchor_restart<<<g, 256, 0, st>>>(D.V, D.W, ld, m, D.ys, D.y2s, N, D.x2, D.hx2, D.x, D.hx);
            k_copy2<<<g, 256, 0, st>>>(D.x2, D.hx2, N, D.V + ld, D.W + ld);
            ctx->launches += 2;
            dot_to(ctx, pl, D, D.V + ld, 1, D.V + ld, D.dots);
            k_scale_copy<<<g, 256, 0, st>>>(D.V + ld, D.W + ld, D.dots, N, D.V + ld, D.W + ld, nullptr);
            k_copy2<<<g, 256, 0, st>>>(D.x, D.hx, N, D.V + 2 * ld, D.W + 2 * ld);
            ctx->launches += 2;
            for (int pass = 0; pass < 2; ++pass) {
                dot_to(ctx, pl, D, D.V + ld, 1, D.V + 2 * ld, D.dots);
                k_subtract<<<g, 256, 0, st>>>(D.V + ld, D.W + ld, ld, 1, D.dots, N, D.V + 2 * ld, D.W + 2 * ld);
                ++ctx->launches;
            }
            dot_to(ctx, pl, D, D.V + 2 * ld, 1, D.V + 2 * ld, D.dots);
            MBE_CU(cudaMemcpyAsync(h3, D.dots, 8, cudaMemcpyDeviceToHost, st));
            MBE_CU(cudaStreamSynchronize(st));
            const int two = sqrt(h3[0]) > 1e-3 ? 1 : 0;
            if (two) {
                k_scale_copy<<<g, 256, 0, st>>>(D.V + 2 * ld, D.W + 2 * ld, D.dots, N, D.V + 2 * ld, D.W + 2 * ld,
                                                 nullptr);
                ++ctx->launches;
            }
            dot_to(ctx, pl, D, D.W, 1, D.V + ld, D.dots);               // W0.V1
            dot_to(ctx, pl, D, D.V + ld, 1, D.W + ld, D.dots + 1);      // V1.W1
            if (two) {
                dot_to(ctx, pl, D, D.W, 1, D.V + 2 * ld, D.dots + 2);   // W0.V2
                dot_to(ctx, pl, D, D.V + ld, 1, D.W + 2 * ld, D.dots + 3);  // V1.W2
                dot_to(ctx, pl, D, D.V + 2 * ld, 1, D.W + 2 * ld, D.dots + 4);  // V2.W2
            }
            k_set_g3<<<1, 32, 0, st>>>(D.Gd, D.dots, two);
            ++ctx->launches;
            m = 2 + two;
            u = D.V + (size_t)m * ld;
            MBE_CU(cudaMemcpyAsync(u, D.t, (size_t)N * 8, cudaMemcpyDeviceToDevice, st));
        } else if (m == MLARGE) {
            // thick restart on the two lowest Ritz vectors (orthogonal by construction)
            k_lincomb2<<<g, 256, 0, st>>>(D.V, D.W, ld, m, D.y2s, N, D.x2, D.hx2);
            k_copy2<<<g, 256, 0, st>>>(D.x, D.hx, N, D.V, D.W);
            k_copy2<<<g, 256, 0, st>>>(D.x2, D.hx2, N, D.V + ld, D.W + ld);
            ctx->launches += 3;
            for (int pass = 0; pass < 2; ++pass) {
                dot_to(ctx, pl, D, D.V, 1, D.V + ld, D.dots);
                k_subtract<<<g, 256, 0, st>>>(D.V, D.W, ld, 1, D.dots, N, D.V + ld, D.W + ld);
                ++ctx->launches;
            }
            dot_to(ctx, pl, D, D.V + ld, 1, D.V + ld, D.dots);
            k_scale_copy<<<g, 256, 0, st>>>(D.V + ld, D.W + ld, D.dots, N, D.V + ld, D.W + ld, nullptr);
            dot_to(ctx, pl, D, D.W, 2, D.V, D.dots);
            dot_to(ctx, pl, D, D.W + ld, 1, D.V + ld, D.dots + 2);
            k_set_g2<<<1, 32, 0, st>>>(D.Gd, D.dots, 1);
            ctx->launches += 2;
            m = 2;
            u = D.V + (size_t)m * ld;
            MBE_CU(cudaMemcpyAsync(u, D.t, (size_t)N * 8, cudaMemcpyDeviceToDevice, st));
        }
        k_project_sector<<<g, 256, 0, st>>>(u, Ns, sgn, N);
        ++ctx->launches;
        for (int pass = 0; pass < 2; ++pass) {
            dot_to(ctx, pl, D, D.V, m, u, D.dots);
            k_subtract<<<g, 256, 0, st>>>(D.V, nullptr, ld, m, D.dots, N, u, nullptr);
            ++ctx->launches;
        }
        dot_to(ctx, pl, D, u, 1, u, D.dots);
        MBE_CU(cudaMemcpyAsync(h3, D.dots, 8, cudaMemcpyDeviceToHost, st));
        MBE_CU(cudaStreamSynchronize(st));
        const double tn = sqrt(h3[0]);
        if (!(tn > 1e-12 * t0n) || !(tn > 0.0)) {
            if (!steer && rn > tol) *status = MBE_STATUS_MAXITER;
            break;
        }
        k_scale_copy<<<g, 256, 0, st>>>(u, nullptr, D.dots, N, u, nullptr, nullptr);
        ++ctx->launches;
        if ((rc = large_apply<T>(ctx, pl, D, u, D.W + (size_t)m * ld, sgn))) return rc;
        ++*nsig;
        k_project_sector<<<g, 256, 0, st>>>(D.W + (size_t)m * ld, Ns, sgn, N);
        ++ctx->launches;
        if (anch) {
            k_shift_image<<<g, 256, 0, st>>>(u, shift, N, D.W + (size_t)m * ld);
            ++ctx->launches;
        }
        dot_to(ctx, pl, D, D.V, m + 1, D.W + (size_t)m * ld, D.dots);
        if (anch) dot_to(ctx, pl, D, D.W, 1, u, D.dots);  // x0.(A u) as u.r0
        k_set_gcol<<<1, 32, 0, st>>>(D.Gd, m, D.dots);
        ++ctx->launches;
        ++m;
    }
    return MBE_OK;
}

}  // namespace mbe

extern "C" int casci_solve(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                           int n_cas, const int32_t *cas_orbs, const mbe_opts *opts, double *result,
                           int32_t *info, double *cvec)
{
    MBE_CHECK(ctx && h1 && eri && occ && cas_orbs && result && info, MBE_EINVAL, "casci_solve: NULL argument");
    MBE_CHECK(norb >= 1 && norb <= MBE_MAX_NORB, MBE_EINVAL, "casci_solve: norb %d", norb);
    MBE_CHECK(n_cas >= 1 && n_cas <= MBE_MAX_STRING_ORB && n_cas <= norb, MBE_EUNSUPPORTED,
              "casci_solve: n_cas %d outside 1..%d", n_cas, MBE_MAX_STRING_ORB);
    mbe_opts o;
    if (opts) o = *opts; else mbe_default_opts(&o);
    MBE_CHECK(o.precision == MBE_PREC_FP64 || o.precision == MBE_PREC_MIXED, MBE_EINVAL,
              "casci_solve: unknown precision %d", o.precision);
    MBE_CHECK(o.tol > 0 && o.tol_switch > 0 && o.max_iter >= 1 && o.fp64_final_iters >= 0 &&
                  (o.sectors == MBE_SECTORS_BOTH || o.sectors == MBE_SECTORS_EVEN), MBE_EINVAL,
              "casci_solve: bad options");
    MBE_CHECK(o.s2_penalty == 0.0, MBE_EUNSUPPORTED, "casci_solve: the S^2 penalty is not supported for one large CAS");
    MBE_CU(cudaSetDevice(ctx->device));
    std::vector<uint8_t> occ_h(norb);
    MBE_CU(cudaMemcpyAsync(occ_h.data(), occ, norb, cudaMemcpyDeviceToHost, ctx->stream));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    int k0 = 0;
    for (int i = 0; i < n_cas; ++i) k0 += (cas_orbs[i] >= 0 && cas_orbs[i] < norb && occ_h[cas_orbs[i]]) ? 1 : 0;
    const int64_t N = binom(n_cas, k0) * binom(n_cas, k0);
    const size_t vec = align256((size_t)N * 8);
    LargeDav D;
    D.ld = vec / 8;
    D.nblk = ctx->sm_count * 4;
    const bool mixed = o.precision == MBE_PREC_MIXED;
    size_t bytes = large_bytes(norb, n_cas, k0, false, mixed) + vec * (2 * MLARGE + 6) + align256((size_t)N * 4) +
                   align256((size_t)D.nblk * LRED * 8) + 8 * 256 + 4096;
    void *ws = nullptr;
    int rc = workspace(ctx, bytes, &ws);
    if (rc) return rc;
    Bump bump(ws);
    D.V = bump.take<double>(D.ld * MLARGE);
    D.W = bump.take<double>(D.ld * MLARGE);
    D.x = bump.take<double>(D.ld);
    D.hx = bump.take<double>(D.ld);
    D.t = bump.take<double>(D.ld);
    D.x2 = bump.take<double>(D.ld);
    D.hx2 = bump.take<double>(D.ld);
    D.xs = bump.take<double>(D.ld);
    D.c32 = bump.take<float>((size_t)N);
    D.partial = bump.take<double>((size_t)D.nblk * LRED);
    D.dots = bump.take<double>(32);
    D.Gd = bump.take<double>(MMAX * MMAX);
    D.ys = bump.take<double>(MMAX);
    D.y2s = bump.take<double>(MMAX);
    D.misc = bump.take<double>(8);
    D.best = bump.take<int64_t>(4);
    LargePlan pl;
    int k = 0;
    int64_t dphi = 0;
    // The dense one-spin Hamiltonian of the set-up lives in the (not yet used) basis region.
    rc = large_setup(ctx, norb, h1, eri, occ, n_cas, cas_orbs, bump, D.V, mixed, &pl, &k, &dphi);
    if (rc) return rc;
    const int Ns = pl.L.Ns;
    k_argmin<<<1, 1024, 0, ctx->stream>>>(pl.L.diag, N, Ns, 0, D.best);
    k_argmin<<<1, 1024, 0, ctx->stream>>>(pl.L.diag, N, Ns, 1, D.best + 1);
    ctx->launches += 2;
    double lam = 0.0, rn = 0.0;
    int n32 = 0, n64 = 0, st = 0;
    bool degen = false;
    // the two spin-flip sectors (see sector_guess); each runs the float32 phase
    // (mixed mode) and the float64 phase; the second sector first runs a float64
    // pass to the residual SECTOR_TOL only and stops there when sector_loses
    for (int sector = 0; sector < 2; ++sector) {
        if (sector == 1 && (Ns < 2 || st != MBE_STATUS_OK || o.sectors == MBE_SECTORS_EVEN)) break;
        const int sgn = sector == 0 ? 1 : -1;
        if (sector == 1) MBE_CU(cudaMemcpyAsync(D.xs, D.x, (size_t)N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        k_large_guess<<<pl.grid_vec, 256, 0, ctx->stream>>>(D.best + sector, Ns, sgn, N, D.x);
        ++ctx->launches;
        double l = 0.0, r = 0.0;
        int s64 = 0, s32 = 0, ss = MBE_STATUS_OK;
        bool lose = false, refined = false;
        if (mixed) {
            // float32 phase (tensor-core sigma), then anchored refinements (struct
            // Anchor): one float64 sigma per anchor, float32 sigmas for the
            // corrections; the second sector is decided once its residual reaches
            // SECTOR_TOL. A refinement that fails hands over to the float64 phase.
            int n = 0;
            rc = large_phase<float>(ctx, pl, D, sgn, o.tol_switch, 0, o.max_iter, 3, &l, &r, &n, &ss);
            if (rc) return rc;
            s32 += n;
            bool decided = sector == 0;
            if (ss == MBE_STATUS_NONFINITE) {
                k_large_guess<<<pl.grid_vec, 256, 0, ctx->stream>>>(D.best + sector, Ns, sgn, N, D.x);
                ++ctx->launches;
            } else {
                for (int anc = 0; anc < LARGE_ANCHORS && !lose && !refined; ++anc) {
                    const double tgt = decided ? o.tol : SECTOR_TOL;
                    double y0 = 1.0;
                    int n64a = 0;
                    n = 0;
                    rc = large_phase<float>(ctx, pl, D, sgn, tgt, decided ? o.fp64_final_iters : 0, o.max_iter,
                                            LARGE_ANCHOR_STALL, &l, &r, &n, &ss, &n64a, &y0);
                    if (rc) return rc;
                    s32 += n;
                    s64 += n64a;
                    if (ss == MBE_STATUS_NONFINITE) break;
                    if (!decided && r <= SECTOR_TOL) {
                        decided = true;
                        lose = sector_loses(l, r, lam, 0.0);
                        continue;
                    }
                    const double dn = sqrt(std::max(0.0, 1.0 - y0 * y0)) / std::max(fabs(y0), 1e-300);
                    refined = decided && r <= o.tol && dn <= MIX_DMAX;
                }
            }
        } else if (sector == 1) {
            // a float64 pass from the start vector to SECTOR_TOL decides
            int n = 0;
            rc = large_phase<double>(ctx, pl, D, sgn, SECTOR_TOL, 0, o.max_iter, LARGE_STALL, &l, &r, &n, &ss);
            if (rc) return rc;
            s64 += n;
            lose = ss == MBE_STATUS_NONFINITE || sector_loses(l, r, lam, 0.0);
        }
        if (refined) ss = MBE_STATUS_OK;
        if (!lose && !refined) {
            int n = 0;
            rc = large_phase<double>(ctx, pl, D, sgn, o.tol, (mixed && sector == 0) ? o.fp64_final_iters : 0,
                                     o.max_iter, 0, &l, &r, &n, &ss);
            if (rc) return rc;
            s64 += n;
        }
        n64 += s64;
        n32 += s32;
        if (sector == 0) {
            lam = l;
            rn = r;
            st = ss;
        } else if (!lose && ss != MBE_STATUS_NONFINITE && l < lam) {
            degen = degen || (ss == MBE_STATUS_OK && st == MBE_STATUS_OK && fabs(l - lam) <= DEGEN_TOL);
            lam = l;
            rn = r;
            st = ss;
        } else {
            degen = degen || (!lose && ss == MBE_STATUS_OK && st == MBE_STATUS_OK && fabs(l - lam) <= DEGEN_TOL);
            MBE_CU(cudaMemcpyAsync(D.x, D.xs, (size_t)N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        }
    }
    double ephi = 0.0;
    MBE_CU(cudaMemcpyAsync(&ephi, pl.L.diag + dphi, 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (cvec) MBE_CU(cudaMemcpyAsync(cvec, D.x, (size_t)N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    MBE_CU(cudaStreamSynchronize(ctx->stream));
    result[0] = lam;
    result[1] = lam - ephi;
    result[2] = rn;
    info[0] = with_degeneracy(st, degen);
    info[1] = n64;
    info[2] = n32;
    return MBE_OK;
}
