/*
 * Oracle, determinant-basis full CI from the Slater-Condon rules.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a small host library
 * that the tests, the smoke check and the CPU-baseline leg of the benchmark
 * load through ctypes.  The CUDA product path never includes, links or calls
 * it, and it shares no code with that path.
 *
 * What it computes: the matrix elements <I|H|J> of the spin-free electronic
 * Hamiltonian
 *     H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps)
 * between Slater determinants, i.e. the Hamiltonian of each CASCI calculation
 * that the MBE-FCI expansion (Eqs. 1-2) is built from.  The paper only names
 * the CASCI solver; the rules used here are the textbook Slater-Condon rules
 * written in a spin-orbital basis.
 *
 * Determinant convention.  A determinant over n spatial orbitals is a 2n-bit
 * occupation word: bit p (0 <= p < n) is orbital p with spin alpha, bit n+p is
 * orbital p with spin beta.  The state is the product of creation operators in
 * ascending bit order acting on the vacuum, so a creator or annihilator on bit
 * k picks up (-1)^(number of occupied bits below k) (Jordan-Wigner order).
 * Strings of one spin are listed in ascending integer order; the determinant
 * with alpha string I_a and beta string I_b has index I_a * N_b + I_b.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef uint64_t word;

static int popc(word x) { return __builtin_popcountll(x); }
static int lowbit(word x) { return __builtin_ctzll(x); }
static int highbit(word x) { return 63 - __builtin_clzll(x); }

/* (-1)^(number of occupied bits strictly below bit k of d) */
static int jw_sign(word d, int k)
{
    word below = (k == 0) ? 0 : (d & ((((word)1) << k) - 1));
    return (popc(below) & 1) ? -1 : 1;
}

static double ERI(const double *eri, int n, int p, int q, int r, int s)
{
    return eri[(((size_t)p * n + q) * n + r) * n + s];
}

int64_t oracle_binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    int64_t c = 1;
    for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
    return c;
}

/* All strings with k bits set among n bits, ascending.  Returns the count. */
int64_t oracle_strings(int n, int k, word *out)
{
    int64_t c = 0;
    if (n < 0 || n > 30) return -1;
    for (word x = 0; x < (((word)1) << n); ++x) {
        if (popc(x) == k) {
            if (out) out[c] = x;
            ++c;
        }
    }
    return c;
}

/* Position of string s in the ascending list, or -1. */
static int64_t find_string(const word *list, int64_t len, word s)
{
    int64_t lo = 0, hi = len - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (list[mid] == s) return mid;
        if (list[mid] < s) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/*
 * <I|H|J> for two 2n-bit determinants.
 *   same determinant : sum_K h_kk + 1/2 sum_{K,L} [ (kk|ll) - d(s_K,s_L) (kl|lk) ]
 *   single K=Q -> P  : G * [ h_pq + sum_{K in J, K != Q} ( (pq|kk) - d(s_P,s_K) (pk|kq) ) ]
 *   double Q,S -> P,R: G * [ d(s_P,s_Q) d(s_R,s_S) (pq|rs) - d(s_P,s_S) d(s_R,s_Q) (ps|rq) ]
 * where G is the phase of the replacement operator applied to J
 * (a+_P a_Q, resp. a+_P a+_R a_S a_Q, rightmost operator first).
 */
double oracle_hij(int n, const double *h, const double *eri, word I, word J)
{
    word diff = I ^ J;
    int nd = popc(diff);
    if (nd == 0) {
        double e = 0.0;
        for (word a = J; a; a &= a - 1) {
            int K = lowbit(a), k = K % n;
            e += h[k * n + k];
            for (word b = J; b; b &= b - 1) {
                int L = lowbit(b), l = L % n;
                e += 0.5 * ERI(eri, n, k, k, l, l);
                if (K / n == L / n) e -= 0.5 * ERI(eri, n, k, l, l, k);
            }
        }
        return e;
    }
    word ann = J & diff, cre = I & diff;
    if (popc(ann) != popc(cre)) return 0.0;
    if (nd == 2) {
        int Q = lowbit(ann), P = lowbit(cre);
        if (Q / n != P / n) return 0.0;
        int g = jw_sign(J, Q);
        word d = J & ~(((word)1) << Q);
        g *= jw_sign(d, P);
        int p = P % n, q = Q % n;
        double v = h[p * n + q];
        for (word a = J; a; a &= a - 1) {
            int K = lowbit(a), k = K % n;
            if (K == Q) continue;
            v += ERI(eri, n, p, q, k, k);
            if (K / n == P / n) v -= ERI(eri, n, p, k, k, q);
        }
        return g * v;
    }
    if (nd == 4) {
        int Q = lowbit(ann), S = highbit(ann);
        int P = lowbit(cre), R = highbit(cre);
        int g = jw_sign(J, Q);
        word d = J & ~(((word)1) << Q);
        g *= jw_sign(d, S);
        d &= ~(((word)1) << S);
        g *= jw_sign(d, R);
        d |= ((word)1) << R;
        g *= jw_sign(d, P);
        int p = P % n, q = Q % n, r = R % n, s = S % n;
        double v = 0.0;
        if (P / n == Q / n && R / n == S / n) v += ERI(eri, n, p, q, r, s);
        if (P / n == S / n && R / n == Q / n) v -= ERI(eri, n, p, s, r, q);
        return g * v;
    }
    return 0.0;
}

/*
 * All determinants connected to J by H (J itself, single and double
 * replacements conserving the alpha and beta counts).  Returns the count.
 */
static int64_t connections(int n, word J, word *out)
{
    word all = (2 * n >= 64) ? ~(word)0 : ((((word)1) << (2 * n)) - 1);
    word occ = J, vir = all & ~J;
    int64_t c = 0;
    out[c++] = J;
    /* singles */
    for (word a = occ; a; a &= a - 1) {
        int Q = lowbit(a);
        for (word b = vir; b; b &= b - 1) {
            int P = lowbit(b);
            if (Q / n != P / n) continue;
            out[c++] = J ^ (((word)1) << Q) ^ (((word)1) << P);
        }
    }
    /* doubles: annihilate Q < S, create P < R, same total spin */
    for (word a = occ; a; a &= a - 1) {
        int Q = lowbit(a);
        for (word a2 = a & (a - 1); a2; a2 &= a2 - 1) {
            int S = lowbit(a2);
            int sz_ann = (Q / n) + (S / n);
            for (word b = vir; b; b &= b - 1) {
                int P = lowbit(b);
                for (word b2 = b & (b - 1); b2; b2 &= b2 - 1) {
                    int R = lowbit(b2);
                    if ((P / n) + (R / n) != sz_ann) continue;
                    out[c++] = J ^ (((word)1) << Q) ^ (((word)1) << S) ^ (((word)1) << P) ^
                               (((word)1) << R);
                }
            }
        }
    }
    return c;
}

static int64_t max_connections(int n)
{
    int64_t m = 2 * n;
    return 1 + m * m + (m * m) * (m * m);
}

typedef struct {
    int n, na, nb;
    int64_t Na, Nb;
    word *sa, *sb;
} space_t;

static int space_init(space_t *s, int n, int na, int nb)
{
    s->n = n; s->na = na; s->nb = nb;
    s->Na = oracle_binom(n, na);
    s->Nb = oracle_binom(n, nb);
    s->sa = (word *)malloc(sizeof(word) * (size_t)(s->Na > 0 ? s->Na : 1));
    s->sb = (word *)malloc(sizeof(word) * (size_t)(s->Nb > 0 ? s->Nb : 1));
    if (!s->sa || !s->sb) return -1;
    oracle_strings(n, na, s->sa);
    oracle_strings(n, nb, s->sb);
    return 0;
}

static void space_free(space_t *s)
{
    free(s->sa);
    free(s->sb);
}

static word det_word(const space_t *s, int64_t idx)
{
    return s->sa[idx / s->Nb] | (s->sb[idx % s->Nb] << s->n);
}

static int64_t det_index(const space_t *s, word d)
{
    word amask = (((word)1) << s->n) - 1;
    int64_t ia = find_string(s->sa, s->Na, d & amask);
    int64_t ib = find_string(s->sb, s->Nb, d >> s->n);
    if (ia < 0 || ib < 0) return -1;
    return ia * s->Nb + ib;
}

/* Determinant words in index order. */
int oracle_dets(int n, int na, int nb, word *out)
{
    space_t s;
    if (space_init(&s, n, na, nb)) return -1;
    for (int64_t i = 0; i < s.Na * s.Nb; ++i) out[i] = det_word(&s, i);
    space_free(&s);
    return 0;
}

/* Diagonal H_II for all determinants of the (na, nb) sector. */
int oracle_hdiag(int n, int na, int nb, const double *h, const double *eri, double *out)
{
    space_t s;
    if (space_init(&s, n, na, nb)) return -1;
    for (int64_t i = 0; i < s.Na * s.Nb; ++i) {
        word d = det_word(&s, i);
        out[i] = oracle_hij(n, h, eri, d, d);
    }
    space_free(&s);
    return 0;
}

/*
 * Sparse H in coordinate form: entries (row, col, value) for every connected
 * pair.  Returns the number of entries, or -(needed) if cap is too small.
 */
int64_t oracle_h_coo(int n, int na, int nb, const double *h, const double *eri, int64_t cap,
                     int64_t *rows, int64_t *cols, double *vals)
{
    space_t s;
    if (space_init(&s, n, na, nb)) return -1;
    word *con = (word *)malloc(sizeof(word) * (size_t)max_connections(n));
    int64_t N = s.Na * s.Nb, cnt = 0;
    for (int64_t j = 0; j < N; ++j) {
        word J = det_word(&s, j);
        int64_t nc = connections(n, J, con);
        for (int64_t c = 0; c < nc; ++c) {
            int64_t i = det_index(&s, con[c]);
            if (i < 0) continue;
            if (cnt < cap) {
                rows[cnt] = i;
                cols[cnt] = j;
                vals[cnt] = oracle_hij(n, h, eri, con[c], J);
            }
            ++cnt;
        }
    }
    free(con);
    space_free(&s);
    return cnt <= cap ? cnt : -cnt;
}

/* sigma = H c, with H applied column by column from the connection lists. */
int oracle_sigma(int n, int na, int nb, const double *h, const double *eri, const double *c,
                 double *sigma)
{
    space_t s;
    if (space_init(&s, n, na, nb)) return -1;
    word *con = (word *)malloc(sizeof(word) * (size_t)max_connections(n));
    int64_t N = s.Na * s.Nb;
    for (int64_t i = 0; i < N; ++i) sigma[i] = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        if (c[j] == 0.0) continue;
        word J = det_word(&s, j);
        int64_t nc = connections(n, J, con);
        for (int64_t k = 0; k < nc; ++k) {
            int64_t i = det_index(&s, con[k]);
            if (i < 0) continue;
            sigma[i] += oracle_hij(n, h, eri, con[k], J) * c[j];
        }
    }
    free(con);
    space_free(&s);
    return 0;
}

/*
 * Selected rows of sigma = H c: out[i] = sum_J <rows[i]|H|J> c_J, with J running
 * over the determinants connected to rows[i].  For spaces too large for a full
 * oracle sigma.
 */
int oracle_sigma_rows(int n, int na, int nb, const double *h, const double *eri, const double *c,
                      int64_t nrows, const int64_t *rows, double *out)
{
    space_t s;
    if (space_init(&s, n, na, nb)) return -1;
    word *con = (word *)malloc(sizeof(word) * (size_t)max_connections(n));
    for (int64_t r = 0; r < nrows; ++r) {
        word I = det_word(&s, rows[r]);
        int64_t nc = connections(n, I, con);
        double acc = 0.0;
        for (int64_t k = 0; k < nc; ++k) {
            int64_t j = det_index(&s, con[k]);
            if (j < 0) continue;
            acc += oracle_hij(n, h, eri, I, con[k]) * c[j];
        }
        out[r] = acc;
    }
    free(con);
    space_free(&s);
    return 0;
}

/*
 * Spin-free reduced density matrices of the state c in the (na, nb) sector,
 * by explicit action of creation and annihilation operators on determinants:
 *   gamma[p*n+q]             = sum_s      <c| a+_ps a_qs |c>
 *   Gamma[((p*n+q)*n+r)*n+s] = sum_{s,t}  <c| a+_ps a+_rt a_st a_qs |c>
 * (chemists' order, so that E = sum h_pq gamma_pq + 1/2 sum (pq|rs) Gamma_pqrs).
 * Gamma may be NULL.  Operators act rightmost first, each with its
 * Jordan-Wigner sign.
 */
int oracle_rdm12(int n, int na, int nb, const double *c, double *gamma, double *Gamma)
{
    space_t s;
    if (space_init(&s, n, na, nb)) return -1;
    int64_t N = s.Na * s.Nb;
    for (int i = 0; i < n * n; ++i) gamma[i] = 0.0;
    if (Gamma)
        for (int64_t i = 0; i < (int64_t)n * n * n * n; ++i) Gamma[i] = 0.0;
    int m = 2 * n;
    for (int64_t j = 0; j < N; ++j) {
        double cj = c[j];
        if (cj == 0.0) continue;
        word J = det_word(&s, j);
        for (int Q = 0; Q < m; ++Q) {
            if (!((J >> Q) & 1)) continue;
            int g1 = jw_sign(J, Q);
            word d1 = J & ~(((word)1) << Q);
            /* one-body: a+_P a_Q, same spin */
            for (int P = 0; P < m; ++P) {
                if (P / n != Q / n || ((d1 >> P) & 1)) continue;
                int g2 = jw_sign(d1, P);
                word I = d1 | (((word)1) << P);
                int64_t i = det_index(&s, I);
                if (i >= 0) gamma[(P % n) * n + (Q % n)] += c[i] * g1 * g2 * cj;
            }
            if (!Gamma) continue;
            /* two-body: a+_P a+_R a_S a_Q, spin(P) = spin(Q), spin(R) = spin(S) */
            for (int S = 0; S < m; ++S) {
                if (!((d1 >> S) & 1)) continue;
                int g2 = jw_sign(d1, S);
                word d2 = d1 & ~(((word)1) << S);
                for (int R = 0; R < m; ++R) {
                    if (R / n != S / n || ((d2 >> R) & 1)) continue;
                    int g3 = jw_sign(d2, R);
                    word d3 = d2 | (((word)1) << R);
                    for (int P = 0; P < m; ++P) {
                        if (P / n != Q / n || ((d3 >> P) & 1)) continue;
                        int g4 = jw_sign(d3, P);
                        word I = d3 | (((word)1) << P);
                        int64_t i = det_index(&s, I);
                        if (i < 0) continue;
                        int p = P % n, q = Q % n, r = R % n, ss = S % n;
                        Gamma[(((int64_t)p * n + q) * n + r) * n + ss] += c[i] * g1 * g2 * g3 * g4 * cj;
                    }
                }
            }
        }
    }
    space_free(&s);
    return 0;
}
