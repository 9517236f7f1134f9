/*
 * mbe.h -- C ABI of the GB300 (sm_103a) engine for the MBE-FCI tuple-CASCI
 * hot path (generalized many-body expanded full configuration interaction).
 *
 * The method: the orbitals are split into a reference space R and an
 * expansion space X (Eq. 1).  Every tuple Omega of n expansion orbitals
 * defines a complete active space A = R u Omega whose CASCI energy gives the
 * tuple energy eps(Omega); the increments of Eq. 2,
 *     Delta eps(Omega) = eps(Omega) - sum over proper sub-tuples S of Delta eps(S),
 * summed order by order give E = E_ref + E^(1) + E^(2) + ... (Eq. 1, and Eq. 3
 * for an empty, "vacuum", reference space).
 *
 * Conventions shared by every call:
 *  - Integrals are real, float64, row-major: h1[p*norb+q] = h_pq and
 *    eri[((p*norb+q)*norb+r)*norb+s] = (pq|rs) in chemists' notation, with the
 *    8-fold permutational symmetry of real orbitals.
 *  - occ[p] = 1 marks an orbital doubly occupied in the closed-shell reference
 *    determinant Phi, 0 a virtual one.
 *  - Orbital indices are 0-based global indices.  Tuples are rows of `order`
 *    int32 indices, each row strictly ascending; tuple lists are in
 *    lexicographic order (the order mbe_tuples produces).
 *  - "device" pointers are CUDA global memory of the context's device; "host"
 *    pointers are ordinary host memory.  The caller allocates and owns every
 *    input and output buffer; the library owns only its context's workspace
 *    and string-table cache.
 *  - Calls are asynchronous on the context's stream unless stated otherwise.
 *  - Every call returns MBE_OK (0) or a negative MBE_E* code; mbe_last_error()
 *    then describes the failure.  No call aborts, exits or traps on the device.
 */
#ifndef MBE_H
#define MBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ errors */
#define MBE_OK 0
#define MBE_EINVAL (-1)       /* an argument is out of range or inconsistent   */
#define MBE_ENOMEM (-2)       /* device or host allocation failed              */
#define MBE_ECUDA (-3)        /* a CUDA runtime call failed                    */
#define MBE_EUNSUPPORTED (-4) /* sizes beyond the compiled limits (see below)  */

/* Compiled limits. */
#define MBE_MAX_NORB 64       /* orbitals in the full space                    */
#define MBE_MAX_CAS 12        /* orbitals in one tuple active space |R u Omega| of
                                 casci_batch (casci_batch_routed: MBE_MAX_LARGE_CAS) */
#define MBE_MAX_ORDER 16      /* tuple order n                                 */
#define MBE_MAX_STRING_ORB 16 /* orbitals of one string table (mbe_string_table) */

/* Per-tuple status codes written by casci_batch. */
#define MBE_STATUS_OK 0        /* converged: residual 2-norm <= tol              */
#define MBE_STATUS_MAXITER 1   /* iteration cap reached; eps holds the last Ritz value */
#define MBE_STATUS_NONFINITE 2 /* a NaN or Inf appeared; eps is NaN              */
#define MBE_STATUS_BADINPUT 3  /* malformed tuple (index range, order, overlap with R) */
#define MBE_STATUS_DEGENERATE 4 /* converged, and the lowest eigenvalues of the two spin-flip
                                   sectors (the alpha-beta string exchange, P c = +c and
                                   P c = -c) lie within 1e-8 E_h: eps is valid, the ground
                                   state and its density matrices are not unique */

/* Tuple-enumeration flags. */
#define MBE_SKIP_NO_OCC_OR_VIRT 1 /* drop a tuple whose active space R u Omega has no
                                     occupied or no virtual orbital (such tuples have
                                     vanishing increments for an empty reference space,
                                     the statement after Eq. 3) */

/* Precision modes of casci_batch. */
#define MBE_PREC_FP64 0  /* every sigma and every Davidson step in float64             */
#define MBE_PREC_MIXED 1 /* float32 sigma and Davidson until the residual reaches
                            tol_switch; then an anchored refinement in every solver
                            (warp, block and single large CAS): one float64 sigma of
                            the float32 Ritz vector x0 (the anchor: theta0 = its
                            Rayleigh quotient, r0 = H x0 - theta0 x0), then the
                            Davidson continues in float32 on H - theta0 from x0 (at
                            least fp64_final_iters iterations), so that the energy
                            theta0 + mu keeps float64 accuracy.  A refinement is
                            accepted when its residual is <= tol and its correction
                            |d| <= 3e-4; otherwise x0 + d becomes the next anchor.
                            A tuple that does not converge within the anchor limit
                            (6 warp, 8 block, 8 large) is solved again in float64.   */

typedef struct mbe_ctx mbe_ctx;

typedef struct mbe_opts {
    int precision;        /* MBE_PREC_FP64 or MBE_PREC_MIXED                       */
    double tol;           /* converged when ||H x - lambda x||_2 <= tol (x unit norm) */
    double tol_switch;    /* mixed mode: float32 phase ends at this residual         */
    int max_iter;         /* cap on Davidson iterations per phase                    */
    int fp64_final_iters; /* mixed mode: minimum refinement iterations (see above)   */
    int sectors;          /* MBE_SECTORS_BOTH: the lowest state of the determinant
                             space; MBE_SECTORS_EVEN: the lowest state that is even
                             under the exchange of the alpha and beta strings (the
                             closed-shell determinant's sector; for n_alpha = n_beta
                             the states of even total spin)                         */
    double s2_penalty;    /* state targeting by total spin (the paper converges its
                             Cr2 expansion onto a singlet, 1Sigma_g+): mu >= 0; the
                             solvers find the lowest eigenvalue of H + mu S^2.  A
                             singlet's energy is unchanged (S^2 = 0) and a state of
                             spin S is raised by mu S(S+1), so with mu above the
                             largest singlet-high-spin gap the result is the lowest
                             singlet energy.  0 (default): off.  casci_batch and
                             casci_rdm_batch only; casci_solve (and the tuples that
                             casci_batch_routed hands to it) reject mu != 0 with
                             MBE_EUNSUPPORTED.  Costs up to k^2 extra terms per
                             determinant in every sigma product.                   */
} mbe_opts;

#define MBE_SECTORS_BOTH 0
#define MBE_SECTORS_EVEN 1

/* Fills *opts with the defaults: FP64, tol 1e-7, tol_switch 1e-5, max_iter 2000,
   fp64_final_iters 2, MBE_SECTORS_BOTH, s2_penalty 0.  Host only, synchronous.  The residual
   tolerance 1e-7 keeps every tuple energy within ~1e-13 E_h of the exact lowest
   eigenvalue (the error is about |r|^2 / gap), which the Eq. 2 sums need: the
   Rayleigh-quotient errors of ~10^5 tuples all have the same sign. */
void mbe_default_opts(mbe_opts *opts);

/* ------------------------------------------------------------------ context */

/* Creates a context on CUDA device `device`, issuing work on `cuda_stream`
   (a cudaStream_t; NULL = the legacy default stream).  The context owns a
   growable device workspace and a cache of string tables.  Synchronous.
   Errors: MBE_EINVAL (ctx NULL or bad device), MBE_ECUDA, MBE_ENOMEM. */
int mbe_ctx_create(mbe_ctx **ctx, int device, void *cuda_stream);

/* Changes the stream later calls issue work on.  Host only. */
int mbe_ctx_set_stream(mbe_ctx *ctx, void *cuda_stream);

/* Waits for all work of the context, frees its workspace, its worker contexts
   (casci_batch_routed) and the context. */
void mbe_ctx_destroy(mbe_ctx *ctx);

/* Text of the last error raised by a call on this thread (never NULL). */
const char *mbe_last_error(void);

/* Synchronises the context's stream and reports any pending CUDA error. */
int mbe_ctx_sync(mbe_ctx *ctx);

/* Number of kernels this context has launched since it was created.  Host only. */
int mbe_ctx_launches(const mbe_ctx *ctx, int64_t *count);

/* Per-launch timing of the tuple-CASCI solver kernels, for measurement.  While
   enabled, casci_batch brackets every solver launch with a pair of CUDA events
   on the context's stream.  mbe_ctx_timings synchronises the stream, copies up
   to `max` records into `out` (host), sets *count to the number of records and
   clears them.  solver: 0 = one tuple per warp (dpl = determinants per lane),
   1 = one tuple per thread block.  Not for use during stream capture. */
typedef struct mbe_timing {
    int order;  /* tuple order of the casci_batch call (n_cas for solver 2) */
    int solver; /* 0 warp solver, 1 block solver, 2 large-CAS sigma         */
    int dpl;    /* determinants per lane (warp solver); 64 or 32 (solver 2: precision) */
    float ms;   /* elapsed time of the launch             */
} mbe_timing;
int mbe_ctx_set_timing(mbe_ctx *ctx, int enable);
int mbe_ctx_timings(mbe_ctx *ctx, int max, mbe_timing *out, int *count);

/* Launch choices of casci_batch, chosen per precision and active-space size (the
   paper names no solver shapes; these are the engine's own):
     warp_max_ndet  tuple spaces of at most this many determinants (and at most 8
                    orbitals) run one per warp with the Davidson vectors in registers,
                    the others one per thread block (1..416; default 416)
     warp_warps     warps per thread block of the warp solver (1..4; default 4)
     block_basis    Davidson basis of the block solver (4..20; default 20)       */
typedef struct mbe_tuning {
    int warp_max_ndet;
    int warp_warps;
    int block_basis;
} mbe_tuning;

/* Sets the tuning of later casci_batch calls for one precision (MBE_PREC_*) and
   active-space size n_cas = |R| + order (1..MBE_MAX_CAS), or for every size when
   n_cas is 0; reads it back.  Host only.  Errors: MBE_EINVAL (values out of range). */
int mbe_ctx_set_tuning(mbe_ctx *ctx, int precision, int n_cas, const mbe_tuning *t);
int mbe_ctx_get_tuning(const mbe_ctx *ctx, int precision, int n_cas, mbe_tuning *t);

/* Autotuner of the launch choices: runs casci_batch (same arguments; outputs into
   its own temporary buffers) on the given tuples, typically a sample of one order,
   for candidates of each tuning field in turn, starting from the current tuning:
   warp_warps in {2, 4}, then warp_max_ndet in {100, 225, 416}, then block_basis in
   {12, 16, 20}; each candidate is timed (CUDA events, best of two calls after one
   warm-up call) and the fastest kept.  The result is set on the context for this
   precision and |R| + order and returned in *best; records[0..*n_records) (host,
   up to max_records) list every candidate with its time.  Synchronous.
   Errors: as casci_batch. */
typedef struct mbe_tune_record {
    mbe_tuning tuning;
    float ms;
} mbe_tune_record;
int mbe_autotune(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ, int n_ref,
                 const int32_t *ref_orbs, double e_ref_corr, int order, int64_t n_tuples, const int32_t *tuples,
                 const mbe_opts *opts, mbe_tuning *best, mbe_tune_record *records, int max_records,
                 int *n_records);

/* Measurement helper, not part of the method: the fused multiply-add throughput
   of the context's GPU, the denominator of the roofline fraction of the solver
   kernels (which are bound by plain float64 / float32 arithmetic).  Runs one
   warm-up and `reps` (1..1000) timed launches of a kernel in which every thread
   of 4 x 256-thread blocks per SM advances 8 independent chains a <- a*b + c,
   and returns the best rate in TFLOP/s (2 flops per FMA), CUDA events on the
   context's stream.  kind: 0 = float64, 1 = float32.  Synchronous.
   Errors: MBE_EINVAL, MBE_ENOMEM, MBE_ECUDA. */
int mbe_fma_peak(mbe_ctx *ctx, int kind, int reps, double *tflops);

/* ------------------------------------------------------------------ a1: tuples */

/*
 * Tuple enumeration (Eq. 2's order-n tuples; skip rule after Eq. 3).
 * All order-`order` subsets of the expansion space, listed in lexicographic
 * order of the sorted expansion orbitals, optionally without the tuples that
 * MBE_SKIP_NO_OCC_OR_VIRT drops.
 *   exp_orbs [n_exp]  host, distinct orbital indices (any order; sorted inside)
 *   ref_orbs [n_ref]  host, the reference space (only used by the skip rule)
 *   occ      [norb]   host, reference occupations
 *   n_tuples          host out: number of tuples
 *   tuples   [n_tuples*order] device out, or NULL to query the count only
 *                     (the count query is synchronous and launches nothing).
 * The enumeration itself runs on the device: rank -> lexicographic unranking ->
 * filter -> order-preserving compaction.
 * Errors: MBE_EINVAL (bad indices, order < 1 or > n_exp, order > MBE_MAX_ORDER),
 * MBE_ECUDA.
 */
int mbe_tuples(mbe_ctx *ctx, int norb, const uint8_t *occ, int n_exp, const int32_t *exp_orbs,
               int n_ref, const int32_t *ref_orbs, int order, int flags, int64_t *n_tuples,
               int32_t *tuples);

/* ------------------------------------------------------------------ a3: strings */

/*
 * String table of one (n_orb, n_el) class, built on the device.
 *   strings [C(n_orb, n_el)]            device out (uint32 bit patterns), ascending;
 *                                       string rank = sum_i C(c_i, i) over its set bits
 *                                       c_1 < c_2 < ... (combinatorial number system)
 *   table   [C(n_orb,n_el) * n_el*(n_orb-n_el+1)]  device out, or NULL.
 * Row I lists every non-zero single replacement E_pq |I> = sign |J> (q occupied in
 * I, p empty in I or p == q), ordered by q ascending then p ascending, packed as
 *   entry = (J << 9) | (pair(p,q) << 1) | (sign < 0),
 * pair(p,q) = max(p,q)*(max(p,q)+1)/2 + min(p,q);  sign = (-1)^(number of occupied
 * orbitals of I strictly between p and q).  These replacement lists carry the
 * CASCI sigma (the CASCI solver is the one the paper names; the layout is ours).
 * Errors: MBE_EINVAL, MBE_EUNSUPPORTED (n_orb > MBE_MAX_STRING_ORB), MBE_ECUDA.
 */
int mbe_string_table(mbe_ctx *ctx, int n_orb, int n_el, uint32_t *strings, int32_t *table);

/* ------------------------------------------------------------------ a2-a7: CASCI */

/*
 * Reference-determinant energy E_Phi = sum_{i in O} 2 h_ii + sum_{i,j in O}
 * [2 (ii|jj) - (ij|ji)], O = {p : occ[p] = 1}.  h1, eri, occ device; e_phi device
 * out (one double).
 */
int mbe_phi_energy(mbe_ctx *ctx, int norb, const double *h1, const double *eri,
                   const uint8_t *occ, double *e_phi);

/*
 * Batched tuple CASCI (eps in Eq. 1 and Eq. 2).  For every tuple t:
 *   A = R u tuple_t (sorted), n_alpha = n_beta = |O n A|; the orbitals of O outside
 *   A are a frozen core (their mean field enters through the core Fock matrix
 *   F = h + sum_{i in O}(2 J_i - K_i), computed on the device), the other
 *   orbitals are deleted; lambda = lowest eigenvalue of the active-space
 *   Hamiltonian in the (n_alpha, n_beta) determinant sector, found by a batched
 *   Davidson solver; and
 *     eps_out[t] = lambda - <Phi_A|H_A|Phi_A> - e_ref_corr,
 *   which equals E_CAS(A) - E_Phi - e_ref_corr.
 *   h1 [norb^2], eri [norb^4], occ [norb]   device
 *   ref_orbs [n_ref]                         host, sorted, disjoint from tuples
 *   e_ref_corr                               E_CAS(R) - E_Phi (0 for R empty)
 *   tuples [n_tuples*order]                  device; order 0 is allowed with n_tuples = 1
 *                                            and tuples = NULL: the CAS is R itself, and
 *                                            with e_ref_corr = 0 the call returns
 *                                            E_ref,corr = E_CAS(R) - E_Phi
 *   opts                                     host; NULL = mbe_default_opts
 *   eps_out [n_tuples]                       device out
 *   status_out [n_tuples]                    device out, MBE_STATUS_*
 *   iters_out [n_tuples]                     device out or NULL: sigma products used
 *                                            (float64 ones in the high 16 bits,
 *                                            float32 ones in the low 16 bits)
 * |R| + order <= MBE_MAX_CAS.  Tuple problems of up to 416 determinants run one per
 * warp with the Davidson vectors in registers; larger ones one per thread block
 * with the vectors in the context's device workspace.
 * Errors: MBE_EINVAL, MBE_EUNSUPPORTED, MBE_ENOMEM, MBE_ECUDA.  A malformed tuple is
 * not an error of the call: its status is MBE_STATUS_BADINPUT and its eps NaN.
 */
int casci_batch(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                int n_ref, const int32_t *ref_orbs, double e_ref_corr, int order,
                int64_t n_tuples, const int32_t *tuples, const mbe_opts *opts, double *eps_out,
                int32_t *status_out, int32_t *iters_out);

/*
 * One sigma product sigma = H_A c for a single active space (the inner kernel of
 * casci_batch, exposed for parity tests and sigma throughput measurement).
 *   cas_orbs [n_cas] host, sorted; the active space A
 *   c, sigma [C(n_cas,k)^2] device, float64, determinant index I_a*N_b + I_b with
 *            strings in ascending bit-pattern order, k = |O n A|
 *   diag     [C(n_cas,k)^2] device out or NULL: the diagonal H_II
 * Errors: MBE_EINVAL, MBE_EUNSUPPORTED, MBE_ENOMEM, MBE_ECUDA.
 */
int casci_sigma(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                int n_cas, const int32_t *cas_orbs, const double *c, double *sigma,
                double *diag);

/*
 * Allocation-free variant of casci_sigma.  The paper has no counterpart: it
 * serves callers that cannot allocate device memory when they call, such as a
 * host application whose memory is owned by its own pool or allocator, code
 * running under a hard real-time discipline in which cudaMalloc would stall,
 * or a plug-in that must not grow device memory behind its host's back.
 *
 * The call computes the same sigma = H_A c (and the diagonal) as casci_sigma,
 * for the sector with n_el alpha and n_el beta electrons in the active space
 * cas_orbs (occ still defines the frozen core), but it allocates nothing: it
 * calls no cudaMalloc, cudaFree or allocating library routine and needs no
 * mbe_ctx.  Its scratch (core Fock matrix, string tables, packed integrals,
 * one-spin Hamiltonian, and the diagonal when diag is NULL) is one fixed
 * file-scope device array of MBE_NOALLOC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits.
 *   device         CUDA device to run on (made current for the call, then restored)
 *   cuda_stream    cudaStream_t the work is issued on (NULL = legacy default stream)
 *   n_cas <= MBE_NOALLOC_MAX_CAS; larger problems, or any whose scratch would
 *   exceed MBE_NOALLOC_SCRATCH_BYTES, are rejected with MBE_EUNSUPPORTED and a
 *   message saying so.  The caller still passes and owns inputs and outputs
 *   (device pointers, same layouts as casci_sigma).
 * Every call looks up the array's device address (cudaGetSymbolAddress, with the
 * device current; the lookup allocates nothing), so a device reset that reloads
 * the module leaves no stale address; the very first call on a device loads the
 * module, so make it before any stream capture.  Every call reuses the same array and
 * leaves the last call's contents in it; each call fully rewrites what it reads,
 * so nothing carries over.  Calls whose work overlaps on the GPU (other streams,
 * other host threads) race on the array: serialise them.
 * Errors: MBE_EINVAL, MBE_EUNSUPPORTED, MBE_ECUDA.  Asynchronous on cuda_stream.
 */
#define MBE_NOALLOC_MAX_CAS 10
#define MBE_NOALLOC_SCRATCH_BYTES (2u << 20) /* 2 MiB per device */
#define MBE_MAX_DEVICES 64
int casci_sigma_noalloc(int device, void *cuda_stream, int norb, const double *h1, const double *eri,
                        const uint8_t *occ, int n_cas, const int32_t *cas_orbs, int n_el, const double *c,
                        double *sigma, double *diag);

/* ------------------------------------------------------------------ a10: adjoint */

/*
 * Adjoint weights of the increment recursion.  The paper defines the energy
 * only; its gradient follows from the linearity of Eq. 2: E_MBE - E_CAS(R) =
 * sum_S w(S) eps(S) over the computed tuples, with
 *     w(S) = 1 - sum over computed proper supersets U of S of w(U),
 * the transpose of Eq. 2 (a skipped tuple is absent, as in Eq. 2).  Orders are
 * processed from n_orders down to 1; supersets are enumerated in a fixed order,
 * so the result is deterministic.
 *   n_tuples [n_orders], tuples [n_orders]  host arrays (tuples: device pointers to
 *                                           lexicographic order-m lists, m = 1..n_orders)
 *   exp_orbs [n_exp]                        host, the expansion space
 *   scale                                   every output is multiplied by scale (1 for
 *                                           dE_MBE/dE_CAS itself; the upstream derivative
 *                                           of a scalar loss otherwise)
 *   weights [n_orders]                      host array of device pointers, out:
 *                                           scale * w(S)
 *   ref_weight [1]                          device out, or NULL: scale * w(R), the weight
 *                                           of the reference-space CASCI, w(R) = 1 -
 *                                           sum_S w(S) over every computed tuple (E_CAS(R)
 *                                           enters the total directly and, through every
 *                                           eps(S), with -w(S)); a fixed-order device
 *                                           reduction
 * Errors: MBE_EINVAL, MBE_ECUDA.
 */
int mbe_weights(mbe_ctx *ctx, int n_orders, const int64_t *n_tuples, const int32_t *const *tuples,
                int n_exp, const int32_t *exp_orbs, double scale, double *const *weights,
                double *ref_weight);

/*
 * Weighted Hellmann-Feynman gradients of tuple CASCI energies (the adjoint of
 * casci_batch).  Re-solves every tuple as casci_batch does (same opts; use a
 * tighter tol for gradients: the density matrices are first-order in the
 * eigenvector error), forms the spin-free 1-RDM (and 2-RDM when grad_eri is not
 * NULL) of the converged state from the replacement lists, and adds
 *     weights[t] * ( dE_CAS(R u tuple_t)/dtheta - dE_Phi/dtheta )
 * to the gradients, theta = h_pq (dE/dh_pq = gamma_pq) and theta = (pq|rs)
 * (dE/d(pq|rs) = 1/2 Gamma_pqrs), every tensor element treated as independent;
 * frozen-core contributions (core-core cancel against Phi, core-active ones are
 * 2 gamma_pq on (cc|pq), (pq|cc) and -gamma_pq on (cq|pc), (pc|cq)) included.
 *   same inputs as casci_batch (order 0 with tuples NULL: the CAS is R)
 *   weights [n_tuples]   device, or NULL for all ones
 *   grad_h1 [norb^2]     device, accumulated (+=); atomics, so the summation order
 *                        (last bits) is not deterministic
 *   grad_eri [norb^4]    device or NULL, accumulated (+=); needs |R| + order <= 10
 *   status_out [n_tuples] device or NULL
 * Errors: as casci_batch; MBE_EUNSUPPORTED for the 2-RDM beyond 10 orbitals.
 */
int casci_rdm_batch(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                    int n_ref, const int32_t *ref_orbs, int order, int64_t n_tuples, const int32_t *tuples,
                    const mbe_opts *opts, const double *weights, double *grad_h1, double *grad_eri,
                    int32_t *status_out);

/*
 * Adds scale * dE_Phi/dtheta: 2 scale on (i,i) of grad_h1 for i in O, and on
 * grad_eri (if not NULL) 2 scale on (ii|jj), scale on (ii|ii), -scale on (ij|ji),
 * i != j in O.  occ, grad_h1, grad_eri device.
 */
int mbe_phi_gradient(mbe_ctx *ctx, int norb, const uint8_t *occ, double scale, double *grad_h1,
                     double *grad_eri);

/* ------------------------------------------------------------------ a5-a6: one large CAS */

#define MBE_MAX_LARGE_CAS 16 /* orbitals of casci_sigma_large / casci_solve */

/*
 * sigma = H_A c for one large active space (the tuple CASCI sigma of a5 at the
 * sizes of a single big CASCI: up to 16 orbitals, (16e,16o) = 165,636,900
 * determinants), spread over the whole GPU.  Same operator, determinant order
 * and layouts as casci_sigma; the same-spin part uses a compressed (CSR) copy
 * of the one-spin Hamiltonian.
 *   precision   MBE_PREC_FP64: float64 arithmetic; MBE_PREC_MIXED: float32
 *               arithmetic on a float32 copy of c (result written as float64), the
 *               opposite-spin product on the tensor cores (tcgen05, TF32 split into
 *               hi + lo pairs, hi*hi + hi*lo + lo*hi accumulated in float32)
 *   c, sigma    device [N], N = C(n_cas, k)^2, k = |O n A|; diag device or NULL
 * Synchronous set-up (occupations read back), then asynchronous on the stream
 * (MBE_PREC_MIXED: synchronous, to report a tensor-core wait that ran out).
 * Errors: MBE_EINVAL, MBE_EUNSUPPORTED (n_cas > 16), MBE_ENOMEM, MBE_ECUDA.
 */
int casci_sigma_large(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                      int n_cas, const int32_t *cas_orbs, int precision, const double *c, double *sigma,
                      double *diag);

/*
 * Lowest eigenpair of one large active space (a6 for a single big CASCI): the
 * Davidson of casci_batch (12-vector basis, thick restart on the two lowest
 * Ritz vectors) with every vector operation in grid-wide kernels and the
 * projected eigenproblem solved by one warp on the device; float32 then
 * float64 phase in mixed mode, as in casci_batch.  Both spin-flip sectors
 * (alpha and beta strings exchanged, P c = +c and P c = -c) are solved and the
 * lower eigenvalue kept.  Synchronous: the host reads one residual norm per
 * iteration.
 *   result [3]  host out: lambda, eps = lambda - <Phi_A|H_A|Phi_A>, residual norm
 *   info [3]    host out: status (MBE_STATUS_*), float64 sigma products, float32 ones
 *   cvec [N]    device out (the unit Ritz vector) or NULL
 * Errors: as casci_sigma_large.
 */
int casci_solve(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ, int n_cas,
                const int32_t *cas_orbs, const mbe_opts *opts, double *result, int32_t *info, double *cvec);

/*
 * casci_batch for the large tuple active spaces of Type-1 and Type-2 expansions
 * (Sec. 1, Fig. 1: a reference space of every virtual, or of every occupied
 * orbital, so that |R u Omega| grows to the sizes of a single big CASCI).  Same
 * arguments, output and meaning as casci_batch (eps_out[t] = E_CAS(R u tuple_t)
 * - E_Phi - e_ref_corr), with |R| + order up to MBE_MAX_LARGE_CAS and one more:
 *   large_ndet   a tuple whose active space has more than large_ndet determinants
 *                (large_ndet > 0), or more than MBE_MAX_CAS orbitals, is solved by
 *                casci_solve with the whole GPU; the others go to casci_batch in
 *                one call (gathered to a temporary list when the order is mixed).
 *                With large_ndet <= 0 and |R| + order <= MBE_MAX_CAS this is
 *                casci_batch itself.
 * A routed tuple's iters_out holds casci_solve's sigma counts in the casci_batch
 * encoding; a routed active space with one determinant (Phi_A) gets eps =
 * -e_ref_corr without a solve.  Routed tuples of up to 4,000,000 determinants
 * are solved four at a time, each on a worker context of ctx (its own
 * non-blocking stream and host thread), after the work already queued on ctx's
 * stream; a solve that size leaves most of the GPU idle while its host loop
 * waits for each iteration's scalars.  The worker contexts (streams, workspaces,
 * string tables) are created on first use and freed by mbe_ctx_destroy; the
 * results do not depend on which worker solved a tuple.  Synchronous when any
 * tuple is routed (the host reads the tuples and occupations, and casci_solve
 * is synchronous); temporary device buffers are stream-ordered allocations
 * freed before return.
 * Errors: as casci_batch and casci_solve; MBE_EUNSUPPORTED for |R| + order
 * above MBE_MAX_LARGE_CAS.  A malformed routed tuple gets MBE_STATUS_BADINPUT
 * and eps NaN, as in casci_batch.
 */
int casci_batch_routed(mbe_ctx *ctx, int norb, const double *h1, const double *eri, const uint8_t *occ,
                       int n_ref, const int32_t *ref_orbs, double e_ref_corr, int order, int64_t n_tuples,
                       const int32_t *tuples, const mbe_opts *opts, int64_t large_ndet, double *eps_out,
                       int32_t *status_out, int32_t *iters_out);

/* ------------------------------------------------------------------ screened expansion */

/*
 * Child spawning of the screened expansion (Sec. 2: children at order k+1 are
 * spawned from the order-k tuples; thresholds by Eq. 4).  An order-(order+1)
 * tuple of the expansion space is listed when
 *     max over its order-`order` sub-tuples S of |Delta eps(S)|  >  T_tup(child),
 *     T_tup = 0 if M_tup < m_init, else t_init * a^(M_tup - m_init) (repeated
 *     products), M_tup = max(occupied, virtual orbitals of the child),
 * a sub-tuple missing from `parents` counting as zero, and the child kept by the
 * skip rule when MBE_SKIP_NO_OCC_OR_VIRT is set.  Output in lexicographic order.
 *   occ [norb], exp_orbs [n_exp], ref_orbs [n_ref]   host, as for mbe_tuples
 *   order                                            parent order k (1 <= k, k+1 <= n_exp)
 *   parents [n_parents*order], parent_incs [n_parents]
 *                                                    device: the computed order-k
 *                                                    tuples (lexicographic, as listed
 *                                                    by mbe_tuples or mbe_screen) and
 *                                                    their increments
 *   capacity                                         rows available in `children`
 *   n_children                                       host out: number of children
 *   children [capacity*(order+1)]                    device out, or NULL to count only
 * The call synchronises the context stream once (to read the count); with
 * children != NULL the children are then written asynchronously.  A count
 * query and the writing call run the same selection.
 * Errors: MBE_EINVAL (bad indices or orders, negative thresholds, count above
 * capacity), MBE_EUNSUPPORTED (more than 2^31 x 256 candidates), MBE_ENOMEM,
 * MBE_ECUDA.
 */
int mbe_screen(mbe_ctx *ctx, int norb, const uint8_t *occ, int n_exp, const int32_t *exp_orbs, int n_ref,
               const int32_t *ref_orbs, int order, int64_t n_parents, const int32_t *parents,
               const double *parent_incs, double t_init, int m_init, double a, int flags, int64_t capacity,
               int64_t *n_children, int32_t *children);

/* ------------------------------------------------------------------ a8-a9: Eqs. 2, 1 */

/*
 * Increment recursion, Eq. 2, for the tuples of one order:
 *   inc_out[t] = eps[t] - sum over every proper, non-empty subset S of tuple t of
 *                Delta eps(S),
 * where Delta eps(S) is looked up (binary search) in the lower-order lists; a
 * subset absent from its list (a skipped tuple) contributes 0.  The subsets are
 * visited in a fixed order (bit mask 1 .. 2^order-2 over the tuple's positions),
 * so the result is deterministic.
 *   tuples [n_tuples*order], eps [n_tuples]              device
 *   n_lower                                              number of lower orders given
 *                                                        (must be order - 1)
 *   n_lower_tuples [n_lower]                             host: list lengths, orders 1..n_lower
 *   lower_tuples [n_lower], lower_incs [n_lower]         host arrays of device pointers;
 *                                                        lower_tuples[m-1] holds order-m
 *                                                        tuples in lexicographic order
 *   inc_out [n_tuples]                                   device out
 * Errors: MBE_EINVAL, MBE_ECUDA.
 */
int mbe_increments(mbe_ctx *ctx, int order, int64_t n_tuples, const int32_t *tuples,
                   const double *eps, int n_lower, const int64_t *n_lower_tuples,
                   const int32_t *const *lower_tuples, const double *const *lower_incs,
                   double *inc_out);

/*
 * Order sums and total, Eq. 1 (Eq. 3 for an empty reference space):
 *   e_order_out[m] = sum_t incs[m][t]          (fixed-shape tree reduction)
 *   e_total_out[0] = e_phi + e_ref_corr + sum_m e_order_out[m]
 *   n_tuples [n_orders], incs [n_orders]       host arrays (incs: device pointers)
 *   e_phi                                      device pointer to one double, or NULL
 *                                              for 0 (e.g. to sum correlation only)
 *   e_order_out [n_orders], e_total_out [1]    device out
 * Errors: MBE_EINVAL, MBE_ECUDA.
 */
int mbe_total(mbe_ctx *ctx, int n_orders, const int64_t *n_tuples, const double *const *incs,
              const double *e_phi, double e_ref_corr, double *e_order_out, double *e_total_out);

#ifdef __cplusplus
}
#endif

#endif /* MBE_H */
