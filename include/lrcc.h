/*
 * lrcc.h -- C ABI of a single-GPU (GB300, sm_103a) four-component LR-CCSD
 * polarizability library in a truncated natural-spinor (FNS++) basis.
 *
 * Method: Chakraborty, Manna, Crawford, Dutta, "A low-cost four-component
 * relativistic coupled cluster linear response theory based on perturbation
 * sensitive natural spinors", arXiv:2503.23144.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Complex numbers are interleaved (re, im) doubles, layout-compatible with
 *    C99 `double _Complex` and `std::complex<double>`.  Arrays are row-major.
 *  - Spinor index p runs over N = O + V spinors, occupied first.
 *  - The Hamiltonian is given in the molecular-spinor basis: orbital energies
 *    eps[N] (canonical reference, Fock matrix = diag(eps)), a Hermitian
 *    three-index factor B[L][N][N] with <pq|rs> = sum_L B^L_pr B^L_qs
 *    (Sec. II.A, Eq. 7-8 in the no-pair approximation), and Hermitian
 *    perturbation matrices mu[ncomp][N][N] (dipole components).
 *  - Amplitude vectors (t, lambda, X, Y, residuals) are passed as a singles
 *    block [O][V] followed by a FULL antisymmetric doubles block [O][O][V][V]
 *    (t_ij^ab = -t_ji^ab = -t_ij^ba; Eq. 3-4).  Dot products between such
 *    vectors run over unique amplitudes (sum_ia + sum_{i<j,a<b}).
 *  - Host pointers are owned by the caller; the library copies what it needs.
 *    Device memory is owned by the context.  Every call returns a status and
 *    never throws; lrcc_last_error() gives a message for the last failure.
 *  - One context per host thread.  Calls on a context run on its stream in
 *    order; host-pointer calls synchronise before returning.
 */
#ifndef LRCC_H
#define LRCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lrcc_ctx lrcc_ctx;

typedef enum {
    LRCC_OK = 0,
    LRCC_EINVAL = 1,    /* bad argument: shape, Hermiticity, ordering, range   */
    LRCC_ENOMEM = 2,    /* device allocation failed                            */
    LRCC_ENOCONV = 3,   /* iteration cap reached or residual not finite        */
    LRCC_ETIMEOUT = 4,  /* a device wait gave up (kernel-side bounded spin)    */
    LRCC_ECUDA = 5,     /* CUDA runtime / driver / library error               */
    LRCC_ESTATE = 6     /* call out of order (e.g. solve before ground state)  */
} lrcc_status;

typedef enum {
    LRCC_FP64 = 0,          /* every contraction in FP64                        */
    LRCC_MIXED_TF32 = 1,    /* ladder/ring on tcgen05 kind::tf32, FP64 refine   */
    LRCC_MIXED_BF16X3 = 2,  /* ladder/ring as 3 bf16 products, FP64 refine      */
    LRCC_FP64_EMULATED = 3  /* FP64 solver; large contractions as exact integer-
                               slice products on bf16 tensor cores (7 slices of
                               6 bits, FP64 sums; ~1e-12 relative per product) */
} lrcc_precision;

typedef struct {
    double r_tol;          /* max |residual| for T, Lambda (default 1e-10)        */
    double x_tol;          /* max |residual| for X, Y (default 1e-9)              */
    int max_iter;          /* per solve (default 200)                             */
    int diis_size;         /* Pulay subspace per right-hand side (default 8)      */
    int rhs_chunk;         /* right-hand sides per batched solve (default 12)     */
    lrcc_precision prec;   /* contraction precision of the response solves        */
    double inner_tol;      /* mixed mode: residual reduction asked of the tensor-core
                              iterations, relative (default 1e-5)                  */
    int plus_omega;        /* FNS++ denominator Dbar + omega (Eq. 46 as printed)
                              instead of Dbar - omega (diagonal of Eq. 29)        */
    int slab_rows;         /* ladder: > 0 never caches <ab||ef>; it is assembled per call in
                              slabs of at most this many (a<b) rows.  0 = automatic: cached
                              when it fits in a third of free memory, else slabs sized to it */
    int pm_omega;          /* 1: response function of Eq. 36 (solves X(+w) and X(-w),
                              no Y); 0 (default): Eq. 35 (X(w) and Y(w))            */
    int fp64_products;     /* mixed modes: the FP64-accurate maps (outer residuals,
                              F X, ground-state polish) use 1 (default): integer-slice
                              products on the tensor cores (as LRCC_FP64_EMULATED),
                              0: FP64 SIMT products                                  */
    int fns_density;       /* lrcc_fns_truncate: 0 (default) FNS++, the component-averaged
                              density of the dipole-perturbed first-order amplitudes
                              (Eq. 45); 1: plain FNS, the ground-state MP2 virtual
                              density (Eq. 40)                                      */
    int solver;            /* response and Lambda equations: 0 (default) preconditioned
                              DIIS per right-hand side; 1: one shared subspace for every
                              right-hand side of a batch (Galerkin projections; each
                              product M v serves all frequencies and components).
                              1 needs prec LRCC_FP64 or LRCC_FP64_EMULATED          */
    int subspace_max;      /* solver 1: vectors kept before a restart from the current
                              solutions; 0 (default) automatic (8 per right-hand side,
                              48..400, within 30 % of free device memory); a value below
                              2 x the right-hand sides of a batch gives LRCC_EINVAL  */
    int ladder_hermitian;  /* per-call <ab||ef> assembly (mixed precisions): 1 assembles only the
                              columns (ef) >= (ab) of each row group and contracts the rest
                              through the conjugate transpose (<ef||ab> = conj <ab||ef>);
                              -1 assembles whole rows; 0 (default) automatic: 1 when a row
                              group holds at least 1024 rows                          */
    int embed_budget_mb;   /* tensor-core contractions: bytes (MiB) that the transient split
                              copies of one GEMM's two operands may take; a larger GEMM runs
                              as sub-GEMMs over halves of N, M or K.  0 (default) automatic:
                              min(6 GiB, 10 % of free device memory)                 */
} lrcc_options;

/* Fill *opt with the defaults above. */
void lrcc_default_options(lrcc_options* opt);

/*
 * lrcc_setup -- create a context for one spinor Hamiltonian (Sec. II.A).
 *   eps  [N]            host, real orbital energies, occupied first; every
 *                       occupied energy must be below every virtual one.
 *   B    [L][N][N]      host, complex interleaved, Hermitian per L to
 *                       1e-12 * max|B| (else LRCC_EINVAL).
 *   mu   [ncomp][N][N]  host, complex interleaved, Hermitian (ncomp 1..3).
 *   O, V, L             sizes; N = O + V; O >= 2, V >= 2.
 *   opt                 may be NULL (defaults).
 *   out                 receives the context; NULL on failure.
 * Copies all inputs to the device and builds the integral blocks
 * <pq||rs> = <pq|rs> - <pq|sr> that the residual needs (never the
 * <ab||ef> block, which the ladder assembles on the fly from B).
 */
lrcc_status lrcc_setup(const double* eps, const double* B, int L, const double* mu, int ncomp,
                       int O, int V, const lrcc_options* opt, lrcc_ctx** out);

/* Release all device memory of the context.  NULL is allowed. */
void lrcc_destroy(lrcc_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failing
 * lrcc_setup when ctx is NULL).  Never NULL. */
const char* lrcc_last_error(const lrcc_ctx* ctx);

/*
 * lrcc_ccsd_ground -- solve the CCSD amplitude equations R(T) = 0 (Eq. 9-10)
 * and the left-CCSD equations lambda A + dE/dT = 0 (Lambda of Eq. 20, 33-35).
 *   e_corr[2]  out, complex CCSD correlation energy (Re = energy, Im = diagnostic).
 *   iters_T, iters_L  out, iteration counts (may be NULL).
 * Returns LRCC_ENOCONV if either solve hits max_iter.
 */
lrcc_status lrcc_ccsd_ground(lrcc_ctx* ctx, double e_corr[2], int* iters_T, int* iters_L);

/*
 * lrcc_fns_truncate -- FNS++ (Sec. II.C, Eq. 39-50 with Eq. 41-44).
 * Call after lrcc_setup and before lrcc_ccsd_ground.  Builds the MP2 doubles,
 * the Hbar diagonals (Eq. 49-50), first-order perturbed amplitudes for every
 * dipole component (Eq. 46-48), the component-averaged perturbation-sensitive
 * virtual density (Eq. 45), its eigenvectors (natural spinors, Eq. 41), keeps
 * them by |occupation| descending, semicanonicalises (Eq. 42-44), and
 * replaces the context's virtual space, B, mu and eps by the rotated ones.
 * With opt.fns_density = 1 the density is the ground-state MP2 one of plain
 * FNS (Eq. 40, 1/2 sum_ijc t_ij^ac conj t_ij^bc) and omega is not used.
 *   by_count       1: keep the first round(value) natural spinors;
 *                  0: keep every one with |n| >= value.
 *   omega          frequency of the perturbed amplitudes.
 *   v_kept         out, new V (may be NULL).
 *   occ_out [V]    out, |n| sorted descending over the ORIGINAL V (may be NULL).
 */
lrcc_status lrcc_fns_truncate(lrcc_ctx* ctx, int by_count, double value, double omega,
                              int* v_kept, double* occ_out);

/*
 * lrcc_mp2_correction -- MP2 energies of the last lrcc_fns_truncate (Eq. 51):
 * e_full: 1/4 sum <ij||ab> t_ij^ab with MP2 doubles in the full virtual space,
 * e_trunc: the same in the truncated semicanonical space,
 * delta = e_full - e_trunc, the correction added to the truncated CCSD
 * correlation energy (Eq. 52).  Complex pairs (Re, Im); any pointer may be
 * NULL.  LRCC_ESTATE if no truncation was made on this context.
 */
lrcc_status lrcc_mp2_correction(const lrcc_ctx* ctx, double e_full[2], double e_trunc[2], double delta[2]);

/*
 * lrcc_mp2_alpha -- MP2-level polarisability in the context's current virtual
 * basis, the ingredient of the Delta alpha_MP2 correction (Eq. 53-54): call
 * it before lrcc_fns_truncate (canonical full space) and after it (truncated
 * semicanonical space); Delta alpha = alpha_full - alpha_truncated is added to
 * the truncated LR-CCSD alpha.  The paper names the ingredients (MP2 doubles,
 * the Eq. 46 first-order amplitudes) but prints no expression; this library
 * evaluates the sum-over-states response function (Eq. 18) over the singly
 * and doubly excited determinants mu with the MP2-dressed transition moments
 * Abar_mu of Eq. 48 (singles: A_ai + sum_me A_me t_im^ae) and the excitation
 * energies Dbar_mu of Eq. 47 (Hbar of Eq. 49-50):
 *   alpha_AB(w) = sum_mu conj(Abar_mu) Bbar_mu / (Dbar_mu - w)
 *                      + Abar_mu conj(Bbar_mu) / (Dbar_mu + w),
 * unique mu (i<j, a<b).  Needs only lrcc_setup.
 *   omegas [n_w]                 host, real frequencies; every |w| must lie
 *                                below the lowest Dbar (else LRCC_EINVAL).
 *   comps  [n_c]                 host, component indices into mu.
 *   alpha  [n_w][n_c][n_c] cplx  out, host.
 */
lrcc_status lrcc_mp2_alpha(lrcc_ctx* ctx, const double* omegas, int n_w, const int* comps, int n_c,
                           double* alpha);

/*
 * lrcc_solve -- polarisabilities alpha_AB(omega) = -<<A;B>>_omega (Eq. 35):
 * for every omega and every component B in comps, X^B from (A - omega) X = -xi
 * (Eq. 29-31) and Y^B from Y (A + omega) = -(eta + F X) (Eq. 32-34); then
 * g_AB = Y^B . xi^A + eta^A . X^B and alpha_AB = -(g_AB + conj g_BA)/2.
 * Right-hand sides (component, omega) are batched rhs_chunk at a time.
 * With opt.pm_omega = 1 the Eq. 36 form is used instead: X(+w) and X(-w) for
 * every component (one frequency per batch), and
 * <<A;B>>_w = 1/2 [G_AB(w) + conj G_AB(-w)],
 * G_AB(w) = eta^A.X^B(w) + eta^B.X^A(-w) + X^A(-w).F.X^B(w).
 *   omegas [n_w]                 host, real frequencies (Hartree).
 *   comps  [n_c]                 host, component indices into mu (0..ncomp-1).
 *   alpha  [n_w][n_c][n_c] cplx  out, host, Re = polarisability.
 *   err_est [n_w][n_c]           out (may be NULL): final max |residual| of X
 *                                and Y combined, per right-hand side.
 * Requires lrcc_ccsd_ground first (else LRCC_ESTATE).
 */
lrcc_status lrcc_solve(lrcc_ctx* ctx, const double* omegas, int n_w, const int* comps, int n_c,
                       double* alpha, double* err_est);

/* Kinds of lrcc_residual. */
typedef enum {
    LRCC_RES_T = 0,        /* out = R(in)  (CCSD residual, Eq. 9-10)          */
    LRCC_RES_SIGMA = 1,    /* out = A(T) in  (Jacobian product, Eq. 30)       */
    LRCC_RES_VJP = 2,      /* out = A(T)^T in (holomorphic transpose)         */
    LRCC_RES_XI = 3,       /* out = xi^comp = <nu|e^-T mu e^T|0> (Eq. 31); in = T */
    LRCC_RES_ENERGY = 4,   /* out[r][0..1] = E_corr(in_r)                    */
    LRCC_RES_VJP_FULL = 5  /* out = P J(P t)^T in: adjoint of T -> R(P T) with
                              every full-array entry independent; P projects
                              the doubles block onto its antisymmetric part.
                              This is the map whose conjugate PyTorch's
                              complex autograd expects.                       */
} lrcc_residual_kind;

/*
 * lrcc_residual -- test hook.  Evaluates one residual-type map on R
 * right-hand sides at once.
 *   kind     see lrcc_residual_kind.  The doubles blocks of `t` and `in`
 *            are first projected onto their antisymmetric part (a no-op for
 *            antisymmetric inputs), so every kind is defined for any array.
 *   t        host [O*V + O*O*V*V] complex: the amplitudes T at which
 *            SIGMA / VJP are linearised, or NULL to linearise at the
 *            converged ground state of lrcc_ccsd_ground or at the amplitudes
 *            of the last lrcc_linearize (the primal values kept there are
 *            reused, as in lrcc_solve; LRCC_ESTATE before either).
 *            Required for XI; ignored for T and ENERGY.
 *   in       host [R][O*V + O*O*V*V] complex.
 *   R        number of right-hand sides (>= 1).
 *   comp     dipole component for XI.
 *   prec     precision of the contractions (LRCC_FP64 or a mixed mode).
 *   out      host, same shape as in (ENERGY: [R][2]).
 */
lrcc_status lrcc_residual(lrcc_ctx* ctx, int kind, const double* t, const double* in, int R,
                          int comp, int prec, double* out);

/*
 * lrcc_linearize -- fixes the amplitudes T at which the Jacobian maps of
 * Eq. 30 (A = dR/dT, and its transpose) are applied by later lrcc_residual
 * calls with t == NULL, without solving the ground state: the residual
 * program is evaluated once at T (in precision `prec`) and its primal values
 * are kept, exactly as lrcc_ccsd_ground keeps them at the converged T.
 *   t     host [O*V + O*O*V*V] complex (doubles projected onto their
 *         antisymmetric part, as in lrcc_residual).
 *   prec  precision of that evaluation (LRCC_FP64 .. LRCC_FP64_EMULATED).
 * The ground state (and so lrcc_solve) is invalidated: lrcc_solve returns
 * LRCC_ESTATE until lrcc_ccsd_ground runs again.  Errors: LRCC_EINVAL (bad
 * arguments), LRCC_ENOMEM, LRCC_ECUDA.
 */
lrcc_status lrcc_linearize(lrcc_ctx* ctx, const double* t, int prec);

/*
 * Device-pointer variants for the PyTorch binding: same semantics, but every
 * array argument is a device pointer on the context's device and the call is
 * stream-ordered on `stream` (a cudaStream_t; NULL = legacy default stream).
 * The call does not synchronise; outputs are valid in stream order.
 */
lrcc_status lrcc_residual_dev(lrcc_ctx* ctx, int kind, const double* t_dev, const double* in_dev,
                              int R, int comp, int prec, double* out_dev, void* stream);

/*
 * lrcc_ladder_dev -- the particle-particle ladder alone (the dominant
 * contraction of the doubles residual, Eq. 9-10 / 30):
 *   Z_ij^ab = 1/2 sum_ef <ab||ef> X_ij^ef,   <ab|ef> = sum_L B^L_ae B^L_bf,
 * for X antisymmetric in (i,j) and in (e,f).
 *   x_dev  [R][O][O][V][V] complex, device.
 *   z_dev  [R][O][O][V][V] complex, device, overwritten (antisymmetric).
 *   transpose  0: the map above; 1: its holomorphic transpose (B -> B^T).
 *   prec   LRCC_FP64, LRCC_MIXED_TF32 or LRCC_MIXED_BF16X3.
 */
lrcc_status lrcc_ladder_dev(lrcc_ctx* ctx, const double* x_dev, double* z_dev, int R,
                            int transpose, int prec, void* stream);

/*
 * lrcc_ladder_packed_dev -- the particle-particle ladder on packed (unique-pair)
 * amplitudes, reading only the virtual-virtual block of B (the other integral
 * blocks are not built, so it runs at virtual spaces where they would not fit):
 *   Zt[n][ab] = sum_{e<f} <ab||ef> Xt[n][ef]   (= 1/2 sum_ef <ab||ef> X_ij^ef,
 *   the ladder term of Eq. 30 for X antisymmetric in (e,f)),
 *   <ab||ef> = <ab|ef> - <ab|fe>,  <ab|ef> = sum_L B^L_ae B^L_bf.
 *   xt_dev  [ncol][P_V] complex, device: one row per column n (e.g. n = r P_O + ij
 *           for R right-hand sides and the pairs i<j); pairs e<f in row-major
 *           order of the strict upper triangle.  Not modified.
 *   zt_dev  [ncol][P_V] complex, device, overwritten; must not overlap xt_dev.
 *   transpose  1: <ef||ab> = conj <ab||ef>, the holomorphic transpose.
 *   prec    LRCC_FP64, LRCC_MIXED_TF32 or LRCC_MIXED_BF16X3.
 * The context caches <ab||ef> (FP64 or embedded) when it fits in a third of the
 * free device memory; otherwise every call assembles it in slabs from B (an
 * embedded copy of B_vv is then kept for the mixed precisions).  LRCC_ENOMEM
 * if the slab buffers do not fit.  Stream-ordered on `stream`; no sync.
 */
lrcc_status lrcc_ladder_packed_dev(lrcc_ctx* ctx, const double* xt_dev, double* zt_dev, int64_t ncol,
                                   int transpose, int prec, void* stream);

/*
 * lrcc_get_amplitudes -- copy the converged ground-state amplitudes to the host.
 *   which  0: T (CCSD, Eq. 9-10), 1: Lambda (left CCSD).
 *   out    host [O*V + O*O*V*V] complex (singles, then full antisymmetric doubles).
 * LRCC_ESTATE before lrcc_ccsd_ground.
 */
lrcc_status lrcc_get_amplitudes(lrcc_ctx* ctx, int which, double* out);

/* Residual-map applications in the last lrcc_solve: FP64 (outer) and
 * tensor-core (inner) sigma / transpose products, summed over all RHS chunks. */
lrcc_status lrcc_solve_counts(const lrcc_ctx* ctx, int* n_fp64, int* n_mixed);

/* Device timing of the last lrcc_solve / lrcc_ccsd_ground phases (ms):
 * [0] ground T, [1] Lambda, [2] xi/eta, [3] X, [4] F.X, [5] Y, [6] alpha. */
lrcc_status lrcc_phase_times(const lrcc_ctx* ctx, double* ms7);

/* Number of kernels this library launched on ctx since creation. */
int64_t lrcc_kernel_launches(const lrcc_ctx* ctx);

/* Device memory of ctx's allocator since creation, in bytes: held now (live),
 * the most held at once (peak), and the largest single buffer requested
 * (largest; every integral block, amplitude array and workspace is one
 * buffer).  Host-side counters only: no device work, no synchronisation.
 * LRCC_EINVAL on a NULL argument. */
lrcc_status lrcc_memory_stats(const lrcc_ctx* ctx, int64_t* live, int64_t* peak, int64_t* largest);

/*
 * Measurement hooks.  lrcc_profile(ctx, 1) starts recording a CUDA-event pair
 * around every GEMM launch on the context's stream (and clears old records);
 * lrcc_profile(ctx, 0) stops.  lrcc_kernel_stats aggregates the records by
 * kernel name: call with idx = 0, 1, ... until it returns LRCC_EINVAL.
 *   name     out, static string (kernel family)
 *   count    out, launches
 *   ms       out, summed device time of those launches
 *   flops    out, summed algorithmic flops (8 per complex multiply-add)
 *   bytes    out, summed algorithmic operand + result bytes
 * Synchronises the context's stream.
 */
lrcc_status lrcc_profile(lrcc_ctx* ctx, int enable);
/* Write every recorded launch as CSV (kernel,M,N,K,batch,ms,flops) to path. */
lrcc_status lrcc_profile_dump(lrcc_ctx* ctx, const char* path);
lrcc_status lrcc_kernel_stats(lrcc_ctx* ctx, int idx, const char** name, int64_t* count, double* ms,
                              double* flops, double* bytes);

/*
 * lrcc_ladder_noalloc -- the same ladder as lrcc_ladder_dev (FP64 path),
 *   Z_ij^ab = 1/2 sum_ef <ab||ef> X_ij^ef,  <ab|ef> = sum_L Bvv^L_ae Bvv^L_bf,
 * for callers that cannot allocate device memory: it needs no context and
 * calls no allocator (no cudaMalloc, cudaFree or allocating library routine).
 * The paper has no counterpart; this exists for users whose code may not
 * allocate -- e.g. inside a host framework that owns every device byte through
 * its own allocator, or in a latency-critical loop where cudaMalloc/cudaFree
 * (which synchronise the device) must not run.
 *   bvv_dev [L][V][V]        device, complex: the virtual-virtual block of B.
 *   x_dev   [R][O][O][V][V]  device, complex, antisymmetric in (i,j) and (e,f).
 *   z_dev   [R][O][O][V][V]  device, complex, overwritten.
 *   transpose  0: the map above; 1: its holomorphic transpose (B -> conj B).
 *   stream  cudaStream_t (NULL = legacy default stream); the call is
 *           stream-ordered and does not synchronise.
 * Intermediates live in one fixed 32 MiB array in device global memory that
 * every GPU loading this library keeps until process exit.  Problems whose
 * packed amplitudes plus one ladder slab exceed it (2 P_V R P_O complex +
 * one row of <ab|ef> slab, P_n = n(n-1)/2) return LRCC_EINVAL with a message
 * for lrcc_last_error(NULL).  The first call on a device looks up that array's
 * device address (with the device current); with lazy module loading (the
 * CUDA default) that lookup also loads this library's device code and commits
 * the 32 MiB on that device, so make the first call as a warm-up before any
 * stream capture and outside any region where allocation is forbidden.  The
 * looked-up address is cached per device for the life of the process: it is
 * not valid after cudaDeviceReset, so do not call this entry point after a
 * device reset.  All calls share the array: calls whose kernels overlap on
 * the GPU race on it, so serialise them on one stream.
 */
lrcc_status lrcc_ladder_noalloc(const double* bvv_dev, int L, int O, int V, int R, const double* x_dev,
                                double* z_dev, int transpose, void* stream);

/*
 * Host-only planning queries (no device calls): the layout rules of the
 * tensor-core operands and of the per-call <ab||ef> assembly, exposed so that
 * they can be checked without a GPU.
 *
 * lrcc_embed_layout -- layout of one embedded operand of the tcgen05 GEMM:
 * rows of slots * K real values (slots = 6 for LRCC_MIXED_BF16X3, 2 for
 * LRCC_MIXED_TF32).  With batch 1 and rows longer than 16 KB the rows are
 * stored as *n_panels equal panels of *panel_width elements
 * ([panel][row][panel_width], panel_width a multiple of 128 bytes); otherwise
 * one panel whose width is the row padded to 16 bytes.  LRCC_EINVAL for
 * another precision or a size < 1.
 */
lrcc_status lrcc_embed_layout(int prec, int64_t K, int64_t rows, int64_t batch, int64_t* n_panels,
                              int64_t* panel_width);

/*
 * lrcc_plan_slabs -- how the ladder cuts the P_V = V(V-1)/2 rows (a<b) of
 * <ab||ef> into assembly chunks when it is not cached: chunk c covers the
 * pairs (a, b) with a0 <= a < a1 and b0 <= b < b1 (b > a), which are rows
 * [prow0, prow0 + nrows) in pair order.  budget_el bounds the elements of the
 * chunk's GT[(b,f)][(a,e)] intermediate; row_cap > 0 forces single-a chunks of
 * at most row_cap rows (options.slab_rows); consecutive chunks are grouped
 * into contraction GEMMs of at most cap_rows rows (a chunk larger than
 * cap_rows forms its own group).
 *   out [max_slabs][7]   host, per chunk: a0, a1, b0, b1, prow0, nrows, group.
 * Returns the number of chunks (only the first max_slabs are written), or -1
 * for V < 2, budget_el < 1, row_cap < 0, cap_rows < 1 or a NULL out.
 */
int64_t lrcc_plan_slabs(int64_t V, int64_t budget_el, int64_t row_cap, int64_t cap_rows, int64_t* out,
                        int64_t max_slabs);

#ifdef __cplusplus
}
#endif
#endif /* LRCC_H */
