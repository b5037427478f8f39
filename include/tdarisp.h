/*
 * tdarisp.h -- C ABI of the GB300 TDA-risp library (libtdarisp.so).
 *
 * The library computes the Tamm-Dancoff TDA-risp excitation energies of
 * arXiv 2603.29257 on one GPU:
 *
 *   A_{ia,jb} = (e_a - e_i) d_ij d_ab + 2 (ia|jb) - c_x (ij|ab)          Sec. 2, Eq. TDA-risp
 *
 * and, with tr_options.tddft = 1, full TDDFT-risp with B_{ia,jb} = 2 (ia|jb)
 * - c_x (ib|ja) (Sec. 2, Eqs. tddft and hessian),
 * with both electron-repulsion terms factorised through the minimal
 * auxiliary basis (Sec. 2, Eqs. RI and g(r)): one s and one p primitive per
 * non-hydrogen atom for the Coulomb term, the s primitive only for the
 * exchange term, no auxiliary functions on hydrogen (Sec. 3.2), exchange
 * restricted to the orbital-energy window |e| < window_ev (Sec. 3.2), and
 * range-separated exchange with the operator (alpha + beta erf(omega r))/r
 * used both in the three-centre integrals and in the metric (Sec. 3.2, Eqs.
 * RSH and K_mia_RSH).  Davidson diagonalisation follows Sec. 3.3.
 *
 * Conventions
 *   - Units: bohr and Hartree.
 *   - AO function: chi(r) = sum_k coef[k] * Y(r - A) * exp(-exp[k] |r - A|^2);
 *     the coefficients are used as given (normalisation folded in).
 *     Y = 1 (l=0); x, y, z (l=1); for l=2 the real solid harmonics in the
 *     order xy, yz, (2zz - xx - yy)/(2 sqrt 3), xz, (xx - yy)/2.
 *   - Auxiliary function on atom A with exponent c: exp(-c |r-A|^2) (s) and
 *     x, y, z times it (p), unnormalised; order per atom: s, px, py, pz.
 *   - Matrices are row-major.  Trial vectors are X[m][nocc][nvir] with the
 *     virtual index fastest.
 *   - Orbital energies must be in ascending order; the exchange window is
 *     then the contiguous block occ [nocc - noccK, nocc) x vir [0, nvirK).
 *
 * Ownership: the caller owns every buffer it passes; the library copies what
 * it keeps.  The context owns its device memory until tr_destroy.  A pointer
 * flagged "on_device" must be a device pointer of the context's device.
 *
 * Errors: every call returns TR_OK (0) or a negative code; tr_last_error()
 * describes the last failure.  No call aborts the process.  Calls on one
 * context must not run concurrently from several host threads.
 */
#ifndef TDARISP_H
#define TDARISP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TR_OK 0
#define TR_EINVAL (-1)    /* invalid argument or call order */
#define TR_ENOMEM (-2)    /* device or pinned host allocation failed / budget exceeded */
#define TR_ECUDA (-3)     /* CUDA runtime error */
#define TR_ENOCONV (-4)   /* Davidson hit max_iter; outputs hold the best estimates */
#define TR_ENOTPD (-5)    /* an auxiliary metric is not positive definite */
#define TR_ETIMEOUT (-6)  /* a bounded device wait ran out (tensor-core pipelines, see
                             tr_options.wait_cycles); the kernel gave up, awaited its own
                             copies and products in flight and freed its tensor memory, so
                             the context stays usable; the outputs of that call are invalid */

#define TR_FP64 0   /* every step in FP64 */
#define TR_MIXED 1  /* MO tensors and J/K contractions in FP32 / 3xTF32 tensor cores;
                       integrals, metrics and the Davidson driver in FP64 */
#define TR_FP64_TC 2 /* FP64 results with the MO transforms and the J and K
                        contractions on the bf16 tensor cores: every FP64 operand is
                        split into 7 integer slices (Ozaki scheme), slice products are
                        summed exactly; integrals, metrics, Davidson in FP64 */

typedef struct tr_ctx tr_ctx;

/* One contracted AO shell (l = 0, 1 or 2). */
typedef struct {
    int atom;            /* index into the molecule's atoms */
    int l;               /* angular momentum */
    int nprim;           /* 1..16 */
    const double *exp;   /* nprim exponents */
    const double *coef;  /* nprim literal coefficients */
} tr_shell;

typedef struct {
    /* exchange term: coefficient cx and operator (k_alpha + k_beta erf(omega r))/r.
       Global hybrid: k_alpha = 1, k_beta = 0, omega = 0.
       Range-separated (Sec. 3.2, Eq. RSH): cx = 1, k_alpha = SR fraction,
       k_alpha + k_beta = LR fraction, omega > 0. */
    double cx, k_alpha, k_beta, omega;
    double window_ev;    /* exchange window in eV (Sec. 3.2); <= 0 disables it */
    int aux_on_h;        /* 0 (default): no auxiliary functions on hydrogen (Sec. 3.2) */
    int nstates;         /* number of excited states */
    int block;           /* initial trial vectors (0: 2 * nstates) */
    int max_space;       /* subspace size that triggers a restart (0: 20 * nstates) */
    int max_iter;        /* Davidson iterations (0: 200) */
    double tol;          /* residual 2-norm threshold per state */
    int precision;       /* TR_FP64, TR_MIXED or TR_FP64_TC */
    double screen;       /* primitive-pair screening threshold (0: 1e-22) */
    size_t hbm_budget;   /* bytes of device memory the context may hold (0: 90% of free) */
    size_t aux_chunk_bytes; /* scratch for AO integral chunks (0: 12 GiB) */
    size_t host_budget;  /* pinned host bytes for spilled Davidson vectors (0: unlimited);
                            the subspace is capped so that V and W fit, which triggers
                            restarts earlier (Sec. 3.3) */
    int dav_dev_rows;    /* cap on Davidson vectors kept on the device (0: as many as the
                            HBM budget allows); rows beyond it live in pinned host memory */
    size_t matvec_ws_bytes; /* scratch for the exchange intermediate M (0: 4 GiB) */
    int xform_slices;    /* MO transforms: -1 FP64 pipe; 2..7 bf16 tensor cores with that many
                            Ozaki slices per operand (7 + 8 (S-1) bits below each row's
                            largest element); 0: FP64 pipe in TR_FP64, 5 slices in TR_MIXED,
                            7 in TR_FP64_TC */
    int j_ao;            /* Coulomb term: 0 (default) from the stored (P|ia); 1 on the fly in
                            the AO basis (Sec. 3.1, Eq. J_mia): AO transition densities D^m,
                            R = (Q|kl) D^m with the three-centre integrals generated per
                            auxiliary chunk, R~ = (P|Q)^-1 R, U^m = (mn|P) R~, J = C_occ^T U^m
                            C_vir, all in FP64 in every precision; no (P|ia) tensor is built
                            (tr_get_tensor 0 then fails) */
    int tddft;           /* 0 (default): Tamm-Dancoff (Eq. TDA-risp); 1: full TDDFT-risp
                            (Sec. 2, Eqs. tddft and hessian, no XC kernel):
                              A + B = D + 4 (ia|jb) - c_x [(ib|ja) + (ij|ab)]
                              A - B = D + c_x [(ib|ja) - (ij|ab)]
                            (the printed A + B has 2 (ia|jb); 4 is the coefficient for
                            which (A+B + A-B)/2 is the A above).  tr_build then also forms
                            T_ia^P' on the exchange window (Sec. 3.2, the tensor only full
                            TDDFT needs), and tr_solve solves (A-B)(A+B)|X+Y> = Omega^2|X+Y>.
                            FP64 results: needs precision TR_FP64 or TR_FP64_TC (then the
                            (ib|ja) products run as 7-slice tensor-core products too);
                            not available in tr_solve_batch or the server (TR_EINVAL);
                            tr_matvec and tr_matvec_noalloc still give A X */
    long long wait_cycles; /* bounded device waits: SM clock cycles before a pipeline wait of
                            the tensor-core kernels (TR_MIXED exchange stages, every sliced
                            product of TR_FP64_TC and of the sliced MO transforms) gives up
                            (0: 2e9, about 1 s).  The call that finds a wait ran out returns
                            TR_ETIMEOUT: tr_build, tr_solve, and tr_matvec / tr_matvec_tddft
                            with host buffers (with device buffers they are asynchronous and
                            report nothing).  Must be >= 0 */
    int wait_test;       /* test of the bounded waits only (0 default): 1 = the tensor-core
                            kernels load no operands, so their first pipeline wait can only
                            end by running out (after wait_cycles); the calls above then
                            return TR_ETIMEOUT.  Nothing is faulted or left in flight */
} tr_options;

typedef struct {
    int nao, nmo, nocc, nvir;
    int naux_j, naux_k;  /* auxiliary functions for J (s+p) and K (s) */
    int occ_k0, nocc_k;  /* exchange window: occupied [occ_k0, occ_k0 + nocc_k) */
    int nvir_k;          /*                  virtual  [0, nvir_k) (relative to nocc) */
    int npair;           /* AO shell pairs kept by screening */
    int ntotal_pair;     /* AO shell pairs before screening */
} tr_dims;

typedef struct {
    int niter, nmatvec, nrestart, converged;
    double t_matvec_ms, t_ortho_ms, t_eigh_ms, t_other_ms;
    int max_space;       /* subspace size used (after the memory caps) */
    int dev_rows;        /* Davidson vectors (V and W rows) held on the device */
    long long host_bytes_moved; /* bytes streamed between pinned host memory and HBM */
} tr_solve_info;

/* Per-kernel timing, recorded with CUDA events on the context stream when
   profiling is enabled. */
typedef struct {
    char name[32];
    long launches;
    double total_ms;
    double flops;        /* algorithmic flops of all recorded launches */
    double bytes;        /* algorithmic bytes of all recorded launches */
} tr_prof_entry;

/* Library version (major*10000 + minor*100 + patch). */
int tr_version(void);

/* Fill opt with the defaults named above (cx = 0.25 global hybrid, 40 eV window,
   5 states, tol 1e-5). */
void tr_options_default(tr_options *opt);

/* Create a context on the current CUDA device.  cuda_stream: a cudaStream_t
   (NULL = the legacy default stream); all work of the context is ordered on it.
   Errors: TR_EINVAL (opt NULL or out NULL), TR_ECUDA. */
int tr_create(tr_ctx **out, const tr_options *opt, void *cuda_stream);

/* Release every device and host resource of ctx (NULL is accepted). */
void tr_destroy(tr_ctx *ctx);

/* Text of the last error of ctx (never NULL; "" if none). */
const char *tr_last_error(const tr_ctx *ctx);

/* Replace the options (takes effect at the next tr_build / tr_solve). */
int tr_set_options(tr_ctx *ctx, const tr_options *opt);

/* Molecule (Sec. 2: geometry, AO and auxiliary basis).
   Z[natm] nuclear charges; xyz[natm*3] in bohr; aux_exp[natm] exponent of the
   auxiliary s/p primitive of each atom (<= 0: none; hydrogen gets none unless
   aux_on_h); shells[nshell] AO shells.  Host pointers; the library copies them.
   Errors: TR_EINVAL for l outside 0..2, nprim outside 1..16, atom out of range. */
int tr_set_molecule(tr_ctx *ctx, int natm, const int *Z, const double *xyz,
                    const double *aux_exp, int nshell, const tr_shell *shells);

/* MO coefficients C[nao][nmo] (row-major) and orbital energies eps[nmo]
   (ascending, Hartree); the first nocc orbitals are occupied.  on_device != 0:
   both pointers are device pointers.  Errors: TR_EINVAL (sizes, order). */
int tr_set_orbitals(tr_ctx *ctx, int nao, int nmo, int nocc, const double *C,
                    const double *eps, int on_device);

/* Sizes derived from the molecule, orbitals and options. */
int tr_get_dims(tr_ctx *ctx, tr_dims *out);

/* Build the factorised response operator (Sec. 2 Eq. RI, Sec. 3.2):
   the metrics (P|Q) and their Cholesky factors, the three-centre integrals
   (P|mu nu) over screened AO pairs, the Coulomb tensor (P|ia) and the window
   exchange tensors T_ij^P = sum_Q (ij|Q)(Q|P)^-1 and T_ab^P = (ab|P).
   Errors: TR_EINVAL (call order), TR_ENOMEM, TR_ENOTPD, TR_ECUDA. */
int tr_build(tr_ctx *ctx);

/* Raw AO three-centre integrals for auxiliary functions [p0, p0+np) of set
   which (0 = Coulomb set s+p, Coulomb operator; 1 = exchange set s, exchange
   operator) into out_dev[np][nao][nao] (device, full square; pairs dropped by
   screening are zero).  Valid after tr_set_molecule. */
int tr_int3c(tr_ctx *ctx, int which, int p0, int np, double *out_dev);

/* Auxiliary metric of set which into out_dev[n][n] (device). */
int tr_int2c(tr_ctx *ctx, int which, double *out_dev);

/* Copy a built tensor to out (host, or device if on_device):
   0: (P|ia)      [naux_j][nocc][nvir]
   1: T_ij^P      [naux_k][nocc_k][nocc_k]   (inverse K metric applied)
   2: T_ab^P      [naux_k][nvir_k][nvir_k]
   3: e_a - e_i   [nocc][nvir]
   4: L^-1 (P|ia) [naux_k][nocc_k][nvir_k]   (full TDDFT only: K operator, window,
                  L the Cholesky factor of the K metric, so that
                  sum_P t^P_ib t^P_ja = (ib|ja) in the RI approximation) */
int tr_get_tensor(tr_ctx *ctx, int which, double *out, int on_device);

/* AX = A X for m trial vectors X[m][nocc][nvir] -> AX[m][nocc][nvir].
   on_device != 0: device pointers, the call is asynchronous on the context
   stream; otherwise host pointers and the call returns when AX is written.
   X and AX must not overlap.  Requires tr_build. */
int tr_matvec(tr_ctx *ctx, int m, const double *X, double *AX, int on_device);

/* Full TDDFT-risp products (Sec. 2, Eq. hessian) for m trial vectors
   X[m][nocc][nvir]: ApBX = (A + B) X and AmBX = (A - B) X, same layout.  Needs
   a context built with tddft = 1.  on_device: device pointers, asynchronous on
   the context stream; otherwise host pointers, returns when both are written.
   The three arrays must not overlap.  Errors: TR_EINVAL (tddft = 0, not built,
   null pointers, overlap). */
int tr_matvec_tddft(tr_ctx *ctx, int m, const double *X, double *ApBX, double *AmBX, int on_device);

/* Electric transition dipoles of n states in the dipole length form with Y = 0
   (Tamm-Dancoff; Sec. 2, Eq. transition):
       mu[k][d] = sqrt(2) sum_ia <i| r_d - origin_d |a> X[k][i][a],   d = x, y, z,
   atomic units (bohr).  The sqrt(2) is the singlet spin adaptation for unit-norm
   X (the vectors tr_solve returns).  X [n][nocc][nvir], mu [n][3]; origin: 3
   host doubles (NULL: the coordinate origin; the dipoles of orthogonal states do
   not depend on it).  on_device: X and mu device pointers, else host.  Needs
   tr_set_molecule and tr_set_orbitals (not tr_build); synchronous.
   Errors: TR_EINVAL (n < 0, null pointers, no molecule or orbitals). */
int tr_transition_dipoles(tr_ctx *ctx, int n, const double *X, const double *origin, double *mu,
                          int on_device);

/* Oscillator strengths f[k] = 2/3 omega[k] |mu_k|^2 of n states (Sec. 2, Eq.
   oscillator_strength) from their excitation energies omega[n] (Ha) and vectors
   X [n][nocc][nvir], with mu_k as in tr_transition_dipoles.  on_device: omega, X
   and f device pointers, else host.  Synchronous.  Errors: as above. */
int tr_oscillator_strengths(tr_ctx *ctx, int n, const double *omega, const double *X, double *f,
                            int on_device);

/* Size of the static device scratch used by tr_matvec_noalloc. */
#define TR_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

/* AX = A X like tr_matvec with device pointers, for callers that cannot
   allocate device memory: code recording the product into a CUDA graph (no
   cudaMalloc/cudaFree during stream capture), code living under another
   allocator with a hard cap, and loops that cannot afford cudaMalloc's implicit
   device synchronisation.  The paper has no counterpart; it is a deployment
   variant of the same product.
   All scratch (J and K intermediates, split-K partial sums) comes from one
   file-scope device array of TR_NOALLOC_SCRATCH_BYTES that every GPU loading
   the library holds until exit; nothing is allocated.  The first call on a
   device looks up that array's address with the device current, so make it
   before any stream capture.  Calls whose GPU work overlaps (other streams or
   contexts at the same time) race on the shared array; no region relies on
   what a previous call left in it.  X and AX: device pointers [m][nocc][nvir],
   not overlapping; asynchronous on the context stream; requires tr_build.
   Errors: TR_EINVAL when 2 naux_j + 2 nocc_k nvir_k doubles per vector plus
   65536 doubles exceed the array (the message says so), when the context's
   device is not current, for a TR_MIXED context (only the FP64 form is
   available here), or as tr_matvec. */
int tr_matvec_noalloc(tr_ctx *ctx, int m, const double *X, double *AX);

/* Davidson solve for the lowest nstates (Sec. 3.3).  Outputs (host, or device
   if on_device): omega[nstates] (Hartree, ascending); X[nstates][nocc][nvir]
   (may be NULL; unit norm, largest-magnitude component positive);
   resid[nstates] (may be NULL).  info may be NULL.  Returns TR_ENOCONV when
   max_iter is reached (outputs filled with the current estimates). */
int tr_solve(tr_ctx *ctx, double *omega, double *X, double *resid, int on_device,
             tr_solve_info *info);

/* Davidson solve of full TDDFT-risp (tddft = 1; Sec. 2, Eq. tddft; Sec. 3.3):
   one expansion basis V serves X+Y and X-Y; (A+B) and (A-B) are both projected
   on it, the projected problem M- M+ a = Omega^2 a is solved through the
   Cholesky factor L of M- (L^T M+ L symmetric), and each unconverged state adds
   the two directions of the diagonal preconditioner of the 2 x 2 response system.
   Outputs (host, or device if on_device): omega[nstates] (Ha, ascending);
   XpY and XmY [nstates][nocc][nvir] (either may be NULL), X+Y and X-Y with
   (X+Y).(X-Y) = 1, the largest-magnitude component of X+Y positive;
   resid[nstates] = sqrt(|(A+B)(X+Y) - Omega (X-Y)|^2 + |(A-B)(X-Y) - Omega (X+Y)|^2)
   (may be NULL).  tr_solve on such a context is this call with XmY = NULL.
   Transition dipoles and oscillator strengths of these states: pass X+Y to
   tr_transition_dipoles / tr_oscillator_strengths (Eq. transition).
   Errors: TR_EINVAL (tddft = 0 or not built), TR_ECUDA (A - B projected on the
   subspace not positive definite, subspace eigensolver), TR_ENOCONV. */
int tr_solve_tddft(tr_ctx *ctx, double *omega, double *XpY, double *XmY, double *resid, int on_device,
                   tr_solve_info *info);

/* tr_build of n contexts concurrently: nthreads host threads (0: 8), each
   context on a stream of its own for the duration of the call.  Returns TR_OK
   or the first error (each context keeps its own error text). */
int tr_build_batch(tr_ctx **ctxs, int n, int nthreads);

/* Davidson solves of n built contexts (n molecules, each with its own options)
   advanced in lockstep: every molecule works on a stream of its own, and the
   matrix-vector products of one Davidson step of all molecules are one CUDA
   graph launch (recorded once, replayed every step, recorded again when the set
   of unconverged molecules changes).  autotune_tiles != 0: before the solve, each
   TR_MIXED context times its tensor-core K stages with 64- and 128-wide output
   tiles and keeps the faster.  Outputs per molecule as tr_solve (omega[i], X[i]
   may be NULL, resid[i] may be NULL; infos may be NULL, else n entries; the
   graph time is reported as every molecule's t_matvec_ms).  Returns TR_OK, or
   TR_ENOCONV if any molecule did not converge, or the first error; the error
   text is copied to every context.  The contexts must be distinct and on the
   current device; their streams are synchronised at entry and exit. */
int tr_solve_batch(tr_ctx **ctxs, int n, double **omega, double **X, double **resid, int on_device,
                   tr_solve_info *infos, int autotune_tiles);

/* ---- Serving runtime -------------------------------------------------------
   Continuous batching of solves as requests arrive (not in the paper, which
   runs one molecule at a time).  A builder thread admits requests in arrival
   order when their estimated device footprint (tr_memory) fits in what is left
   of the server budget -- a request larger than the whole budget is rejected with
   TR_ENOMEM -- and builds them on streams of their own; a solver thread keeps
   each built molecule's tensors and Davidson state resident and advances all of
   them in lockstep, the products of one step being one CUDA-graph launch.
   Molecules join at the next step after their build and leave when converged,
   returning their memory to the budget.  Builds overlap with solver steps. */
typedef struct tr_server tr_server;

typedef struct {
    int max_active;      /* molecules in the solver at once (0: 64) */
    size_t hbm_budget;   /* device bytes for all admitted requests (0: 90% of free) */
    int autotune_tiles;  /* pick the tensor-core tile width per molecule (TR_MIXED) */
    int build_threads;   /* builds in flight at once (0: 4); admission stays in arrival order */
} tr_server_options;

typedef struct {
    int natm;
    const int *Z;
    const double *xyz;
    const double *aux_exp;
    int nshell;
    const tr_shell *shells;
    int nao, nmo, nocc;
    const double *C;     /* host, [nao][nmo] */
    const double *eps;   /* host, [nmo] ascending */
    tr_options opt;      /* functional, window, states, tolerance, precision */
    int want_x;          /* return the excitation vectors (tr_result.X) */
} tr_request;

typedef struct {
    long long id;
    int status;          /* TR_OK, TR_ENOCONV, TR_ENOMEM (rejected), ... */
    int nstates;
    double omega[64];
    double resid[64];
    double *X;           /* [nstates][nocc][nvir] if requested; release with tr_free */
    double t_submit, t_admit, t_built, t_done;  /* seconds on the server clock */
    int niter, nmatvec;
    char error[160];
    int j_ao;            /* 1 if the request ran with the Coulomb term on the fly in the AO
                            basis (its (P|ia) did not fit in the server budget) */
} tr_result;

/* Lowest nev eigenpairs of the symmetric k x k matrix H (row-major, not
   modified) with the device eigensolver of the Davidson driver (the small
   subspace eigenproblem of Sec. 3.3): Householder tridiagonalisation, Sturm
   multisection and inverse iteration in one thread-block cluster, on the
   context's stream.  w[nev] ascending; Y[k][nev] row-major, column i the unit
   eigenvector of w[i] (sign arbitrary).  on_device: H, w, Y are device
   pointers.  Needs no molecule.  Errors: TR_EINVAL (nev > k, null pointers). */
int tr_subspace_eigh(tr_ctx *ctx, int k, const double *H, int nev, double *w, double *Y, int on_device);

/* Start a server on the current device (opt may be NULL). */
int tr_server_create(tr_server **out, const tr_server_options *opt);
/* Queue a request (all arrays copied); *id receives its identifier. */
int tr_server_submit(tr_server *srv, const tr_request *req, long long *id);
/* Move up to max finished results to out; waits up to timeout_ms (< 0: until a
   result arrives or nothing is outstanding; 0: no wait).  Returns the count. */
int tr_server_poll(tr_server *srv, tr_result *out, int max, int timeout_ms);
/* Requests submitted whose results have not been polled yet. */
int tr_server_outstanding(tr_server *srv);
/* Seconds since the server started (the clock of tr_result times). */
double tr_server_clock(tr_server *srv);
/* Stop the threads (unfinished requests are dropped) and release everything. */
void tr_server_destroy(tr_server *srv);
void tr_free(void *p);

/* Kernel timing: enable (1) / disable (0) and reset the counters. */
int tr_profile(tr_ctx *ctx, int enable);
/* Copy up to max entries; returns the number of entries (>= 0) or an error. */
int tr_profile_get(tr_ctx *ctx, tr_prof_entry *out, int max);
/* Device memory of the context: bytes held now, the peak so far, and an
   estimate of the peak of tr_build + tr_solve from the sizes (valid after
   tr_set_orbitals; used for admission by the serving runtime).  Any pointer may
   be NULL. */
int tr_memory(tr_ctx *ctx, size_t *used, size_t *peak, size_t *estimate);

/* Number of kernels this context has launched since creation. */
long tr_launch_count(const tr_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* TDARISP_H */
