/*
 * lqcd.h -- C ABI of the GB300 (sm_103a) Incremental eigBiCG library.
 *
 * Method: A. Abdel-Rehim, K. Orginos, A. Stathopoulos, "Extending the eigCG
 * algorithm to non-symmetric linear systems with multiple right-hand sides"
 * (Lattice 2009, arXiv:0911.2285).  The library solves the paper's problem
 * (Sec. 1, Eq. main-problem)
 *
 *     A x_i = b_i,   i = 1 .. N_r,
 *
 * for the Wilson-Dirac matrix A = 1 - kappa * D_hop of Sec. 3 (unpreconditioned,
 * periodic boundaries), with two-sided Lanczos / BiCG (Sec. 2), the eigBiCG
 * residual window and its BiCG-eigen restart (Algorithms eigBiCG and
 * BiCG-eigen), and the incremental oblique deflation of later initial guesses
 * (Algorithm Incremental eigBiCG).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice dims = {Lx, Ly, Lz, Lt}; site s = x + Lx*(y + Ly*(z + Lz*t)).
 * Vectors ("fields") hold N = 12*V complex numbers, V = Lx*Ly*Lz*Lt, ordered
 * [site][spin 4][colour 3], each complex as two doubles (re, im): a field is
 * 24*V doubles.  Batches of k fields are k such arrays back to back.
 * Links: [mu 4][site][3][3] complex128 (mu = 0..3 = x, y, z, t), row-major 3x3.
 * D_hop psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)
 *                     + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu),
 * gamma matrices Hermitian in the chiral basis, gamma5 = diag(1,1,-1,-1);
 * A^+ = gamma5 A gamma5 (Sec. 4).
 *
 * Memory: the caller owns every buffer it passes.  With on_device = 0 the
 * pointers are host memory (pageable or pinned); with on_device = 1 they are
 * device pointers on the context's GPU, ordered on the context's stream
 * (managed memory is accepted either way).  lqcd_solve, lqcd_submit,
 * lqcd_deflate and lqcd_apply return LQCD_ERR_ARG, before any copy or launch,
 * when a buffer's memory kind does not match on_device.
 * The context owns its device copies of the links, the residual windows and
 * the accumulated eigenspace.
 *
 * Errors: every call returns lqcd_status; nothing throws across the ABI.  On a
 * non-OK return, outputs are unspecified except the lqcd_solve_info entries,
 * which are always written for every right-hand side that was started.
 * The context stays usable after LQCD_ERR_NOCONV, LQCD_ERR_BREAKDOWN,
 * LQCD_ERR_ARG and LQCD_ERR_STATE; after LQCD_ERR_CUDA or LQCD_ERR_OOM destroy it.
 * Contexts are not thread safe: one host thread per context at a time.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LQCD_OK = 0,
    LQCD_ERR_ARG = 1,        /* invalid argument or unsupported size */
    LQCD_ERR_OOM = 2,        /* device allocation failed / over the HBM budget */
    LQCD_ERR_CUDA = 3,       /* CUDA runtime error (message in lqcd_last_error) */
    LQCD_ERR_NOCONV = 4,     /* maxiter reached before ||b - A x|| <= tol ||b|| */
    LQCD_ERR_BREAKDOWN = 5,  /* BiCG breakdown: |rho| or |sigma| below 1e-14 of its scale */
    LQCD_ERR_TIMEOUT = 6,    /* a bounded device wait gave up */
    LQCD_ERR_STATE = 7       /* call not valid in this state (e.g. empty eigenspace) */
} lqcd_status;

typedef enum {
    LQCD_FP64 = 0,   /* every vector and all arithmetic in FP64 */
    LQCD_MIXED = 1   /* FP32 Krylov vectors/links (third-row reconstruction),
                        FP64 solution and small dense algebra; reliable updates
                        against a double-float (or FP64) true residual; the
                        reported residual of each solution is native FP64 */
} lqcd_precision;

typedef enum {
    LQCD_MODE_AUTO = 0,      /* eigBiCG until n1 sources have fed the eigenspace, then deflated */
    LQCD_MODE_EIGBICG = 1,   /* Algorithm Incremental eigBiCG, phase 1 (deflate, eigBiCG, grow) */
    LQCD_MODE_DEFLATED = 2,  /* phase 2: deflate the initial guess, then BiCG */
    LQCD_MODE_PLAIN = 3      /* BiCG from the given initial guess, no deflation */
} lqcd_mode;

typedef struct {
    int dims[4];              /* Lx, Ly, Lz, Lt; each >= 2 */
    double kappa;             /* hopping parameter (Sec. 3: kappa = 1/(8 + 2 m_q)) */
    int nev;                  /* Ritz pairs kept per restart / per solve (Sec. 2) */
    int m;                    /* window size; must satisfy 2*nev < m <= 64 (Sec. 2: m > 2 nev) */
    int n1;                   /* sources solved by eigBiCG before deflated solves (Alg. Incremental) */
    double tol;               /* stop when ||b - A x|| <= tol ||b|| (FP64 true residual) */
    int maxiter;              /* BiCG iterations per source */
    lqcd_precision precision;
    double deftol;            /* DefTol of Alg. Incremental; 0 disables the re-deflation restart */
    int k_max;                /* right-hand sides per batched launch (1..8); 0 = autotuned: init
                                 times one BiCG iteration on 1, 2, 4 and 8 slots and keeps the
                                 batch size with the most right-hand sides per second */
    size_t hbm_budget_bytes;  /* device memory the context may hold; 0 = whatever is free.
                                 Init fails with LQCD_ERR_OOM when the fixed plan (links,
                                 batch slots, eigenspace, scratch) exceeds it; each eigBiCG
                                 window (2 (m+1) Krylov fields) is allocated when a source
                                 starts eigBiCG and only if it fits: see lqcd_solve and
                                 lqcd_progress */
    int n_def_max;            /* eigenspace capacity in vectors (<= 80); 0 = min(80, n1*nev) */
    double delta;             /* MIXED reliable update when ||r|| < delta * ||r at the last update||
                                 (or < 1e-3 * max||r|| since then); 0 = 0.01 */
    int gamma5;               /* 1 = the gamma5-Hermitian variant of Sec. 4 (A^+ = gamma5 A gamma5):
                                 shadow start rhat_0 = gamma5 r_0, so rhat_j = gamma5 r_j and
                                 phat_j = gamma5 p_j are never stored and A^+ phat = gamma5 A p:
                                 one operator product per BiCG iteration, real scalars; the
                                 eigBiCG window's left vectors are gamma5 images of the right
                                 ones.  0 = general two-sided BiCG with rhat_0 = r_0. */
    int bicgstab;             /* 1 = phase 2 as the paper runs it (Alg. Incremental eigBiCG,
                                 step 3): DEFLATED and PLAIN solves use BiCGStab (shadow
                                 rhat = r_0, two products with A per step, none with A^+),
                                 with the same reliable updates and DefTol restart; eigBiCG
                                 and its correction leg stay BiCG.  0 = BiCG throughout.
                                 Not combinable with gamma5. */
    int evenodd;              /* 1 = even-odd (Schur complement) preconditioning, the form of the
                                 paper's test matrices (Sec. 3): the solver works on the odd half
                                 lattice with A_hat = 1 - kappa^2 D_oe D_eo and
                                 b_hat = b_o + kappa D_oe b_e, and returns the full solution with
                                 x_e = b_e + kappa D_eo x_o; the tolerance and the reported
                                 true_resid are those of the full system in FP64.  Sources and
                                 solutions of lqcd_solve, lqcd_deflate and the session stay full
                                 fields; the eigenspace (lqcd_eigs, lqcd_eigspace_get/set) and
                                 lqcd_apply (which applies A_hat) use half fields of 12 V / 2
                                 complex, odd sites in site order.  All extents must be even;
                                 not combinable with gamma5 or bicgstab. */
    int no_autotune;          /* 1 = skip the init-time autotuners (no counterpart in the paper):
                                 operator-kernel shape 0 (lqcd_set_dslash_variant pins another),
                                 the first FP64 residual shape, and batches of k_max (8 when
                                 k_max = 0).  Faster context creation, and kernel launches
                                 that a profiler can count on.  0 = autotune. */
} lqcd_params;

typedef struct {
    int iters;               /* BiCG iterations */
    int matvecs;             /* products with A or A^+ (the paper's cost unit, Sec. 3) */
    int restarts;            /* BiCG-eigen restarts (eigBiCG mode) */
    int reliable_updates;    /* true-residual recomputations inside the iteration */
    int outer_steps;         /* DefTol re-deflation restarts */
    double true_resid;       /* ||b - A x|| / ||b|| in FP64 at return */
    double seconds;          /* wall time of this right-hand side's batch */
    lqcd_mode mode_used;
} lqcd_solve_info;

typedef struct lqcd_ctx lqcd_ctx;

/* Create a context for one gauge field and parameter set.
 * links: host array [4][V][3][3] complex128 (interleaved doubles); copied.
 * cuda_stream: cudaStream_t to order all work on, or NULL for a private stream.
 * Allocates the device links (FP64 and, for MIXED, FP32 two-row), the batch
 * slots (k_max) and the eigenspace (n_def_max).  Returns LQCD_ERR_ARG for bad
 * dims/kappa/nev/m, LQCD_ERR_OOM when the device memory (or hbm_budget_bytes)
 * is insufficient.  Sec. 2 (m > 2 nev), Sec. 3 (operator). */
lqcd_status lqcd_eigbicg_init(lqcd_ctx **ctx, const lqcd_params *params,
                              const double *links, void *cuda_stream);

/* Solve A x_i = b_i for k right-hand sides (Sec. 1, Eq. main-problem).
 * b: k fields; x: k fields, in = initial guesses (zeros allowed), out = solutions.
 * mode: see lqcd_mode.  EIGBICG: each source is deflated against the current
 * eigenspace, solved by eigBiCG(nev, m) and its nev Ritz pairs are
 * bi-orthogonalized against the eigenspace and appended (Alg. Incremental,
 * phase 1).  When k > 1 all k deflate against the eigenspace as it was at the
 * call and append in index order at the end.  DEFLATED: deflate, BiCG, and with
 * deftol > 0 one re-deflation restart at ||r|| < deftol ||b|| (phase 2).
 * info: k entries (may be NULL).  k may exceed k_max: the sources are then
 * processed in consecutive batches of k_max (for continuous refill of freed
 * slots use the serving session below).  An eigBiCG batch holds one window per
 * source, allocated for as many sources as the memory plan admits (the batch
 * shrinks to fit; LQCD_ERR_OOM if not even one window fits) and released when
 * the batch's Ritz vectors have joined the eigenspace.  In MIXED precision an
 * eigBiCG source runs in two legs: the windowed iteration without reliable
 * updates (which would break the window's Lanczos relation) to the recursive
 * tolerance, then, after its Ritz vectors joined the eigenspace, a deflated
 * correction leg from the FP64 residual with reliable updates (outer_steps = 1).
 * Returns LQCD_ERR_NOCONV / LQCD_ERR_BREAKDOWN if any source failed; x then
 * holds the best iterate. */
lqcd_status lqcd_solve(lqcd_ctx *ctx, int k, const double *b, double *x,
                       int on_device, lqcd_mode mode, lqcd_solve_info *info);

/* Serving session (continuous batching): requests wait in a queue, take a
 * batch slot as soon as one frees up and leave it when their solve ends, while
 * the other slots keep iterating; the gauge field and the eigenspace stay
 * resident.  The mode is resolved at admission (AUTO: eigBiCG while fewer than
 * n1 sources have fed or are feeding the eigenspace, deflated BiCG after).
 * Admission is by device memory: an eigBiCG request also needs a window, which
 * is allocated only if it fits the memory plan (hbm_budget_bytes, else the free
 * device memory less 1 GiB); a request that does not fit waits in the queue and
 * is admitted when a window is released, while later requests that need no
 * window are admitted past it.  When no window is held (none will be released),
 * an AUTO request runs deflated BiCG instead and an explicit EIGBICG request
 * finishes with LQCD_ERR_OOM.
 * The context must not run lqcd_solve while requests are in flight
 * (LQCD_ERR_STATE).
 *
 * lqcd_submit: queue one right-hand side.  b and x are one field each (host or
 * device as on_device says); b is read when the request is admitted, x holds
 * the initial guess until then and receives the solution when it completes:
 * both must stay valid until lqcd_poll reports it done.  *ticket identifies it. */
lqcd_status lqcd_submit(lqcd_ctx *ctx, const double *b, double *x, int on_device, lqcd_mode mode,
                        long long *ticket);

/* Advance the session: wait for the iterations in flight, retire finished
 * requests (final FP64 residual, eigenspace growth, solution written), admit
 * queued requests into free slots (deflation, start vectors) and launch the
 * next chunk of 8 BiCG iterations for every busy slot without waiting for it.
 * wait = 0: if the chunk in flight has not finished yet, return at once and
 * change nothing (lets one host thread drive several contexts, each on its
 * own stream); wait != 0: block until it has.
 * *pending = requests queued or in slots (may be NULL). */
lqcd_status lqcd_progress(lqcd_ctx *ctx, int wait, int *pending);

/* Completion of a submitted request: *done = 1 and *info / *result (the solve's
 * own status, e.g. LQCD_ERR_NOCONV) once it finished (each reported once);
 * *done = 0 while it is queued or running.  LQCD_ERR_ARG for an unknown ticket. */
lqcd_status lqcd_poll(lqcd_ctx *ctx, long long ticket, int *done, lqcd_solve_info *info,
                      lqcd_status *result);

/* Oblique deflation of k initial guesses (Alg. Incremental, steps 2 and 3):
 * x0 <- x0 + U_r d,  with  H d = U_l^+ (b - A x0),  H = U_l^+ A U_r.
 * LQCD_ERR_STATE if the eigenspace is empty. */
lqcd_status lqcd_deflate(lqcd_ctx *ctx, int k, const double *b, double *x0, int on_device);

/* Eigenpairs of A from Rayleigh-Ritz on the accumulated spaces (Sec. 2, last
 * paragraph): the pencil (U_l^+ A U_r, U_l^+ U_r).  *n_inout: in = capacity of
 * the outputs, out = pairs written (<= eigenspace size), smallest |lambda| first.
 * evals: n complex (2n doubles).  evecs_r, evecs_l: n host fields each or NULL.
 * resid: n doubles ||A u - lambda u|| / ||u|| or NULL.  Host pointers only.
 * LQCD_ERR_STATE if the eigenspace is empty. */
lqcd_status lqcd_eigs(lqcd_ctx *ctx, int *n_inout, double *evals,
                      double *evecs_r, double *evecs_l, double *resid);

/* out = A in (dagger = 0) or A^+ in (dagger = 1), in the precision given
 * (LQCD_FP64 or LQCD_MIXED = FP32 operator on FP32-rounded input).  k fields. */
lqcd_status lqcd_apply(lqcd_ctx *ctx, int dagger, lqcd_precision prec, int k,
                       const double *in, double *out, int on_device);

/* Device memory of the context: *plan_bytes = the fixed plan (allocated at init),
 * *window_bytes = one eigBiCG window, *windows_attached = windows held now.
 * Any output may be NULL. */
lqcd_status lqcd_memory_info(const lqcd_ctx *ctx, size_t *plan_bytes, size_t *window_bytes,
                             int *windows_attached);

/* Right-hand sides per batched launch: k_max, or the autotuned size (k_max = 0). */
int lqcd_batch_size(const lqcd_ctx *ctx);

/* Measurement hook: ms[k] (k = 0..8) = device time of one BiCG iteration
 * (operator kernel, residual update, direction update) over k slots as the
 * batch-size autotuner measured it (0 where not timed).  LQCD_ERR_STATE if the
 * context was created with k_max > 0 (no autotuning). */
lqcd_status lqcd_batch_timings(const lqcd_ctx *ctx, double *ms);

/* Size of the eigenspace (number of right/left vector pairs). */
int lqcd_eigspace_size(const lqcd_ctx *ctx);

/* Copy the eigenspace out (checkpoint): Ur, Ul host fields (n each, may be
 * NULL), H = U_l^+ A U_r as n x n complex row-major (may be NULL). */
lqcd_status lqcd_eigspace_get(lqcd_ctx *ctx, double *Ur, double *Ul, double *H);

/* Replace the eigenspace (resume / tests): n pairs of host fields; H is
 * recomputed on the device as U_l^+ A U_r in FP64 and factorised.
 * n = 0 empties it and restarts the LQCD_MODE_AUTO count of eigBiCG sources;
 * n > 0 counts as a complete eigenspace (AUTO then deflates).
 * LQCD_ERR_ARG if n > n_def_max. */
lqcd_status lqcd_eigspace_set(lqcd_ctx *ctx, int n, const double *Ur, const double *Ul);

/* Inspect the eigBiCG window of the most recent eigBiCG solve (batch slot
 * 'slot'): *vs = vectors in the window, H = vs x vs complex row-major (capacity
 * m*m), ritz = its nev final Ritz values (complex, may be NULL), restarts. */
lqcd_status lqcd_last_window(lqcd_ctx *ctx, int slot, int *vs, double *H,
                             double *ritz, int *restarts);

/* Device eigensolver for small dense complex matrices, exposed for tests:
 * C is n x n complex row-major (host), n <= 80.  Returns all eigenvalues
 * (smallest |lambda| first, exact ties by Im), right vectors Y (column j of an
 * n x n row-major array, unit 2-norm, largest-modulus entry real > 0) and left
 * vectors Z (Z^H Y = I on the diagonal).  Y, Z may be NULL. */
lqcd_status lqcd_small_eig(int n, const double *C, double *evals, double *Y, double *Z);

/* Coefficient part of Algorithm BiCG-eigen on the device, exposed for tests:
 * H is m x m complex row-major (host).  Outputs *r (vectors kept, <= 2 nev),
 * Yc, Zc (m x r row-major complex, capacity m*2nev) and lam (r complex). */
lqcd_status lqcd_restart_coefficients(int m, int nev, const double *H, int *r,
                                      double *Yc, double *Zc, double *lam);

/* Measurement hook (not part of the paper's method): number of kernels this
 * library has launched in the process so far (graph replays count their nodes). */
long long lqcd_kernel_launches(void);

/* Measurement hook: average device time (CUDA events on the context's stream)
 * of one launch of an iteration kernel over batch slots 0..k-1, on whatever the
 * slot buffers hold, repeated reps times. kernel: 0 = operator pair
 * A p, A^+ phat (Krylov precision) with the fused sigma reduction; 1 = residual
 * update; 2 = direction update; 3 = FP64 true residual + reliable-update
 * replacement; 10 + v = operator pair in kernel shape v (v < 30), 99 = the plane-
 * streaming operator pair (see lqcd_dslash_variant). Leaves the slots idle. */
lqcd_status lqcd_time_kernel(lqcd_ctx *ctx, int kernel, int k, int reps, double *avg_ms);

/* Implementation switch (no counterpart in the paper): on != 0 (the default)
 * runs the FP32 Galerkin projections (U_l^H r, growth blocks) and the FP32
 * restart window product V <- V Yc, W <- W Zc on the tensor cores (3xTF32
 * tcgen05 MMAs) where the shapes allow (m <= 64, 2 nev <= 24, 12 V a multiple
 * of 128); on = 0 uses the CUDA-core kernels. Results agree to FP32 rounding,
 * not bit for bit. Waits for the context's stream; LQCD_ERR_STATE while
 * serving requests are in flight. */
lqcd_status lqcd_set_tensor_cores(lqcd_ctx *ctx, int on);

/* Measurement hook: the operator-kernel shape the autotuner picked at init
 * (timing every shape on this lattice with a full batch): 0..29, or 100 for
 * the plane-streaming kernel; -1 for NULL. Shapes 25..29 are the 4-D brick
 * kernels that compute every slot of a batch in one block. */
int lqcd_dslash_variant(const lqcd_ctx *ctx);

/* Pins the operator-kernel shape (0..29 or 100, as above) instead of the
 * autotuner's choice; the iteration graphs are rebuilt on next use. Waits for
 * the context's stream. LQCD_ERR_ARG for a shape this context cannot use
 * (lattice extents, FP64 Krylov vectors: shape 0 only, gamma5 variant: the
 * one-operator shapes, even-odd operator: none), LQCD_ERR_STATE while serving
 * requests are in flight. */
lqcd_status lqcd_set_dslash_variant(lqcd_ctx *ctx, int variant);

/* Test hook: one launch of the BiCG operator-pair kernel of shape 'variant'
 * (0..29 or 100, see lqcd_dslash_variant) on k host fields p, phat (Krylov
 * precision of the context): Ap = A p, Ahp = A^+ phat (host outputs), and
 * sigma = (phat, A p) per field (k complex, may be NULL).  Uses batch slots
 * 0..k-1 and leaves them idle.  LQCD_ERR_ARG for a shape this lattice cannot
 * use; LQCD_ERR_TIMEOUT if a bounded wait in the kernel gave up. */
lqcd_status lqcd_apply_pair(lqcd_ctx *ctx, int variant, int k, const double *p, const double *phat,
                            double *Ap, double *Ahp, double *sigma);

/* Inner-product matrix of FP32 fields, the Galerkin projections of the
 * deflation and the eigenspace growth (Sec. 2, Alg. Incremental eigBiCG:
 * U_l^H r and U_l^H A U_r): C[i*b + j] = sum_e conj(X_i(e)) Y_j(e) for i < a,
 * j < b.  X, Y: DEVICE pointers to a (resp. b) consecutive fields of n complex
 * FP32 numbers (re, im interleaved, 16-byte aligned).  C: HOST, a*b complex
 * (2ab doubles).  path 0 = CUDA cores (FP32 products, FP64 block sums),
 * path 1 = tensor cores (3xTF32 tcgen05 MMAs, FP32 runs summed in FP64;
 * needs 2n divisible by 32 and a <= 512, else LQCD_ERR_ARG).  With reps > 0
 * the call is repeated reps more times and *avg_ms receives the mean device
 * time of one call.  Allocates its scratch; synchronises the device. */
lqcd_status lqcd_field_dots(int a, const float *X, int b, const float *Y, long long n, int path, int reps,
                            double *C, double *avg_ms);

/* Allocation-free eigen-solver (no counterpart in the paper; a service for
 * callers that cannot allocate device memory when they need a small
 * eigen-solve: applications that give all device memory to their own pool or
 * a fixed budget up front, and latency-critical loops where the implicit device
 * synchronisation of cudaMalloc/cudaFree would stall other streams).
 * Same results as lqcd_small_eig, but C (n x n complex row-major), evals (n
 * complex) and Y, Z (n x n, or both NULL for eigenvalues only) are DEVICE
 * pointers on the current device, and nothing is allocated: the scratch lives
 * in a file-scope device array sized for n <= 80 (about 200 KiB, held by every
 * GPU that loads the library until the process exits).  n > 80 returns
 * LQCD_ERR_ARG.  The first call on a device looks up that array's device
 * address and sets the kernel's shared-memory limit, so make the first call
 * before any stream capture; that set-up is kept for the life of the process
 * (a cudaDeviceReset between calls is not supported).  Work is ordered on
 * 'cuda_stream' (cudaStream_t, NULL = default stream) and the call returns
 * after it completes.  All calls on
 * a device share the scratch array and it keeps the last call's contents: calls
 * whose kernels overlap on the GPU (other streams, other host threads) race.
 * LQCD_ERR_NOCONV if the QR iteration did not converge. */
lqcd_status lqcd_small_eig_noalloc(int n, const double *C, double *evals, double *Y, double *Z,
                                   void *cuda_stream);

/* Failure-detection hook (no counterpart in the paper): bound of every
 * device-side wait in this library's kernels (TMA/mbarrier pipelines, the flag
 * wait below), in SM clock cycles, on the current device.  A kernel whose wait
 * runs out records an error word and returns; the call that launched it then
 * returns LQCD_ERR_TIMEOUT.  cycles <= 0 restores the default (4e9 cycles,
 * about 2 s at 2 GHz).  Affects kernels launched after the call. */
lqcd_status lqcd_set_wait_limit(long long cycles);

/* Failure-detection hook: one kernel whose single thread waits, with the
 * library's bounded wait, for the device word *flag (DEVICE pointer) to become
 * nonzero.  LQCD_OK if it was (or became) nonzero within the limit,
 * LQCD_ERR_TIMEOUT if the wait gave up.  Ordered on 'cuda_stream' (NULL =
 * default stream); returns after the kernel has finished. */
lqcd_status lqcd_wait_flag(const int *flag, void *cuda_stream);

/* Text for a status code. */
const char *lqcd_status_str(lqcd_status s);

/* Last error message recorded by this thread (CUDA error text etc.). */
const char *lqcd_last_error(void);

/* Release every device resource of the context. NULL is accepted. */
void lqcd_destroy(lqcd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
