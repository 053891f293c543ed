/*
 * ovl.h -- C ABI of libovl, a single-GPU (GB300, sm_103a) implementation of
 * the overlap Dirac operator and its propagator solve.
 *
 * Method (Lujan, Alexandru, Lee, "Electric polarizability of hadrons with
 * overlap fermions on multi-GPUs", Lattice 2011):
 *   Sec. 2, eq. 1   D_ov = 1 + gamma5 sign(H_w),  H_w = gamma5 D_w;
 *   Sec. 2          sign(H_w) ~ Q P(Q^2) on the large space, Q = H_w/||H_w||,
 *                   P a degree-n polynomial approximating x^{-1/2} on [eps, 1];
 *                   exact on the small space spanned by low eigenvectors of Q;
 *   Sec. 2, eq. 2   delta = |1 - sqrt(x) P(x)| ~ A exp(-b n sqrt(eps));
 *   Sec. 3.2        CG for D^{-1} psi, single precision late in the solve;
 *                   multi-mass CG: several quark masses from one Krylov space;
 *   Sec. 4          background field: U_mu -> exp(-i q A_mu) U_mu, Dirichlet
 *                   boundaries in the field direction and in time.
 *
 * Conventions (the paper does not fix them):
 *   D_w psi(n) = (4 + m0) psi(n) - 1/2 sum_mu [(1 - gamma_mu) U_mu(n) psi(n+mu)
 *                                           + (1 + gamma_mu) U_mu(n-mu)^+ psi(n-mu)]
 *   Euclidean chiral basis, gamma5 = diag(1, 1, -1, -1); mu = 0..3 is x, y, z, t.
 *   The field phase is exp(i phi t) on x links, phi = q E, t = 0..Lt-1.
 *   Massive operator D(m) = (1 - m/2) D_ov + m.
 *   P(x) = sum_k c_k T_k(y), y = (2x - 1 - eps)/(1 - eps), c_0 already halved.
 *
 * Layouts (ABI; "site" = ((t*Lz + z)*Ly + y)*Lx + x, x fastest):
 *   gauge   U[4][site][3][3]           complex (row a, column b)
 *   spinor  psi[nrhs][site][4][3]      complex (spin, colour)
 *   bank    V[n_ev][site][4][3]        complex
 *   complex = interleaved (re, im); complex128 (dtype OV_C128) or complex64 (OV_C64).
 *
 * Memory: every pointer named "device" is a CUDA device pointer owned by the
 * caller; the library never frees it and does not keep it after the call
 * returns (it copies what it needs).  Host pointers are marked "host".  The
 * library owns its internal copies (packed links, eigenvector banks,
 * workspaces) and frees them in ov_destroy.
 *
 * Streams: every call takes a cudaStream_t (0 = legacy default stream) and
 * enqueues its work on it.  apply_* and deflate return once the work is
 * enqueued; solve_overlap, solve_overlap_multimass, ov_eigensolve_Q and
 * ov_estimate_hw_norm read scalars back and so synchronise the stream.  A
 * context is not thread-safe.
 *
 * Errors: every int-returning call returns OV_OK or one of OV_ERR_*;
 * ov_last_error(ctx) gives a message for the last failure on that context.
 * Invalid sizes, pointers or states are rejected on the host before any
 * launch.
 */
#ifndef OVL_H
#define OVL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ov_stream_t; /* = cudaStream_t */
typedef struct ov_ctx ov_ctx;

enum {
    OV_OK = 0,
    OV_ERR_ARG = 1,           /* invalid argument (size, pointer, enum, alias) */
    OV_ERR_CUDA = 2,          /* a CUDA runtime call failed */
    OV_ERR_OOM = 3,           /* device allocation failed */
    OV_ERR_NOT_CONVERGED = 4, /* iteration cap reached; outputs hold the best iterate */
    OV_ERR_BREAKDOWN = 5,     /* CG breakdown: <p, A p> <= 0 */
    OV_ERR_NAN = 6,           /* NaN or Inf met in a reduction */
    OV_ERR_TIMEOUT = 7,       /* a bounded device wait ran out */
    OV_ERR_NO_BANK = 8,       /* no small-space bank registered for a phase */
    OV_ERR_STATE = 9          /* call out of order (e.g. no gauge field set) */
};

enum { OV_BC_PERIODIC = 0, OV_BC_ANTIPERIODIC = 1, OV_BC_DIRICHLET = 2 };

/* Arithmetic of operator applications. F64: FP64 storage and arithmetic.
 * F32: FP32 storage and arithmetic (reductions accumulate in FP64).
 * F16, BF16: the gauge links and the vectors of the Chebyshev recurrence are stored in 16
 * bits (FP16 with one FP32 scale per site, or BF16) and computed in FP32; the small-space
 * projection, the final application of H_w and the caller arrays (complex64) stay FP32.
 * The result carries the 16-bit rounding (relative error ~1e-3 for FP16, ~1e-2 for BF16).
 * As inner_precision of the solver a 16-bit format is allowed only in a context of that
 * precision (the 16-bit links exist there); the solver's FP64 defect correction then
 * removes that rounding over more outer cycles. */
enum { OV_PREC_F64 = 0, OV_PREC_F32 = 1, OV_PREC_F16 = 2, OV_PREC_BF16 = 3 };

/* Element type of caller arrays. */
enum { OV_C128 = 0, OV_C64 = 1 };

typedef struct ov_params {
    int dims[4];          /* Lx, Ly, Lz, Lt; each >= 2 */
    int bc[4];            /* OV_BC_* per direction */
    double m0;            /* Wilson mass in D_w (negative, e.g. -1.5, for overlap) */
    double hw_norm;       /* ||H_w|| used for Q = H_w/hw_norm; <= 0 selects the bound
                             |4 + m0| + 4, which is >= the spectral norm for any links */
    double eps;           /* Q^2 interval [eps, 1] of the polynomial, 0 < eps < 1 */
    int poly_degree;      /* n >= 1 */
    const double* coeffs; /* host [n+1] coefficients of P in the T_k basis, or NULL for the
                             Chebyshev interpolant of x^{-1/2} (see ov_chebyshev_coeffs) */
    int precision;        /* OV_PREC_* of apply_wilson / apply_sign_Hw / apply_overlap */
    int inner_precision;  /* OV_PREC_* of the inner CG in solve_overlap (FP64 outer loop): F64, F32,
                             or the 16-bit format of `precision` (FP32 arithmetic, 16-bit storage
                             of the polynomial loops of the inner CG and of its correction) */
    int max_nrhs;         /* largest nrhs of any call, >= 1 */
    int max_iter;         /* cap on inner CG iterations per solve (<= 0: 100000) */
    double inner_tol;     /* relative tolerance of each inner solve (<= 0: default,
                             1e-6 for F32; for F64 the outer target itself) */
    int launch_shape;     /* Wilson-kernel launch shape of the polynomial loops: 0 = timed per
                             batch size (ov_tune_info); else 1, 2, 4 or 8 systems per thread block,
                             | 16 for the FP32 register budget of 7 blocks per SM instead of 6,
                             | 32 for the kernel that stages x-rows in shared memory (used where
                             the lattice allows it, see ov_tune_info). */
    int poly_kind;        /* coeffs = NULL: 0 = Chebyshev interpolant of x^{-1/2} (ov_chebyshev_coeffs),
                             1 = the polynomial of least relative error max |1 - sqrt(x) P(x)|
                             on [eps, 1] (Remez exchange, ov_minimax_coeffs; its delta follows
                             eq. 2 with A ~ 0.41, where the interpolant's is ~2x larger) */
    int adaptive_order;   /* solve_overlap: 0 = every inner sign application at poly_degree;
                             1 = per outer cycle, the lowest degree (a multiple of 8) whose
                             polynomial (of poly_kind) has delta <= 0.5 m g, g = the cycle's
                             inner tolerance
                             (the true residual keeps poly_degree; needs coeffs = NULL) */
} ov_params;

/* Per-solve statistics, filled on the host when solve_overlap returns. */
typedef struct ov_solve_stats {
    int status;             /* OV_OK / OV_ERR_* of the solve */
    int outer_iters;        /* FP64 true-residual (defect-correction) cycles */
    int inner_iters;        /* inner CG iterations, summed over cycles */
    long long sign_applies; /* sign(H_w) applications, summed over right-hand sides */
    long long dslash_calls; /* Wilson-operator applications, summed over right-hand sides */
    double true_residual;   /* max over rhs of ||b - D(m) x|| / ||b||, FP64 operator (in FP32 and
                               16-bit inner precisions, once every residual is <= min(1e-5, 1e5 tol)
                               the FP64 residual is updated as r - D(m) e with D(m) e from FP32
                               applications to the FP32 hi and lo parts of e, whose rounding,
                               ~1e-6 |r|, is below tol / 10) */
    double seconds;         /* wall time of the solve */
} ov_solve_stats;

/* Timing of the polynomial (Clenshaw) loops, the Wilson-kernel hot loop of every sign
 * application, recorded with CUDA events on the call's stream while profiling is on. */
typedef struct ov_profile {
    double clenshaw_ms;          /* summed event time of the recorded loops */
    long long clenshaw_regions;  /* loops recorded (one per sign application call) */
    long long clenshaw_launches; /* Wilson-kernel launches inside them */
    double clenshaw_bytes;       /* algorithmic bytes of those launches: per launch and site,
                                    the 4 links once (576 B FP64; 192 B FP32, two rows stored)
                                    plus every input, output and epilogue spinor of each system */
    long long kernel_launches;   /* ov_launch_count() at the time of reading */
} ov_profile;

/* ---- context ----------------------------------------------------------- */

/* Create a context for one lattice geometry and operator parameter set.
 * Copies *p (and p->coeffs).  Returns OV_ERR_ARG for invalid parameters. */
int ov_create(const ov_params* p, ov_ctx** out);
int ov_destroy(ov_ctx* ctx);
/* Message of the last failure on ctx (or of the last ov_create failure if ctx is NULL). */
const char* ov_last_error(const ov_ctx* ctx);
/* Human-readable summary of the last eigensolver or solve call on ctx (cycles, residuals). */
const char* ov_last_info(const ov_ctx* ctx);
/* Timings of the Wilson-kernel launch shapes the library tried for each batch size it met
 * (1, 2, 4 or 8 systems per thread block; "d": FP32 registers capped for 7 resident blocks per SM
 * instead of 6; "t": the kernel that stages whole x-rows in shared memory with bulk copies,
 * offered when Lx is a multiple of 4 and rows of Lx sites tile a 32-multiple block); the
 * fastest is used from then on. */
const char* ov_tune_info(const ov_ctx* ctx);
/* Synchronise stream; OV_ERR_TIMEOUT if a bounded wait inside a kernel ran out since the
 * last check (its output is then incomplete), OV_ERR_CUDA if the stream reports an error.
 * solve_overlap and ov_eigensolve_Q make the same check before they return. */
int ov_sync(ov_ctx* ctx, ov_stream_t stream);
/* Exercises the bounded-wait path on stream: one block waits about a millisecond on an mbarrier
 * that nothing completes and records the timeout as a real wait would; the next ov_sync then
 * returns OV_ERR_TIMEOUT and clears it.  For tests of the failure path (no fault, no hang). */
int ov_selftest_bounded_wait(ov_ctx* ctx, ov_stream_t stream);
/* Number of lattice sites. */
long long ov_volume(const ov_ctx* ctx);
/* ||H_w|| in use (after the hw_norm <= 0 default is resolved). */
double ov_hw_norm(const ov_ctx* ctx);
/* delta = max over [eps, 1] of |1 - sqrt(x) P(x)| for the polynomial in use (Sec. 2, eq. 2). */
double ov_poly_delta(const ov_ctx* ctx);
/* delta of the degree-n Chebyshev interpolant of x^{-1/2} on [eps, 1] (as ov_poly_delta, no
 * context needed); -1 for invalid arguments. */
double ov_poly_delta_n(int n, double eps);
/* out[0..n] = coefficients (T_k basis of y = (2x - 1 - eps)/(1 - eps)) of the degree-n
 * polynomial P minimising max over [eps, 1] of |1 - sqrt(x) P(x)| (Sec. 2: the minimax
 * approximation whose error eq. 2 describes), by the Remez exchange algorithm on the host;
 * returns that delta, or -1 for invalid arguments (n in [0, 4000]). */
double ov_minimax_coeffs(int n, double eps, double* out);
/* The degree the adaptive order picks for a polynomial error target: the lowest multiple of 8
 * whose polynomial (of the context's poly_kind) on its interval has delta <= delta_target, else
 * poly_degree. */
int ov_adaptive_degree(ov_ctx* ctx, double delta_target);

/* Turn event timing of the polynomial loops on (on != 0) or off. */
int ov_set_profiling(ov_ctx* ctx, int on);
/* Synchronise the events recorded for loops whose recurrence is stored in the given precision
 * (OV_PREC_*), sum them into *out and reset that record. */
int ov_read_profile(ov_ctx* ctx, int precision, ov_profile* out);
/* Kernels launched by the library so far (all contexts). */
long long ov_launch_count(void);

/* Copy the gauge field (device, [4][site][3][3], dtype OV_C128 or OV_C64) into the
 * context's packed storage (FP64 and FP32 copies).  The caller may free U after
 * the stream reaches this point.  Sec. 2 (D_w), Sec. 4 (links). */
int ov_set_gauge(ov_ctx* ctx, const void* U, int dtype, ov_stream_t stream);

/* Chebyshev coefficients the library uses when coeffs == NULL: the interpolant of
 * x^{-1/2} on [eps, 1] at the n + 1 Chebyshev-Gauss nodes (Sec. 2). out: host [n+1]. */
int ov_chebyshev_coeffs(int n, double eps, double* out);

/* Eigen-decomposition of a small Hermitian matrix on the host (cyclic Jacobi), the
 * routine the library uses for its Rayleigh-Ritz and Gram matrices.  A: host, n x n
 * column-major complex128 (overwritten); w: host [n] eigenvalues ascending; Z: host
 * n x n column-major complex128 eigenvectors (A = Z diag(w) Z^+).  No GPU needed. */
int ov_host_eigh(int n, double* A, double* w, double* Z);

/* ---- operator applications (Sec. 2) ------------------------------------ */

/* out = D_w in (hermitian = 0) or H_w in = gamma5 D_w in (hermitian = 1).
 * in, out: device spinors [nrhs][site][4][3], dtype OV_C128 if ctx precision is F64,
 * OV_C64 otherwise (F16 / BF16: in is rounded to 16 bits, the result read back into FP32);
 * in != out.  phase: host [nrhs] phi_j = q_j E_j (NULL = all zero). */
int apply_wilson(ov_ctx* ctx, const void* in, void* out, int nrhs, const double* phase,
                 int hermitian, ov_stream_t stream);

/* out = sign(H_w) in ~ V diag(sign lambda) V^+ in + Q P(Q^2) (1 - V V^+) in, with the bank
 * registered by deflate() for each phase (an empty small space when none is registered
 * for phase 0; OV_ERR_NO_BANK for a non-zero phase without one).  Costs 2n + 1 Wilson
 * applications.  Layout and dtype as apply_wilson. */
int apply_sign_Hw(ov_ctx* ctx, const void* in, void* out, int nrhs, const double* phase,
                  ov_stream_t stream);

/* out = D(m) in = (1 - m/2)(in + gamma5 sign(H_w) in) + m in  (eq. 1; mass = 0: D_ov). */
int apply_overlap(ov_ctx* ctx, const void* in, void* out, int nrhs, double mass,
                  const double* phase, ov_stream_t stream);

/* Size of the fixed device array apply_wilson_noalloc works in (8 MiB). */
#define OV_NOALLOC_SCRATCH_BYTES (8u << 20)

/* out = D_w in (hermitian = 0) or H_w in (hermitian = 1), like apply_wilson, for callers
 * that cannot allocate device memory: applications whose memory manager owns every device
 * allocation, real-time loops with a fixed memory budget, code that must not make the
 * device synchronisation cudaMalloc and cudaFree can cause.  It needs no context and calls
 * no cudaMalloc, cudaFree or allocating library routine.  The paper has no counterpart to
 * this call.
 * dims: host [4] (Lx, Ly, Lz, Lt), bc: host [4] OV_BC_*, U: device gauge field
 * [4][site][3][3] complex128, in/out: device spinors [nrhs][site][4][3] complex128,
 * in != out, phase: host [nrhs] (NULL = all zero), 1 <= nrhs <= 256; the phases are passed
 * to the GPU by value in a kernel argument, so no host array is read after the call
 * returns.  FP64 arithmetic, the same kernels as apply_wilson.
 * Scratch: one file-scope device array of OV_NOALLOC_SCRATCH_BYTES, held by every GPU
 * that loads the library until the process exits; a call needs
 * 16 (36 V + 24 V nrhs) bytes plus alignment (V = sites), so one rhs fits up to about
 * 8700 sites (8^4 = 4096); larger requests (extents whose product would overflow
 * included) return OV_ERR_ARG with a message in ov_last_error(NULL) before any GPU work.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current): make that first call before any stream capture.  Every call
 * shares the array; each call writes every element it reads, so nothing needs clearing,
 * but calls that overlap on the GPU (other streams or host threads) race on it and must
 * be serialised by the caller. */
int apply_wilson_noalloc(const int dims[4], const int bc[4], double m0, const void* U, const void* in,
                         void* out, int nrhs, const double* phase, int hermitian, ov_stream_t stream);

/* ---- small space (Sec. 2) ---------------------------------------------- */

/* Register the small-space bank for field phase `phase`: V (device, [n_ev][site][4][3],
 * dtype OV_C128 or OV_C64) and lambda (host [n_ev], eigenvalues of Q; only their signs
 * are used, sign(0) = +1).  The library copies V, re-orthonormalises it in FP64
 * (Cholesky QR, twice) and keeps an FP64 and an FP32 copy.  n_ev = 0 clears the bank.
 * Replaces an earlier bank for the same phase. */
int deflate(ov_ctx* ctx, double phase, const void* V, const double* lambda, int n_ev,
            int dtype, ov_stream_t stream);

/* Compute the n_ev eigenpairs of Q (FP64) of smallest |lambda| at field phase `phase` by
 * Chebyshev-filtered subspace iteration with Rayleigh-Ritz, to residual
 * ||Q v - lambda v|| <= tol.  V_out: device [n_ev][site][4][3] complex128 (may be NULL
 * to only register); lambda_out: host [n_ev] (ascending |lambda|).  When a bank is registered for
 * another phase, the iteration starts from that bank's vectors (the nearest phase's; random vectors
 * fill the rest of the block).  If register_bank is
 * non-zero the result is also registered as by deflate().  Returns OV_ERR_NOT_CONVERGED
 * (with the best vectors written) after max_iter filter cycles.  The call's block and filter
 * workspaces (the largest allocations of the library) are freed when it returns, also when it
 * fails part-way (OV_ERR_OOM, OV_ERR_CUDA, OV_ERR_BREAKDOWN). */
int ov_eigensolve_Q(ov_ctx* ctx, double phase, int n_ev, double tol, int max_iter,
                    void* V_out, double* lambda_out, int register_bank, ov_stream_t stream);

/* Working-set budget, in bytes, of ov_eigensolve_Q's chunked passes: its Chebyshev filter runs the
 * recurrence on as many columns of the block at a time as fit three vectors of the iteration's
 * precision per column in `bytes` (at least one column), and its residual pass uses chunks of the
 * same width.  Not counted: the block itself (three sets of m = min(n_ev + max(16, n_ev), 256)
 * vectors, FP32 while the residuals are above FP32 resolution, FP64 after) and the n_ev FP64 result.
 * Results do not depend on it beyond rounding.  Default 16e9 (16 GB); bytes >= 1. */
int ov_set_eigensolver_memory(ov_ctx* ctx, long long bytes);

/* The small-space projection alone (Sec. 2, Fig. 1: the exactly treated low modes), as apply_sign_Hw
 * applies it: with the bank V, s registered for `phase` by deflate(),
 *   xperp = in - V (V^+ in),   ys = V diag(s) (V^+ in)
 * (an empty small space for phase 0 without a bank: xperp = in, ys = 0; OV_ERR_NO_BANK for another
 * phase without one).  in, ys, xperp: device [nrhs][site][4][3], complex128 in an FP64 context,
 * complex64 otherwise (FP32 arithmetic on the FP32 copy of the bank), three different buffers. */
int ov_project_small(ov_ctx* ctx, double phase, const void* in, void* ys, void* xperp, int nrhs,
                     ov_stream_t stream);

/* How FP32 projections of 8 or more vectors run: 0 = on the faster of the two paths, timed once per
 * (bank size, batch size) on the call's own buffers (ov_tune_info lists the times); 1 = CUDA cores;
 * 2 = tensor cores (tcgen05, TF32 with a three-term split for FP32 accuracy; bank size <= 384).
 * FP64 projections and batches below 8 always use the CUDA cores.  Default 0. */
int ov_set_projection(ov_ctx* ctx, int method);

/* ---- propagator solve (Sec. 3.2) --------------------------------------- */

/* Solve D(m) x = b for nrhs right-hand sides to ||b - D(m) x|| / ||b|| <= tol, with D(m)
 * the FP64 operator apply_overlap computes.  b, x: device [nrhs][site][4][3] complex128;
 * x is the initial guess on input and the solution on output; b != x.
 * phase: host [nrhs] (NULL = all zero).  Outer loop: FP64 true residual and FP64 update
 * of x (with an FP32 image of small corrections in the FP64 residual, see ov_solve_stats).  Inner loop: CG in ctx inner_precision on the chiral-sector normal operator
 * P_s [2(1 - m^2/4)(1 + s sign(H_w)) + m^2] P_s (one sign application per iteration and
 * sector), then the correction D(m)^+ y.  stats: host, may be NULL. */
int solve_overlap(ov_ctx* ctx, double mass, const double* phase, const void* b, void* x,
                  int nrhs, double tol, ov_solve_stats* stats, ov_stream_t stream);

/* Change the inner precision of later solves (values as ov_params.inner_precision).  The D_ov
 * deflation spaces serve every inner precision: FP32 and 16-bit inner solves use their FP32
 * vectors and the FP64 low-mode step, FP64 inner solves their FP64 vectors. */
int ov_set_inner_precision(ov_ctx* ctx, int inner_precision);

/* Most masses one solve_overlap_multimass call takes. */
#define OV_MAX_MASSES 32

/* Solve D(m_i) x_i = b for n_mass masses at once (Sec. 3.2, the multi-mass CG), each to
 * ||b - D(m_i) x_i|| / ||b|| <= tol.  The chiral-sector operators of all masses are shifts of
 * one operator, P_s [2(1 - m^2/4)(1 + s sign) + m^2] P_s = (1 - m^2/4)(A0 + m^2/(1 - m^2/4)),
 * A0 = P_s 2 (1 + s sign) P_s; so the first defect-correction cycle, whose residual is b for
 * every mass, runs one multi-shift CG (one sign application per iteration and sector for all
 * masses, the lightest mass's Krylov space, no D_ov deflation) in ctx inner_precision, and
 * x_i = D(m_i)^+ y_i.  Each mass then continues as solve_overlap from x_i (FP64 true residual,
 * deflated inner cycles).  masses: host [n_mass], 1 <= n_mass <= OV_MAX_MASSES, each finite with
 * |m| < 2.  b: device [nrhs][site][4][3] complex128; x: device [n_mass][nrhs][site][4][3]
 * complex128, output only (its contents on input are ignored); b and x must not overlap.
 * phase: host [nrhs] (NULL = all zero).  stats: host [n_mass] or NULL; stats[i] covers mass
 * i's own cycles plus the shared cycle's count in outer_iters and inner_iters, and the shared
 * cycle's sign applications, Wilson applications and time are added to stats[0] only, so that
 * sums over the masses give the call's totals.  Returns the first error other than
 * OV_ERR_NOT_CONVERGED, else OV_ERR_NOT_CONVERGED if any mass missed tol, else OV_OK. */
int solve_overlap_multimass(ov_ctx* ctx, int n_mass, const double* masses, const double* phase,
                            const void* b, void* x, int nrhs, double tol, ov_solve_stats* stats,
                            ov_stream_t stream);

/* Low modes of D_ov for the CG deflation of solve_overlap (Sec. 3.2: the paper deflates its CG
 * with the D_ov eigensystem).  Computes the n_ev lowest eigenpairs of the chiral-sector operator
 * A0 = P_s [2 (1 + s sign(H_w))] P_s = P_s D_ov^+ D_ov P_s, s = chirality (+1 or -1), at the field
 * phase (a small-space bank must be registered for a non-zero phase): thick-restart Lanczos with
 * full reorthogonalisation on FP32 sign applications, bases of krylov vectors (<= 0:
 * max(3 n_ev, n_ev + 32); at least n_ev + 16), restarted from the lowest n_ev + max(8, n_ev/2)
 * Ritz vectors until the n_ev lowest Ritz residual estimates are <= tol (<= 0: 1e-4) or
 * max_restarts restarts ran (< 0: 50), then Rayleigh-Ritz with A0 applied to the Ritz vectors,
 * and D_ov^+ applied to them in FP64 (n_ev FP64 sign applications at the full degree): the
 * solver keeps the space's share of each correction, D(m)^+ W c with c the Galerkin coefficients,
 * in FP64, which removes the FP32 rounding of that large low-mode part.  The space (FP32, n_ev vectors and A0
 * applied to them) is registered for (phase, chirality), replacing an earlier one; from then on
 * the FP32 inner CG of solve_overlap starts each system of that phase and chirality from the
 * Galerkin solution on it and keeps its search directions A-orthogonal to it (deflated CG), for
 * any mass (A(m) = (1 - m^2/4) A0 + m^2).  The Lanczos runs at the lowest degree with
 * delta <= tol / 10; theta_out, res_out: host [n_ev] Ritz values w^+ A0 w of the full-degree
 * operator (FP64) and residual norms |A0 w - theta w|, or NULL.  Synchronises stream. */
int ov_eigensolve_overlap(ov_ctx* ctx, double phase, int chirality, int n_ev, int krylov, double tol,
                          int max_restarts, double* theta_out, double* res_out, ov_stream_t stream);
/* Drop the D_ov deflation spaces of a phase (chirality +1, -1, or 0 for both). */
int ov_clear_overlap_deflation(ov_ctx* ctx, double phase, int chirality);

/* ---- derivatives with respect to the field (Sec. 4) --------------------- */
/* The background field enters as the phase exp(i phi t) on the x links, phi = q E.  The
 * paper takes energy shifts from correlators at several field values; these calls give
 * the derivative of the operator, and with a solve, of the correlator, with respect to
 * phi.  All arrays complex128, FP64 arithmetic, layouts as above. */

/* out = dH_w/dphi in: the x hops with their phase factors differentiated (i t and -i t). */
int ov_apply_dHdphi(ov_ctx* ctx, const void* in, void* out, int nrhs, const double* phase, ov_stream_t stream);

/* out = dD(m)/dphi in = (1 - m/2) gamma5 dF/dphi in, F the implemented sign function
 * (small space registered for each phase plus the polynomial).  dF is the Daleckii-Krein
 * derivative in three blocks: the tangent of the Clenshaw recurrence on the large space
 * (recomputed, nothing stored), (s_i - s_j)/(l_i - l_j) on the small space, and between
 * them (s_i - sign(l))/(l_i - l) (the polynomial error delta below the exact divided
 * difference), applied through per-bank vectors u_i built on first use: the opposite-sign
 * part of the large-space component of dH v_i, times 1/(|t_i| + |Q|) as a Chebyshev
 * polynomial in Q^2 per mode.  Accurate while delta is small against the gap at the cut.
 * Synchronises the stream. */
int ov_apply_dDdphi(ov_ctx* ctx, const void* in, void* out, int nrhs, double mass, const double* phase,
                    ov_stream_t stream);

/* Derivative of the pion correlator with respect to the field E (Sec. 4: the energy shifts come
 * from correlators at several field values; this is their E-derivative through the solve).
 * S: device [nrhs][site][4][3] complex128, the propagator columns S_j = D(m)^-1 b_j at the phase
 * phi = charge E (a small-space bank registered for phi when phi != 0).  u_j = dD(m)/dphi S_j as
 * ov_apply_dDdphi computes it.  dC: host [Lt + 1].
 *  lam == NULL (tangent): dC[t] = dC(t)/dE = 2 Re sum_j <S_j, dS_j/dE>_t with
 *    dS_j/dE = -charge D(m)^-1 u_j, solved here to tol as solve_overlap does (x0 = 0);
 *  lam != NULL (adjoint): dC[t] = -2 charge Re sum_j <lam_j, u_j>_t with lam device [nrhs][site][4][3]
 *    complex128 (for lam = gamma5 D(m)^-1 gamma5 (g o S), the adjoint solution of a loss L with
 *    dL/dC(t) = g(t), the sum over t is dL/dE); tol unused.
 *  dC[Lt] = sum over t of dC[t].  <a, b>_t sums conj(a) b over the sites of time slice t.
 * Synchronises the stream. */
int ov_dcorr_dE(ov_ctx* ctx, double mass, double charge, double E, const void* S, const void* lam, int nrhs,
                double tol, double* dC, ov_stream_t stream);

/* Pion correlator C(t) = sum_rhs sum_{x,y,z} sum_{spin,colour} |S|^2 of propagator columns
 * S (device [nrhs][site][4][3]); C: host [Lt].  Synchronises the stream. */
int ov_correlator(ov_ctx* ctx, const void* S, int nrhs, double* C, ov_stream_t stream);

/* out(x, t) = w(t) G in(x, t), G = gamma5 if gamma5 != 0 else 1; w: host [Lt]. */
int ov_timeslice_scale(ov_ctx* ctx, const void* in, void* out, int nrhs, const double* w, int gamma5,
                       ov_stream_t stream);

/* Inner products <a_j, b_j> (conjugate-linear in a) of device vectors, per right-hand side
 * (per_timeslice = 0; out: host [nrhs][2]) or per right-hand side and timeslice
 * (per_timeslice != 0; out: host [nrhs][Lt][2]).  Deterministic. */
int ov_inner(ov_ctx* ctx, const void* a, const void* b, int nrhs, int per_timeslice, double* out,
             ov_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* OVL_H */
