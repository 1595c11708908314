/*
 * overlap.h -- C ABI of the GB300 overlap-fermion library (libovgb.so).
 *
 * The library implements, on one NVIDIA GB300 (sm_103a), the hot path of the
 * overlap-operator method of Alexandru, Lujan, Pelissier, Gamari and Lee,
 * "Efficient implementation of the overlap operator on multi-GPUs":
 *
 *   D_w(m)  = (m + 4) - 1/2 sum_{mu=+-1..+-4} T_mu                (Sec. II, Eqs. 1-2)
 *   H_w     = gamma5 D_w(-rho)                                     (Sec. II)
 *   sign(H_w) psi ~ sum_i sign(lam_i)(eta_i^dag psi) eta_i
 *                   + Q P(Q^2) (1 - P_l) psi,   Q = H_w / lambda_max  (Eqs. 5-7)
 *   D(m)    = rho (1 + gamma5 sign(H_w)) + m (1 - D/2)              (Eqs. 3, 8)
 *   deflated CG on D(m)^dag D(m)                                   (Eq. 9, Sec. V)
 *
 * Conventions shared by every call:
 *  - Lattice dims[4] = {Lx, Ly, Lz, Lt}, each even and >= 2.  bc_phase[mu] is
 *    a real phase (+1 periodic, -1 antiperiodic) multiplying every hop that
 *    crosses the boundary in direction mu.
 *  - Canonical spinor layout: complex128 (interleaved re, im doubles)
 *    [nrhs][Lt][Lz][Ly][Lx][spin 4][colour 3], x fastest; right-hand sides
 *    outermost.  Gauge layout: complex128 [Lt][Lz][Ly][Lx][mu 4][3][3]
 *    (row-major colour matrix), mu = 0..3 <-> x, y, z, t.
 *  - Gamma matrices: Euclidean chiral basis, gamma_k = [[0,-i s_k],[i s_k,0]],
 *    gamma_4 = [[0,1],[1,0]], gamma5 = gamma1 gamma2 gamma3 gamma4 =
 *    diag(1,1,-1,-1).
 *  - Buffers passed in may be device memory or host memory (pageable or
 *    pinned); the kind is detected with cudaPointerGetAttributes.  Host
 *    buffers are staged through library-owned device memory and the call
 *    synchronises `stream` before returning.  Device buffers are used in
 *    place and the call is stream-ordered on `stream` (a cudaStream_t passed
 *    as void*; NULL = the legacy default stream).  The caller owns every
 *    buffer it passes; the library owns the packed gauge field, the
 *    eigenpairs, all workspaces and the network weights.
 *  - Every call returns OV_OK (0) or a negative ov_status; on error no
 *    output is guaranteed and ov_last_error() describes the failure.
 *  - Precision (ov_prec): OV_F64 stores and computes in FP64; OV_F32 in FP32;
 *    OV_F16S / OV_BF16S store spinors and links in 16 bits (spinors with one
 *    FP32 scale per site) and compute in FP32; OV_DF64 stores every real as an
 *    unevaluated sum of two FP32 numbers (8 bytes, about 48 significand bits)
 *    and computes with error-free FP32 transformations, an FP64-class result
 *    on the FP32 pipes.  Dot products and norms always accumulate in FP64.
 */
#ifndef OVERLAP_GB300_H
#define OVERLAP_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ov_ctx ov_ctx;     /* opaque, library-owned */
typedef struct ov_field ov_field; /* opaque internal-layout field */

typedef enum {
    OV_OK = 0,
    OV_EINVAL = -1,   /* bad argument: null pointer, bad dims, unknown precision, size out of range */
    OV_ENOMEM = -2,   /* device allocation failed */
    OV_ECUDA = -3,    /* a CUDA call failed (text in ov_last_error) */
    OV_ENOTCONV = -4, /* iteration limit reached before the tolerance */
    OV_ESTALL = -5,   /* residual stopped decreasing */
    OV_ETIMEOUT = -6, /* a bounded device wait gave up */
    OV_ENAN = -7,     /* NaN or Inf met in a result */
    OV_ESTATE = -8    /* call made in the wrong state (e.g. overlap before set_gauge) */
} ov_status;

typedef enum { OV_F64 = 0, OV_F32 = 1, OV_F16S = 2, OV_BF16S = 3, OV_DF64 = 4 } ov_prec;

/* Solver report (one per call; per-rhs values up to 64 right-hand sides). */
typedef struct {
    int iterations;          /* CG iterations (max over right-hand sides) */
    int reliable_updates;    /* FP64 true-residual recomputations */
    int fallback;            /* bit 1: the learned preconditioner was switched off; bit 2: the
                                one-sign chiral form was (two reliable updates in a row that did not
                                halve the true residual), the solve continued with the two-sign operator */
    int nrhs;
    double true_residual[64]; /* ||b - A x|| / ||b|| by the FP64 operator, per rhs; with exact
                                 zero modes among the stored D^dag D modes (massless: x carries no
                                 component along them) it is measured on their orthogonal
                                 complement */
    double seconds;          /* wall time of the solve */
} ov_solve_info;

/* Create a context for one lattice on the current CUDA device.
 * dims[4] = {Lx, Ly, Lz, Lt}: each even and >= 2 (even/odd split, Sec. II
 * lattice of Fig. 1).  bc_phase[4]: +1 or -1 per direction.
 * Returns OV_EINVAL on odd or too small dims, or a null pointer. */
int ov_create(ov_ctx** ctx, const int dims[4], const double bc_phase[4]);
int ov_destroy(ov_ctx* ctx);
/* Text of the last error on this context (never NULL; valid until the next call). */
const char* ov_last_error(const ov_ctx* ctx);

/* Load the gauge field U_mu(n) in SU(3) (Sec. II: gluons as parallel
 * transporters on the links).  U: canonical complex128 gauge layout, host or
 * device.  The library packs it to reconstruct-12 form (rows 0 and 1 kept,
 * row 2 = conj(row0 x row1)) in FP32, FP16 and BF16, where the dslash is
 * bound by bandwidth, and keeps all three rows in FP64 and double-float,
 * where it is bound by arithmetic.  Returns OV_EINVAL
 * if any link deviates from SU(3) by more than 1e-9 (|U U^dag - 1| or the
 * reconstructed third row), since reconstruct-12 would change it. */
int ov_set_gauge(ov_ctx* ctx, const void* U, void* stream);

/* out = D_w(m) in for nrhs canonical spinor fields (Eqs. 1-2). */
int ov_apply_dslash(ov_ctx* ctx, const void* in, void* out, double m, int nrhs, int prec, void* stream);
/* out = H_w in = gamma5 D_w(m) in (Sec. II; hermitian by gamma5-hermiticity). */
int ov_apply_Hw(ov_ctx* ctx, const void* in, void* out, double m, int nrhs, int prec, void* stream);

/* out = D(m)^dag D(m) in, the operator of ov_cg_solve (Eqs. 3, 8; the
 * sign polynomial and H_w eigenpairs as for ov_apply_overlap).  chiral = 1:
 * the one-sign chiral-sector form m^2 + (rho^2 - m^2/4)/rho (1 + chi gamma5)
 * D(0), equal to it up to the polynomial's error on fields with
 * gamma5 in = chi in; every right-hand side must have definite chirality
 * (else OV_EINVAL).  Canonical fields, host or device. */
int ov_apply_normal(ov_ctx* ctx, const void* in, void* out, double mass, int nrhs, int prec, int chiral,
                    void* stream);
/* Fix the sign-function polynomial (Eqs. 4-5, Sec. V): rho (the overlap
 * parameter, H_w = gamma5 D_w(-rho)), P = the degree-`degree` Chebyshev
 * interpolant of x^{-1/2} on [eps, 1], evaluated on Q^2 with
 * Q = H_w / lambda_max by Clenshaw's recurrence.  lambda_max <= 0 asks the
 * library to estimate it (1.01 x the largest |eigenvalue| of H_w from 50
 * Lanczos steps on H_w^2; needs the gauge field).  0 < eps < 1, degree >= 0. */
int ov_set_sign_poly(ov_ctx* ctx, double rho, double eps, int degree, double lambda_max);
/* The rational alternative of Sec. V (Eq. 12): P(Q^2) psi_h = sum_i b_i
 * (Q^2 + c_i)^-1 psi_h with Zolotarev's optimal coefficients for x^{-1/2} on
 * [eps, 1] (npoles fractions, 1..64), the shifted inverses by one multi-shift
 * CG on Q^2 = H_w^2 / lambda_max^2 to the relative residual of option
 * "rational_tol" (1e-12; at least 1e-6 for FP32 and 16-bit fields), in the
 * double-pass form (option "rational_pass" = 2, the default: the scalars of
 * one pass, then a second pass that sums the solution; twice the dslash
 * applications, three vector updates per iteration) or the single-pass form
 * (1: 2 npoles shifted vectors).  The deflation of Eq. 7 and the overlap
 * assembly are those of the polynomial.  Replaces the polynomial until the
 * next ov_set_sign_poly.  Applications with this backend are not captured in
 * CUDA graphs (the iteration tests convergence on the host). */
int ov_set_sign_rational(ov_ctx* ctx, double rho, double eps, int npoles, double lambda_max);
/* The rational backend's coefficients: *npoles, b[npoles], c[npoles] (may be
 * NULL) and delta of Eq. 4; OV_ESTATE when the polynomial is in use. */
int ov_get_sign_rational(const ov_ctx* ctx, int* npoles, double* b, double* c, double* delta);
/* Current polynomial parameters (lambda_max after any estimate). */
int ov_get_sign_poly(const ov_ctx* ctx, double* rho, double* eps, int* degree, double* lambda_max);

/* out = D(m) in = rho D in + m (1 - D/2) in with D = 1 + gamma5 sign(H_w)
 * (Eqs. 3, 8), sign by Eq. 7 with the stored H_w eigenpairs (which = 0).
 * Needs set_gauge and set_sign_poly (OV_ESTATE otherwise).  nrhs <= 16. */
int ov_apply_overlap(ov_ctx* ctx, const void* in, void* out, double mass, int nrhs, int prec, void* stream);

/* Compute and store eigenpairs (Sec. V: eigensolvers for H_w and D).
 * which = 0: the nev eigenpairs of H_w with smallest |lambda| (subspace
 *            iteration with a Chebyshev filter of H_w^2, FP64 Gram-Schmidt,
 *            Rayleigh-Ritz of H_w for the signed eigenvalues); they deflate
 *            the sign (Eq. 7).
 * which = 1: the nev smallest eigenpairs of D(0)^dag D(0) (the same method per
 *            chiral sector); they deflate the CG (Eq. 9).
 * tol: relative eigen-residual target.  Returns OV_ENOTCONV if not reached. */
int ov_deflate(ov_ctx* ctx, int which, int nev, double tol, void* stream);
/* Install eigenpairs computed elsewhere: vals[nev] (signed eigenvalues of H_w
 * for which = 0, eigenvalues of D(0)^dag D(0) for which = 1) and vecs, nev
 * orthonormal canonical complex128 fields (host or device).  nev = 0 clears. */
int ov_set_eigenpairs(ov_ctx* ctx, int which, int nev, const double* vals, const void* vecs, void* stream);
/* Copy out the stored eigenpairs.  *nev receives the count; vals and vecs
 * may be NULL to query it.  vecs: canonical complex128 [nev] fields. */
int ov_get_eigenpairs(ov_ctx* ctx, int which, int* nev, double* vals, void* vecs, void* stream);

/* Solve D(m)^dag D(m) x = b for nrhs right-hand sides to
 * ||b - A x|| / ||b|| <= tol (FP64 operator), deflated CG (Eq. 9) with the
 * stored which = 1 eigenpairs.  inner_prec selects the precision of the
 * inner operator; the residual is recomputed in the accurate precision
 * (option "hi_prec": OV_F64 or OV_DF64) whenever the inner residual has
 * dropped by "reliable_delta" (reliable updates).  precond = 1 uses the learned preconditioner in
 * flexible CG (ov_net_train first), falling back to plain deflated CG when
 * the true residual stalls.  x may hold nothing on entry.  info may be NULL.
 * nrhs <= 16. */
int ov_cg_solve(ov_ctx* ctx, const void* b, void* x, int nrhs, double mass, double tol, int max_iter,
                int precond, int inner_prec, ov_solve_info* info, void* stream);

/* Propagators of several quark masses from one multi-shifted CG (Sec. II,
 * the paragraph after Eq. 8: multi-shifted CG for multiple masses, deflated
 * by the low modes of the massless operator, Eq. 9).  With sign^2 = 1,
 * D(m)^dag D(m) = a_m (D(0)^dag D(0) + m^2 / a_m), a_m = 1 - m^2 / (4 rho^2),
 * so one Krylov recursion on D(0)^dag D(0) (in inner_prec, on the
 * complement of the stored which = 1 eigenvectors, the one-sign chiral form
 * when option "chiral" is set) serves every mass; each mass is then refined
 * by the deflated mixed-precision CG of ov_cg_solve from that start, whose
 * true residuals use the full D(m)^dag D(m) in the "hi_prec" precision.
 *   b: nrhs canonical fields (host or device).  masses[nmass]: 0 <= m < 2 rho,
 *   nmass <= 16, nrhs <= 16.
 *   x: nmass x nrhs canonical fields ([mass][rhs], host or device), receiving
 *   output = 0: x_k = (D(m_k)^dag D(m_k))^-1 b;
 *   output = 1: x_k = D(m_k)^-1 b = D(m_k)^dag (D(m_k)^dag D(m_k))^-1 b;
 *   output = 2: x_k = (1 - D/2) D(m_k)^-1 b, the quark propagator (D = D(0)/rho).
 *   info: NULL or nmass reports; iterations count the shared recursion plus
 *   that mass's refinement; true_residual is that of the normal equations.
 * Returns OV_ENOTCONV (with x and info filled) if a mass misses tol within
 * max_iter iterations of its refinement.  Allocates nmass accurate-precision
 * fields and 2 nmass inner-precision fields for the duration of the call. */
int ov_cg_solve_multimass(ov_ctx* ctx, const void* b, void* x, int nrhs, int nmass, const double* masses, double tol,
                          int max_iter, int inner_prec, int output, ov_solve_info* info, void* stream);

/* ---- learned preconditioner (no counterpart in the paper; used by
 * ov_cg_solve with precond = 1).  M = L2 L1, each layer
 *   y_c(n) = sum_{c'} sum_{p=0..8} W[p][c][c'] (T_p x_{c'})(n),
 * T_0 = 1, T_{1+2mu} x(n) = U_mu(n) x(n+mu), T_{2+2mu} x(n) = U_mu(n-mu)^dag x(n-mu)
 * (the parallel transporters of Eq. 2 without spin projectors), W a complex
 * 4x4 spin matrix; channels 1 -> 16 -> 1.  Weights as 9216 doubles
 * (interleaved re, im): layer 1 W[9][16][1][4][4], then layer 2 W[9][1][16][4][4]. */
/* Record (residual, error) pairs from nsolves deflated mixed-precision CG
 * solves of random sources on this context (mass `mass`), then run `steps`
 * Adam steps (learning rate lr) on sum_k |M r_k - e_k|^2 / |e_k|^2.
 * *final_loss (may be NULL) receives the mean loss per pair. */
int ov_net_train(ov_ctx* ctx, int nsolves, int steps, double lr, double mass, double* final_loss, void* stream);
int ov_net_set_weights(ov_ctx* ctx, const double* w, int n /* 9216 */);
int ov_net_get_weights(ov_ctx* ctx, double* w, int n /* 9216 */);
/* out = M in, or (M + M^dag) in / 2 while the option "net_sym" is set (the
 * default): the operator flexible CG applies.  Canonical fields, host or
 * device, computed in FP32. */
int ov_net_apply(ov_ctx* ctx, const void* in, void* out, int nrhs, void* stream);
/* loss = sum_k |M r_k - e_k|^2 / |e_k|^2 over npairs (<= 16) canonical fields
 * and its gradient (9216 doubles, d/dRe W + i d/dIm W; may be NULL). */
int ov_net_loss_grad(ov_ctx* ctx, const void* r, const void* e, int npairs, double* loss, double* grad,
                     void* stream);
/* Number of training pairs recorded by the last ov_net_train. */
int ov_net_pairs(const ov_ctx* ctx);
/* Loss curve of the last ov_net_train: the mean loss per pair before each
 * Adam step and after the last one (steps + 1 values).  Copies up to cap of
 * them to out and returns how many there are (0 before any training;
 * -OV_EINVAL for a bad argument). */
int ov_net_loss_history(const ov_ctx* ctx, double* out, int cap);

/* ---- internal-layout fields: an even/odd field kept on the device in one
 * storage precision, for chaining operators without repacking. ---- */
int ov_field_create(ov_ctx* ctx, int nrhs, int prec, ov_field** f);
int ov_field_destroy(ov_field* f);
/* canonical (host or device) -> field, and back */
int ov_field_import(ov_ctx* ctx, ov_field* f, const void* canonical, void* stream);
int ov_field_export(ov_ctx* ctx, const ov_field* f, void* canonical, void* stream);
/* out = D_w(m) in (gamma5 = 0) or H_w in (gamma5 = 1), both fields of the
 * same precision and nrhs, in != out.  One kernel launch. */
int ov_dslash_field(ov_ctx* ctx, const ov_field* in, ov_field* out, double m, int gamma5, void* stream);
/* out = D(m) in on internal fields (precision of the fields), in != out. */
int ov_overlap_field(ov_ctx* ctx, const ov_field* in, ov_field* out, double mass, void* stream);
/* Low-mode projection coefficients c[i][r] = v_i^dag psi_r of the stored
 * eigenvectors (which = 0: H_w modes, Eqs. 6-7; which = 1: D^dag D modes,
 * Eq. 9), out: 2 * nev * nrhs doubles (re, im; [i][r]), host or device.
 * engine 0: CUDA cores in the field's precision (FP64 for an FP64 field);
 * engine 1: tensor cores (tcgen05, bf16 operands, FP32 accumulation, FP64
 * sum of the split-K partials), nev <= 128; engine 2: the same with the bf16
 * remainders of both operands added (eta_hi psi_hi + eta_hi psi_lo +
 * eta_lo psi_hi: about 16 significand bits per product, FP32-class), which is
 * what the FP32 and 16-bit overlap use (option "proj_tc").  Returns
 * OV_ETIMEOUT if a bounded wait inside the tensor-core kernel gave up. */
int ov_project_lowmodes(ov_ctx* ctx, int which, const ov_field* psi, int engine, double* out, void* stream);
/* The low-mode update of Eq. 7 alone: out1_r = psi_r - sum_i v_i c[i][r] (the
 * high-mode part psi_h) and, if out2 is not NULL, out2_r = gamma5 sum_i
 * sign(val_i) c[i][r] v_i (gamma5 times the exact low-mode part of the sign),
 * with the stored eigenvectors v_i of `which`.  coef: 2 * nev * nrhs doubles
 * (re, im; [i][r]), host or device.  psi, out1 and out2: distinct fields of
 * one precision and nrhs.  engine 0: CUDA cores in the fields' precision;
 * engine 1: tensor cores (tcgen05, FP32 accumulation; bf16 rows for 16-bit
 * fields, bf16 rows plus their bf16 remainders for FP32 fields; FP32 or
 * 16-bit fields, nev <= 128, nrhs <= 16), which the FP32 and 16-bit overlap
 * use (option "proj_tc").  Synchronises `stream`. */
int ov_lowmode_update(ov_ctx* ctx, int which, const ov_field* psi, const double* coef, int engine, ov_field* out1,
                      ov_field* out2, void* stream);
/* Scalar products x_r^dag y_r of every right-hand side r (Sec. III: the
 * global scalar product), accumulated in FP64 whatever the storage precision
 * and reduced in a fixed order (bitwise reproducible).  out: 2 * nrhs doubles
 * (re, im per rhs), host or device.  x and y: same precision and nrhs. */
int ov_field_dot(ov_ctx* ctx, const ov_field* x, const ov_field* y, double* out, void* stream);
/* The paper has no counterpart: the same scalar products as ov_field_dot for
 * callers that cannot allocate device memory when they call (for example
 * while a CUDA graph is being captured in global mode, or under a memory
 * manager that owns the whole device).  It never allocates: the partial sums
 * live in one fixed 311 KB array of the library's device image, which every
 * GPU that loads the library holds until the process exits.  Limits: up to
 * 16 right-hand sides (the field maximum) and 1216 reduction blocks.  The
 * first call on a device looks the array's device address up
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and every call overwrites it completely, so
 * calls that overlap on the GPU (other streams, other threads) race: order
 * them.  The current device must be the fields' device.  out: 2 * nrhs
 * doubles, host or device; a host out makes the call copy the result and
 * synchronise `stream`, which a stream being captured does not allow, so
 * while capturing pass a device out.  The looked-up address belongs to the
 * device's primary context: after cudaDeviceReset this entry point must not
 * be called again in the process.  Errors are returned as status codes only
 * (ov_last_error is not updated, since setting its text could allocate). */
int ov_field_dot_noalloc(const ov_field* x, const ov_field* y, double* out, void* stream);

/* Device bytes held by the context (gauge, eigenpairs, workspaces). */
long long ov_device_bytes(const ov_ctx* ctx);
/* Number of dslash kernel launches issued through this context so far
 * (instrumentation: an overlap application costs 2n+1, Sec. V). */
long long ov_dslash_count(const ov_ctx* ctx);
/* Capture each overlap / D^dag D application in a CUDA graph on first use
 * and replay it afterwards (enable = 1, the default).  The key is the kind
 * of application, the two buffers, precision, nrhs and mass; the first call
 * for a key runs eagerly and then captures, later calls replay.  A caller on
 * the legacy default stream (NULL, which cannot be captured) gets its graphs
 * on a library-owned stream ordered after and before its own by events; a
 * caller whose stream is being captured gets the plain launches recorded
 * into its own graph.  Graphs are dropped whenever the polynomial, the
 * eigenpairs or a workspace pointer changes. */
int ov_set_graphs(ov_ctx* ctx, int enable);
/* Instrumentation: graphs captured and graph replays launched so far. */
int ov_graph_stats(const ov_ctx* ctx, long long* captured, long long* replayed);
/* Throughput of fused multiply-add on this GPU in GFLOP/s (2 flops per FMA),
 * prec = OV_F64 or OV_F32: a kernel of independent FMA chains, 8 blocks of
 * 256 threads per SM, best of 5 timed launches on `stream` (CUDA events).
 * The paper has no counterpart: it is the measured denominator of the
 * ALU-bound rooflines (the FP64 dslash is bound by the FP64 pipe on GB300,
 * the double-float one by the FP32 pipe).  Allocates and frees one small
 * buffer; synchronises `stream`. */
int ov_measure_fma_peak(int prec, double* gflops, void* stream);
/* Solver tunables:
 *   "reliable_delta" (0.1): ov_cg_solve recomputes the FP64 true residual when
 *                    the inner-precision residual has dropped by this factor;
 *   "filter_hw" (100): Chebyshev filter degree on H_w^2 in ov_deflate(0) (Sec. V: T_100);
 *   "filter_dd" (8):  filter degree on D^dag D in ov_deflate(1) (both rounded down
 *                    to an even degree and capped so that the filter's dynamic
 *                    range stays within the work precision);
 *   "eig_prec" (-1):  operator precision inside ov_deflate: -1 picks the
 *                    "hi_prec" precision when tol < 1e-5 and FP32 otherwise
 *                    (Gram-Schmidt and Rayleigh-Ritz stay FP64), or an ov_prec;
 *                    an FP32 run whose final check fails continues in "hi_prec";
 *   "chiral" (0):     1: ov_cg_solve applies D(m)^dag D(m) on the chiral sector
 *                    of each right-hand side as m^2 + (rho^2 - m^2/4)/rho
 *                    (1 + chi gamma5) D(0), one sign application per iteration
 *                    instead of two (equal up to the polynomial's error; the true
 *                    residuals keep the full operator); every right-hand side
 *                    must satisfy gamma5 b = chi b, else OV_EINVAL (point
 *                    sources do).  Where the sign's delta couples the sectors by
 *                    more than the tolerance allows the solve switches to the
 *                    two-sign operator (ov_solve_info.fallback bit 2); a sign
 *                    with delta well below the tolerance ("sign_delta" of
 *                    ov_get_option) avoids that.  ov_deflate(1) uses the same
 *                    operator per sector;
 *   "hi_prec" (OV_F64): precision of the accurate arithmetic in ov_cg_solve
 *                    (true residuals, solution accumulation) and of the
 *                    automatic ov_deflate operator: OV_F64 or OV_DF64;
 *   "proj_tc" (1):    overlap: the low-mode projection on the tensor cores
 *                    (eta^dag psi for 16-bit storage, the V c update for FP32
 *                    and 16-bit storage; 0: everything on the CUDA cores);
 *   "net_sym" (1):    flexible CG applies the learned preconditioner as
 *                    (M + M^dag) / 2 (Hermitian) instead of M;
 *   "rational_pass" (2), "rational_tol" (1e-12): the rational sign
 *                    (ov_set_sign_rational); "rational_iterations" (read only,
 *                    ov_get_option): CG iterations of its last application;
 *   "clenshaw_f32" (1): 16-bit overlap (OV_F16S, OV_BF16S): the Clenshaw
 *                    recurrence's work vectors are FP32 (the links stay 16-bit,
 *                    the operator's input and output keep their 16-bit storage),
 *                    which keeps the roundings of the n stored recurrence vectors
 *                    out of the result; 0: every vector 16-bit;
 *   "adaptive_delta" (0): adaptive-precision CG (Sec. V, propagator paragraph:
 *                    adaptive CG).  > 0: the inner operator of ov_cg_solve and of
 *                    the shared recursion of ov_cg_solve_multimass uses the
 *                    Chebyshev interpolant of the lowest degree whose delta
 *                    (Eq. 4, on [eps, 1]) is at most this value; every true
 *                    residual and reliable update keeps the full polynomial, so
 *                    the solution still meets tol with it.  0: off;
 *   "wait_polls" (4194304): limit, in polls, of the first mbarrier wait of the
 *                    bulk-copy dslash variants (4, 5) for their copies (also
 *                    bounded by 2 s of the GPU timer).  When it runs out the
 *                    block records the timeout, drains its copies with a wait
 *                    of the full limit, writes nothing, and the call returns
 *                    OV_ETIMEOUT; a smaller value only tests that path. */
int ov_set_option(ov_ctx* ctx, const char* name, double value);
/* Current value of an option of ov_set_option, or one of two derived values:
 * "adaptive_degree", the degree of the inner polynomial that "adaptive_delta"
 * selected (the full degree when it is off); "sign_delta", the accuracy
 * delta = max |1 - sqrt(x) P(x)| over [eps, 1] (Eq. 4) of the installed sign
 * approximation (sampled at 4001 points for the polynomial, Zolotarev's
 * closed form for the rational one; OV_ESTATE before any).  OV_EINVAL for an
 * unknown name. */
int ov_get_option(const ov_ctx* ctx, const char* name, double* value);
/* Launch configuration of the dslash for (prec, nrhs): block = bx sites x by
 * right-hand sides, and a kernel variant: 0 unbounded registers; 1, 2
 * registers capped so that more warps are resident; 3 neighbours staged in
 * shared memory by cp.async; 4, 5 staged by bulk copies (bx = 128, by = 1);
 * 6, 7 two or four right-hand sides per thread sharing each link; 8, 9 the
 * loads of four or eight hops issued before their arithmetic (by = 1); 10, 11
 * two or four right-hand sides per thread as pairs on the packed FP32 pipe
 * (for 6, 7, 10, 11 `by` counts groups of right-hand sides and bx * by <=
 * 128).  Variants 3-11 take FP32 arithmetic (FP32 and 16-bit storage) only.
 * ov_tune_dslash times every candidate on `stream` and keeps the fastest
 * (the autotuner). */
int ov_set_dslash_shape(ov_ctx* ctx, int prec, int nrhs, int bx, int by, int variant);
int ov_tune_dslash(ov_ctx* ctx, int prec, int nrhs, int* bx, int* by, int* variant, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OVERLAP_GB300_H */
