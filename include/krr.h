/*
 * krr.h - C ABI of the GB300 (sm_103a) Gaussian kernel ridge regression solver.
 *
 * The solver computes alpha = (K + beta I)^{-1} y for the Gaussian kernel
 *     K_ij = exp(-||x_i - x_j||^2 / (2 sigma^2))
 * by preconditioned conjugate gradient, following Shabat, Choshen, Ben-Or and
 * Carmel, "Fast and Accurate Gaussian Kernel Ridge Regression Using Matrix
 * Decompositions for Preconditioning" (arXiv 1905.10587):
 *   - the problem is Eq. (1) and Eq. (2) of Section 1;
 *   - the kernel product is the discrete Gauss transform (Section 2.4,
 *     Eq. (6)), here evaluated exactly in tiles without storing K;
 *     the paper's width h equals sqrt(2) * sigma;
 *   - anchors come from Algorithm 1 (Gaussian sketch + pivoted QR) or, with
 *     opts.sparse_r > 0, from Algorithm 2 (sparse sketch + pivoted QR);
 *   - the preconditioner is Algorithm 3 (Nystrom factor + Cholesky of
 *     Eq. (10)), applied by Algorithm 4 (Woodbury, Eq. (7));
 *   - the driver is Algorithm 5 (PCG).
 *
 * Conventions (all entry points):
 *   - Every array argument is a DEVICE pointer owned by the caller, unless
 *     the comment says "host".  The library never frees caller memory.
 *   - Point sets are row-major float32: X[i * d + c], i < n, c < d.
 *   - Multi-column vectors (right-hand sides, solutions) are RHS-major:
 *     column r of an n x nrhs block starts at ptr + r * n.
 *   - A context owns its device workspace (allocated with cudaMalloc, grown on
 *     demand, released by krr_destroy) and issues all work on the stream given
 *     to krr_create.  A context is not thread-safe.
 *   - Return value: KRR_OK or a KRR_E_* code.  Nothing aborts or throws; the
 *     message of the last failure is available from krr_last_error().
 *   - Preconditions are checked on the host before any launch: n >= 1,
 *     1 <= d <= KRR_MAX_DIM, sigma > 0, beta > 0 where the method needs it,
 *     1 <= k <= n, 1 <= nrhs <= KRR_MAX_RHS, non-null pointers.  A bad argument
 *     returns KRR_E_INVAL and launches nothing.
 */
#ifndef KRR_H_
#define KRR_H_

#ifdef __cplusplus
extern "C" {
#endif

#define KRR_OK        0
#define KRR_E_INVAL   1   /* bad argument (host-side check; nothing launched)        */
#define KRR_E_CUDA    2   /* a CUDA runtime call failed                              */
#define KRR_E_NOTSPD  3   /* an FP64 Cholesky met a pivot <= 0                       */
#define KRR_E_NOCONV  4   /* tolerance not reached within the iteration limits      */
#define KRR_E_STATE   5   /* call out of order (e.g. solve before build)             */
#define KRR_E_NOMEM   6   /* workspace allocation failed                             */
#define KRR_E_NONFINITE 7 /* NaN or Inf met in an input or a reduction, or PCG met
                             non-positive curvature it could not recover from         */
#define KRR_E_TIMEOUT 8   /* a bounded device wait ran out (the kernel stopped, freed
                             its resources and returned; the context stays usable)   */

#define KRR_MAX_DIM  64
#define KRR_MAX_RHS  16

typedef struct krr_ctx krr_ctx;

/* Solver options.  krr_default_opts() fills the defaults given here. */
typedef struct krr_opts {
    int    max_iter;      /* PCG iterations in total (default 5000)                      */
    int    refine_max;    /* true-residual replacements allowed (default 40)             */
    int    oversample;    /* l = k + oversample random projections (default 5, Sec. 5.1) */
    int    check_every;   /* iterations between host convergence reads (default 1)      */
    double inner_tol;     /* reliable-update factor: the FP32 recursive residual is
                             replaced by the float-float true residual once it has
                             dropped by this factor (default 1e-2)                        */
    double anchor_rtol;   /* pivots with |R_jj| < anchor_rtol |R_11| are dropped (1e-5)  */
    int    precision;     /* kernel product of the PCG iterations: 0 = FP32 FFMA tiles
                             (default); 1 = tcgen05 tensor cores, exponent from a BF16x3
                             split GEMM (d <= 16; larger d uses the FP32 tiles);
                             2 = FP32 FFMA tiles on exact coordinate differences
                             (slower, no cancellation in the exponent)                   */
    int    residual;      /* refinement residual: 0 float-float on the FP32 pipe
                             (default), 1 FP64 pipe                                      */
    double pivot_tol;     /* the anchor set ends at the first anchor whose Cholesky pivot
                             in K_SS (its variance given the earlier anchors; K_SS has a
                             unit diagonal) is <= pivot_tol (default 1e-6)              */
    int    escalate;      /* 1 (default): when PCG meets non-positive curvature, or the
                             true residual stops falling, on precision 0 or 1, switch the
                             product to precision 2 and restart from the current alpha  */
    int    sparse_r;      /* 0 (default): Gaussian sketch (Algorithm 1); r > 0: sparse
                             sketch of Algorithm 2 with r nonzeros per projection (<= 1024) */
    int    wait_limit_log2;   /* bounded device waits of the tensor-core product give up
                                 after 2^wait_limit_log2 cycles and report KRR_E_TIMEOUT;
                                 0 (default) = 2^32 cycles (about 2 s); 10..40 allowed.
                                 Small values are for failure-detection tests            */
    int    test_stall_copies; /* failure-detection tests only: 1 makes the tensor-core
                                 product issue no copies, so its bounded waits run out
                                 (nothing is in flight) and the call returns
                                 KRR_E_TIMEOUT; 0 (default) in all other use             */
    int    no_precond;    /* 1: plain CG without the preconditioner (z = r), for the
                             condition-number experiment of Section 5.1; 0 (default)   */
    int    recurrence;    /* PCG vectors: 0 (default) = FP32 x, r, p, z (fastest; enough
                             when lambda_max(K) / beta is far below 1 / eps32); 1 = FP64
                             x, r, p, z, the product fed p as FP32 hi + lo parts with FP64
                             sums out (in precision 2 the accurate split product), and the
                             apply exact for the stored F; 2 = FP32 until the solve
                             escalates to precision 2, then FP64.  With FP64 vectors the
                             recurrence restarts after every true-residual replacement  */
    int    strong_swaps;  /* with strong_f > 1: most swaps the strong RRQR may make (0 = 64) */
    int    ex2_correct;   /* 1 (default): scale the kernel sums of the tensor-core product
                             (precision 1) by 1 + 0.83 * 2^-24, the mean low bias of the
                             hardware 2^t approximation for t < -1 (see krr_exp2_probe);
                             0: uncorrected                                              */
    int    tc_pv;         /* 1 (default): in the tensor-core product, blocks of 8 or 16
                             right-hand sides contract P V on the tensor cores too (P and
                             V as FP16 hi + lo pairs, about 2^-22 relative per entry;
                             FP32 V and Q only); 2: every block, 1 to 16 right-hand
                             sides; 0: P V as FP32 FMAs                                 */
    int    autotune;      /* 1: the kernel products take their column-split count (and
                             the tensor-core product its P.V form) from the tuning table
                             where it has an entry for the configuration (krr_autotune,
                             krr_tune_load); 0 (default): from the cost model           */
    int    tc_vfold;      /* 1 (default): the tensor-core product with one right-hand side
                             folds v into the exponent (2^(t + log2|v_j|), columns taken
                             in two sign groups), so its epilogue loads no V; 0: FFMA    */
    int    reserved[1];
    double strong_f;      /* 0 (default): the build selects anchors by pivoted QR (Algorithm 1
                             step 3 as Section 3 remarks); f > 1: by strong RRQR with bound
                             f (Gu-Eisenstat; the factorization Eq. (4) assumes), see
                             krr_strong_rrqr                                             */
} krr_opts;

/* Per-solve report (host struct). */
typedef struct krr_solve_info {
    int    status;                        /* KRR_OK or KRR_E_NOCONV                   */
    int    iters;                         /* PCG iterations summed over sweeps        */
    int    sweeps;                        /* true-residual replacements made          */
    int    k_eff;                         /* anchors kept by the build                */
    double rel_residual[KRR_MAX_RHS];     /* ||y - (K+beta I) alpha|| / ||y||, FP64   */
    double build_ms;                      /* time of the last krr_build_precond       */
    double solve_ms;                      /* wall time of this solve (host clock)     */
    int    mvm_count;                     /* kernel products (K+beta I)V issued       */
    int    sweep_iters[8];                /* PCG iterations before each replacement   */
    double sweep_residual[8];             /* worst column's true residual at the start
                                             and after each replacement                */
    int    product_form;                  /* precision of the product at the end (0-2)  */
    int    restarts;                      /* times the CG direction was reset: at an
                                             escalation, after a stall, when a true
                                             residual came out well above the recursive
                                             one, or at every replacement with FP64
                                             vectors                                   */
    int    recurrence64;                  /* 1 if the solve ended with FP64 vectors     */
    int    lanczos_steps;                 /* CG steps behind cond_estimate              */
    int    reserved[2];
    double cond_estimate;                 /* condition number of the system PCG saw
                                             (with the preconditioner: of
                                             (K~ + beta I)^{-1} (K + beta I), Theorem 4.5;
                                             with opts.no_precond: of K + beta I), from
                                             the extreme eigenvalues of the Lanczos
                                             tridiagonal that column 0's CG coefficients
                                             define over its first uninterrupted cycle
                                             (a lower bound that tightens with the steps) */
} krr_solve_info;

/* Fill *opts with the defaults.  Returns KRR_E_INVAL if opts is NULL. */
int krr_default_opts(krr_opts* opts);

/* Create a context on the current CUDA device.  opts may be NULL (defaults);
 * stream is a cudaStream_t (NULL = legacy default stream). */
int krr_create(krr_ctx** ctx, const krr_opts* opts, void* stream);

/* Release the context and all workspace it owns.  NULL is allowed. */
void krr_destroy(krr_ctx* ctx);

/* Message of the last failure on this context ("" if none); host string owned by ctx. */
const char* krr_last_error(const krr_ctx* ctx);

/* Number of kernel launches this context has issued so far (host counter). */
long long krr_launch_count(const krr_ctx* ctx);

/* Phase timers.  krr_profile_enable(ctx, 1) clears the records and brackets each
 * phase of later calls with CUDA events on the context's stream; krr_profile_read
 * sums the recorded durations of one phase ("kmvm", "sketch", "omega", "qrcp",
 * "fgemm", "gram", "chol", "apply", "resid_hp", "cgvec", "prep") and counts its
 * occurrences (host outputs; synchronises on the recorded events). */
int krr_profile_enable(krr_ctx* ctx, int on);
int krr_profile_read(krr_ctx* ctx, const char* phase, double* total_ms, long long* count);

/* Known-answer test of the tensor-core path's shared-memory and instruction
 * descriptors: 128 x 32 BF16 tcgen05.mma products of small integers, compared on
 * the host.  variant 0: one K = 16 step in the unswizzled core-matrix layout (the
 * sketch's P and Omega operands); variant 1 swaps its two strides (must fail);
 * variant 2: K = 64 in four steps in the 128-byte swizzled layout of the point
 * features; variant 3 reads that data through an unswizzled descriptor (must fail);
 * variant 4: FP16 with K = 64, A held in tensor memory (two K-neighbours per 32-bit
 * column, the even one in the low half) and B in the swizzled layout, the form of
 * the multi-RHS product's P.V step.
 * Writes the number of wrong entries and the largest error (host outputs).  No
 * counterpart in the paper: a check of the hardware encoding the tensor-core
 * product relies on. */
int krr_tc_selftest(int variant, int* mismatches, float* max_err, void* stream);

/* Whole-GPU issue-rate probe used for roofline denominators: kind 0 = FP32 FFMA,
 * 1 = MUFU ex2, 2 = FP64 DFMA.  Writes operations per second to *ops_per_s (host).
 * Runs on the current device and the given stream (NULL = default stream). */
int krr_peak_probe(int kind, double* ops_per_s, void* stream);

/* Accuracy probe of the two 2^t evaluations the kernel products use: out[i] = 2^t[i]
 * (t, out: n device floats) by the hardware approximation (method 0, ex2.approx.ftz),
 * by the FMA-pipe polynomial of the accurate split product (method 1: round-to-integer
 * reduction and a degree-7 Taylor polynomial of e^(f ln 2), |f| <= 1/2), or by the
 * hardware approximation on the reduced argument (method 2: 2^round(t) * ex2(t - round(t))).
 * No counterpart in the paper: the tests compare them against the exact 2^t. */
int krr_exp2_probe(const float* t, long long n, int method, float* out, void* stream);

/* ---------------------------------------------------------------------------
 * Kernel products (Section 2.4, Eq. (6); Definition 2.1).
 * Q = K(Xr, Xc) V + beta * V[0:nr]   (Q: nr x nrhs, V: nc x nrhs, RHS-major).
 * K(Xr, Xc)_ij = exp(-||xr_i - xc_j||^2 / (2 sigma^2)), evaluated in FP32 tiles
 * from the expansion ||x||^2 + ||y||^2 - 2 x.y after centring both sets on the
 * mean of Xc; K is never stored.  Each thread sums one 128-column tile in
 * FP32 and folds the tile sums in FP64 (smooth kernels with mixed-sign V cancel
 * heavily, and an FP32 running sum over 10^5 columns loses about beta of the
 * result).  With opts.precision = 2 the exponent is instead -||xr_i - xc_j||^2
 * / (2 sigma^2) from the differences of the given coordinates (no centring), and
 * with opts.precision = 1 (d <= 16) it is the tensor-core BF16x3 split GEMM.
 * beta must be 0 unless nr == nc (square
 * product with the ridge term).  Xr may equal Xc.
 * ------------------------------------------------------------------------- */
int krr_kmvm(krr_ctx* ctx, const float* Xr, long long nr, const float* Xc, long long nc,
             int d, double sigma, double beta, const float* V, int nrhs, float* Q);

/* High-precision residual R = Y - (K(X, X) + beta I) A with FP64 alpha A and FP64
 * output R (n x nrhs each, RHS-major); K entries and sums carried in FP64 from
 * exact differences of the float32 coordinates.  Used for the refinement step. */
int krr_residual_hp(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                    const float* Y, const double* A, int nrhs, double* R);

/* The same residual with every quantity held as a float-float pair on the FP32 pipe
 * (exact products and sums by error-free transformations, 2^t from a 2^(j/64)
 * table and a degree-5 series); kernel values to a few 1e-12 relative.  For d > 16
 * it falls back to the FP64 evaluation above. */
int krr_residual_ff(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                    const float* Y, const double* A, int nrhs, double* R);

/* ---------------------------------------------------------------------------
 * Algorithm 1 pieces.
 * ------------------------------------------------------------------------- */
/* The Gaussian test matrix of Algorithm 1 step 1, written transposed: OmT[j*l + a]
 * = omega_{a,j}, j < n, a < l.  Entry (a, j) is Box-Muller on Philox4x32-10
 * (Salmon et al., SC'11) with counter (j mod 2^32, j div 2^32, a div 2, 0) and key
 * (seed mod 2^32, seed div 2^32): u1 = ((r0 >> 8) + 1) 2^-24, u2 = (r1 >> 8) 2^-24,
 * omega_{2c} = sqrt(-2 ln u1) cos(2 pi u2), omega_{2c+1} = sqrt(-2 ln u1) sin(2 pi u2). */
int krr_omega(krr_ctx* ctx, unsigned long long seed, int l, long long n, float* OmT);

/* Sketch Y = K(X, X) Omega^T of Algorithm 1 step 2: Y is n x l row-major
 * (Y[i*l + a]).  Omega is generated as krr_omega describes.  With opts.precision = 1
 * (and d <= 16) the product runs on tensor cores with Omega and the kernel values
 * rounded to BF16 (about 4e-3 relative error, which only steers the anchor choice);
 * otherwise in FP32 tiles. */
int krr_sketch(krr_ctx* ctx, const float* X, long long n, int d, double sigma, int l,
               unsigned long long seed, float* Y);

/* Algorithm 2, steps 3-4 (Section 3, SparseAnchorSelection): for each of the l
 * projections, r row indices in [0, n) and r Rademacher signs.  Entry (i, m) comes from
 * Philox4x32-10 with counter (i, m, 0x53505253, 0) and key (seed lo, seed hi): the index
 * is the high word of r0 * n, the sign is -1 when the top bit of r1 is set.  Indices are
 * drawn independently (with replacement).  R (int) and S (float): l x r, row-major, device. */
int krr_sparse_draw(krr_ctx* ctx, unsigned long long seed, int l, int r, long long n, int* R, float* S);

/* Algorithm 2, steps 5-6: Y(:, i) = K(X, X_R) v for the draws of krr_sparse_draw, FP32
 * tiles from the packed points (as krr_sketch).  Y: n x l row-major (Y[j * l + i]),
 * device.  The context's build state is reset.  Fails with KRR_E_INVAL when r
 * points of dimension d do not fit 40 KB of shared memory. */
int krr_sparse_sketch(krr_ctx* ctx, const float* X, long long n, int d, double sigma, int l, int r,
                      unsigned long long seed, float* Y);

/* Column-pivoted QR pivot selection of Algorithm 1 steps 3-4 on Y^T (Y is n x l
 * row-major, so the columns of Y^T are the rows of Y): returns the first k pivots
 * (device int32 piv[k]) and |R_jj| (device float rdiag[k]).  Rule: the largest
 * remaining residual norm, lowest index on ties.  Y is overwritten (residuals). */
int krr_qrcp(krr_ctx* ctx, float* Y, long long n, int l, int k, int* piv, float* rdiag);

/* Strong rank-revealing QR (Gu and Eisenstat) on Y^T: the factorization behind the
 * interpolative-decomposition bound of Section 2.3 (Eq. (4)).  Starts from krr_qrcp's pivots,
 * keeps the first k rows of R, and while some pair (pivot position i, other column j) has
 * (R11^{-1} R12)_ij^2 + gamma_j^2 ||row i of R11^{-1}||^2 > f^2 (gamma_j the residual norm of
 * column j) swaps them and refactors, at most max_swaps times.  Y (n x l row-major, device)
 * is overwritten; piv (device int32[k]) and rdiag (device float[k]) as for krr_qrcp; swaps
 * and rho_max (host; may be NULL) receive the swaps made and the final max sqrt(rho), which
 * is <= f (within FP32 rounding) unless max_swaps ran out.  Needs 1 <= k <= l, k < n, f > 1. */
int krr_strong_rrqr(krr_ctx* ctx, float* Y, long long n, int l, int k, double f, int max_swaps,
                    int* piv, float* rdiag, int* swaps, double* rho_max);

/* Anchor selection statistics of the last build: the swaps its strong RRQR made and its final
 * max sqrt(rho) (both 0 when the build used plain pivoted QR).  Host outputs. */
int krr_anchor_stats(krr_ctx* ctx, int* rrqr_swaps, double* rrqr_rho);

/* ---------------------------------------------------------------------------
 * Algorithms 3-5.
 * ------------------------------------------------------------------------- */
/* Build the preconditioner (Algorithm 5 steps 1-2: Algorithm 1, or Algorithm 2 when
 * opts.sparse_r > 0, then Algorithm 3) for (X, sigma, beta) with k anchors and
 * l = k + opts.oversample projections.
 * X must stay valid and unchanged until the last krr_solve/krr_predict on it. */
int krr_build_precond(krr_ctx* ctx, const float* X, long long n, int d, double sigma,
                      double beta, int k, unsigned long long seed);

/* Build with caller-given anchors S (device int32[k], indices into X). */
int krr_build_precond_anchors(krr_ctx* ctx, const float* X, long long n, int d, double sigma,
                              double beta, const int* S, int k);

/* Anchors kept by the last build: writes k_eff (host) and S (device int32[k_eff], may be NULL). */
int krr_get_anchors(krr_ctx* ctx, int* S, int* k_eff);

/* Out = (K~ + beta I)^{-1} In (Algorithm 4; Eq. (7)), In/Out n x nrhs FP32. */
int krr_precond_apply(krr_ctx* ctx, const float* In, int nrhs, float* Out);

/* Solve (K + beta I) alpha = Y (Algorithm 5 step 3) for the built X to
 * ||Y - (K + beta I) alpha|| / ||Y|| <= tol per column, measured with the
 * float-float (or FP64, opts.residual = 1) residual.  The PCG recurrence runs in
 * FP32 with reliable updates: its recursive residual is replaced by the true one
 * (and its iterate folded into the FP64 alpha) each time it drops by
 * opts.inner_tol.  X must be the pointer given to the build.  alpha: n x nrhs FP64.
 * info (host) may be NULL.  Returns KRR_E_NOCONV if the limits are hit first, or
 * KRR_E_NONFINITE if PCG breaks down (non-positive curvature or a non-finite value)
 * in a form it cannot escalate from; in both cases alpha holds, per column, the
 * iterate with the smallest verified true residual seen (info->rel_residual reports
 * that residual).  When PCG meets non-positive curvature in product form 0 or 1 with
 * opts.escalate set, the unverified correction since the last true residual is
 * discarded and the solve goes on in form 2 from the best verified alpha. */
int krr_solve(krr_ctx* ctx, const float* X, const float* Y, int nrhs, double tol,
              double* alpha, krr_solve_info* info);

/* ---------------------------------------------------------------------------
 * Allocation-free kernel product.  The paper has no counterpart: this entry
 * exists for callers that may not allocate device memory, such as an
 * application that owns all GPU memory through its own pool, or code running
 * where a cudaMalloc is not allowed.  It computes the same product as krr_kmvm
 * (no context needed), taking all temporaries from one fixed device array of
 * KRR_NOALLOC_SCRATCH_BYTES that every GPU which runs this call keeps until the
 * process exits.  The array's device address belongs to the CUDA context it was
 * looked up in: the first call on a device (and the first after that device's
 * context is replaced, e.g. by cudaDeviceReset) looks it up with that context
 * current, and under lazy module loading that lookup is what commits the array's
 * memory.  So make the first call before memory runs short and before any stream
 * capture; if the array cannot be committed then, KRR_E_NOMEM is returned.  Calls
 * share the array: calls whose work overlaps on the GPU (other streams, other
 * threads) race on it and must be serialised by the caller.  No temporary needs
 * to start at zero.  If a size needs more scratch than the array holds, nothing
 * is launched, KRR_E_NOMEM is returned and *scratch_needed (if non-NULL) says how
 * many bytes it would take; bad arguments return KRR_E_INVAL.  All pointers are
 * device pointers as for krr_kmvm; stream is a cudaStream_t (NULL = default).
 * ------------------------------------------------------------------------- */
#define KRR_NOALLOC_SCRATCH_BYTES (64u << 20)
int krr_kmvm_noalloc(const float* Xr, long long nr, const float* Xc, long long nc, int d,
                     double sigma, double beta, const float* V, int nrhs, float* Q, void* stream,
                     unsigned long long* scratch_needed);

/* f = K(Xtest, X) alpha (Eq. (1)); Xtest m x d, alpha n x nrhs FP32, f m x nrhs.
 * FP32 tiles, in the exact-difference form when opts.precision = 2. */
int krr_predict(krr_ctx* ctx, const float* Xtest, long long m, const float* alpha, int nrhs,
                float* f);

/* Derivative kernel product Q = (dK(Xr, Xc)/dlog sigma) V for one column: entries
 * K_ij ||xr_i - xc_j||^2 / sigma^2, evaluated in FP32 tiles like krr_kmvm.  V (nc) and
 * Q (nr) are FP32 device vectors.  Used by krr_grad. */
int krr_kmvm_dsigma(krr_ctx* ctx, const float* Xr, long long nr, const float* Xc, long long nc, int d,
                    double sigma, const float* V, float* Q);

/* Gradient of the held-out mean squared error
 *     L = ||K(Xval, X) alpha - yval||^2 / m,   alpha = (K + beta I)^{-1} y,
 * with respect to log sigma, log beta and y, for the built (X, sigma, beta).  The
 * paper has no gradient; this is the adjoint of its solve: with g = 2 (f - yval)/m
 * and lambda = (K + beta I)^{-1} K(X, Xval) g (a second preconditioned solve),
 *     dL/dy = lambda,   dL/dlog beta = -beta lambda . alpha,
 *     dL/dlog sigma = g . (dK(Xval, X)/dlog sigma) alpha - lambda . (dK/dlog sigma) alpha,
 * using dK_ij/dlog sigma = K_ij ||x_i - x_j||^2 / sigma^2 (a derivative kernel product).
 * The four kernel products (f, the adjoint right-hand side and both derivative
 * products) are evaluated in float-float, since the sigma term is a difference of two
 * products that cancel.  Needs d <= 16.
 * Y (n) and yval (m) are FP32 device vectors, Xval m x d; both solves run to tol.
 * loss, dlogsigma, dlogbeta are host outputs; dy is an n-element FP64 device vector. */
int krr_grad(krr_ctx* ctx, const float* Y, const float* Xval, long long m, const float* yval,
             double tol, double* loss, double* dlogsigma, double* dlogbeta, double* dy);

/* ---------------------------------------------------------------------------
 * Batched solves (many independent problems of uneven size; the paper solves one
 * problem at a time).  Each problem is built (Algorithms 1 and 3, anchor seed
 * seed + index) and solved (Algorithm 5) to tol with nrhs right-hand sides, as
 * krr_build_precond + krr_solve would.  W worker threads (workers <= 0: 8), each
 * with its own CUDA stream and context, take problems largest n^2 first, so several
 * problems' kernels overlap on the GPU.  All problem arrays are device pointers;
 * probs, infos and statuses are host arrays of nprob entries (infos, statuses may be
 * NULL).  The call returns when every problem is done: KRR_OK, or the first
 * non-OK status of a problem (KRR_E_NOCONV when some problem stopped early).
 * ------------------------------------------------------------------------- */
typedef struct krr_problem {
    const float* X;     /* n x d, row-major                       */
    long long n;
    int d;
    const float* Y;     /* n x nrhs, RHS-major                    */
    double sigma, beta;
    int k;
    double* alpha;      /* n x nrhs FP64 output, RHS-major        */
} krr_problem;

int krr_batch_solve(const krr_problem* probs, int nprob, int nrhs, double tol, unsigned long long seed,
                    const krr_opts* opts, int workers, krr_solve_info* infos, int* statuses);

/* The same contract, solved in lockstep: after the builds (W threads as above), the PCG
 * recurrences of all problems advance together on one stream, and each step of an
 * iteration is one launch over the work items of every active problem (the tensor-core
 * product with P.V on the tensor cores for problems built with precision 1 and d <= 16,
 * the CG vector updates, the Woodbury apply, the per-problem CG scalars).  Each problem
 * keeps its own scalars, column activity and true-residual replacements; the host reads
 * all problems' recursive residuals once per iteration.  A problem whose recurrence
 * breaks down, stalls, shows repeated residual gaps or runs out of iterations is then
 * solved again from zero by krr_solve on its own context (which escalates the product
 * form), so every problem ends as the one-by-one path would end it; its info counts the
 * grouped iterations too.  solve_ms is the wall time of the grouped phase (shared).
 * Device memory: the five concatenated FP32 vectors (sum of n x nrhs each) plus per
 * problem the Woodbury partials and the product's split partials.  Problems need
 * n <= 2^30.  Returns as krr_batch_solve; KRR_E_TIMEOUT when a bounded wait of the
 * grouped product ran out (every problem is then finished by its own solve). */
int krr_batch_solve_grouped(const krr_problem* probs, int nprob, int nrhs, double tol,
                            unsigned long long seed, const krr_opts* opts, int workers,
                            krr_solve_info* infos, int* statuses);

/* ---------------------------------------------------------------------------
 * Work-split tuning (no counterpart in the paper).  The kernel products split the
 * columns of K into ranges handled by separate work items; the count comes from a
 * cost model unless a tuning-table entry exists for the configuration and
 * opts.autotune = 1.  Keys read "form=F w=W r=R lg=L": product form F (0 FP32
 * expansion, 1 tensor cores, 2 exact differences), feature width W (tensor-core K,
 * else the kernel dimension), R right-hand sides per launch, L = floor(log2 n).
 * Entries hold the split count, the P.V form (1 = on tensor cores) and the time.
 * The table is process-wide and guarded by a lock.
 *
 * krr_autotune: for the built problem of ctx, times the square product (the form of
 * opts.precision) with nrhs in {1, 2, 4, 8, 16} right-hand sides for the cost model's
 * choice and split counts 1 .. 64, and with 64-wide tensor-core features for both P.V
 * forms; each candidate is run once to warm up, then reps times between CUDA events.
 * Stores the fastest under its key and writes it to the host outputs (each may be NULL).
 * KRR_E_STATE before a build, KRR_E_INVAL for a bad nrhs or reps outside 1 .. 100.
 * krr_tune_save / krr_tune_load write and read the table as JSON (load adds entries;
 * KRR_E_INVAL on a missing file or an entry that does not parse, with nothing added).
 * krr_tune_get reads one entry (KRR_E_STATE when absent); krr_tune_set writes one;
 * krr_tune_clear empties the table.
 * ------------------------------------------------------------------------- */
int krr_autotune(krr_ctx* ctx, int nrhs, int reps, int* splits, int* pv, double* ms);
int krr_tune_save(const char* path);
int krr_tune_load(const char* path);
int krr_tune_get(const char* key, int* splits, int* pv, double* ms);
int krr_tune_set(const char* key, int splits, int pv, double ms);
int krr_tune_clear(void);

#ifdef __cplusplus
}
#endif
#endif /* KRR_H_ */
