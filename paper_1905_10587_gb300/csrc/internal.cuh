// Internal declarations shared by the CUDA translation units of libkrr.
// Not part of the public ABI (see include/krr.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/krr.h"

namespace krr {

// ---------------------------------------------------------------- status
struct Status {
    int code = KRR_OK;
    std::string msg;
};

#define KRR_TRY_CUDA(call)                                                            \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return ::krr::fail(ctx, KRR_E_CUDA, std::string(#call) + ": " +           \
                               cudaGetErrorString(e_));                               \
    } while (0)

#define KRR_CHECK_LAUNCH()                                                            \
    do {                                                                              \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess)                                                        \
            return ::krr::fail(ctx, KRR_E_CUDA, std::string("launch: ") +             \
                               cudaGetErrorString(e_));                               \
        ctx->launches++;                                                              \
    } while (0)

#define KRR_RET(expr)                    \
    do {                                 \
        int rc_ = (expr);                \
        if (rc_ != KRR_OK) return rc_;   \
    } while (0)

// Packed point: PS floats per point, PS = round_up(d + 1, 4):
//   [ xh_0 .. xh_{d-1}, a, 0 ... ]   with xh = (x - mu) * sqrt(s), a = -||xh||^2,
//   s = log2(e) / (2 sigma^2), so that K_ij = exp2(a_i + a_j + 2 xh_i . xh_j).
// Kernel dimension used for a data dimension d: exact for d <= 16, else padded with
// zero coordinates to one of the compiled sizes.
inline int kernel_dim(int d) {
    return d <= 16 ? d : d <= 24 ? 24 : d <= 32 ? 32 : d <= 48 ? 48 : 64;
}
inline int packed_stride(int d) { return (kernel_dim(d) + 1 + 3) / 4 * 4; }

// Per-context device scalars of the PCG recurrences (one slot per RHS).
struct CGScalars {
    double rz[KRR_MAX_RHS];
    double rz_new[KRR_MAX_RHS];
    double pq[KRR_MAX_RHS];
    double rr[KRR_MAX_RHS];
    double rr0[KRR_MAX_RHS];
    double a[KRR_MAX_RHS];
    double b[KRR_MAX_RHS];
    int active[KRR_MAX_RHS];
    int all_done;
    int bad;            // a non-finite or non-positive curvature was met
    int tc_err;         // host mirror only: the tensor-core product's error word
};

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Phase timers: CUDA events bracketing a phase on the context's stream.
struct PhaseRec {
    cudaEvent_t start, stop;
    int phase;
};

enum PhaseId { PH_KMVM = 0, PH_SKETCH, PH_OMEGA, PH_QRCP, PH_FGEMM, PH_GRAM, PH_CHOL, PH_APPLY,
               PH_RESID, PH_CGVEC, PH_PREP, PH_COUNT };
extern const char* const kPhaseNames[PH_COUNT];

}  // namespace krr

struct krr_ctx {
    cudaStream_t stream = nullptr;
    krr_opts opts{};
    std::string err;
    int device = 0;
    int num_sms = 0;
    long long launches = 0;
    std::unordered_map<std::string, krr::Buf> bufs;

    // ---- state of the last build
    bool built = false;
    const float* X = nullptr;   // caller's point set (not owned)
    long long n = 0;
    int d = 0, ps = 0;
    double sigma = 0, beta = 0, s = 0;   // s = log2(e)/(2 sigma^2)
    int k = 0, k_eff = 0, l = 0, ldF = 0;
    double build_ms = 0;
    int rrqr_swaps = 0;        // strong RRQR statistics of the last build
    double rrqr_rho = 0;
    // ---- work-split tuning (tune.cu): overrides while krr_autotune times candidates
    bool tuning = false;
    int force_splits = 0;      // > 0: this column-split count
    int force_pv = -1;         // >= 0: P.V form of the tensor-core product (1 tensor cores)
    int last_splits = 0;       // split count of the last product launch
    // device arrays (views into bufs)
    float* P = nullptr;        // n x ps packed points of X
    float* Praw = nullptr;     // n x ps raw coordinates of X (difference form), on demand
    float* PS = nullptr;       // k_eff x ps packed anchors
    float* XS = nullptr;       // k_eff x d raw anchor coordinates
    int* S = nullptr;          // k_eff anchor indices
    float* F = nullptr;        // n x ldF, F = K(X, X_S) L1^{-T}
    double* T2 = nullptr;      // k_eff x k_eff, L2^{-1} (lower)
    double* T2t = nullptr;     // its transpose
    unsigned char* FA = nullptr;   // tensor-core features of X (row role), precision 1
    unsigned char* FB = nullptr;   // tensor-core features of X (column role)
    krr::CGScalars* cg = nullptr;
    krr::CGScalars* cg_host = nullptr;   // pinned mirror

    // ---- phase timers (off unless krr_profile_enable)
    bool prof = false;
    std::vector<krr::PhaseRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
};

namespace krr {

int fail(krr_ctx* ctx, int code, const std::string& msg);

// Brackets a phase with CUDA events when profiling is on (no-op otherwise).
class Phase {
  public:
    Phase(krr_ctx* ctx, int id);
    ~Phase();
  private:
    krr_ctx* ctx_;
    int id_;
    cudaEvent_t start_ = nullptr;
};
// Device buffer named `name`, at least `bytes` long (grown by reallocation).
int buf(krr_ctx* ctx, const char* name, size_t bytes, void** out);
template <class T>
inline int bufT(krr_ctx* ctx, const char* name, size_t count, T** out) {
    return buf(ctx, name, count * sizeof(T), reinterpret_cast<void**>(out));
}

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Float-float accumulation: (hi, lo) += x with Knuth's TwoSum, an error-free transformation
// (hi + x = s + e exactly), so hi + lo carries the running sum to about 2^-44 relative per
// addition.  Six FP32 adds on the FMA pipe, where an FP64 add (after a conversion) takes
// the FP64 unit, which runs at a small fraction of the FP32 rate on this GPU.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float z = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(x, z));
    hi = s;
    lo = __fadd_rn(lo, e);
}
// A running sum of FP32 tile sums: float-float (above), or FP64 where a kernel has no
// registers to spare for the TwoSum temporaries.
struct FoldFF {
    float h = 0.f, l = 0.f;
    __device__ __forceinline__ void add(float x) { ff_add(h, l, x); }
    __device__ __forceinline__ double get() const { return (double)h + (double)l; }
};
struct Fold64 {
    double s = 0.0;
    __device__ __forceinline__ void add(float x) { s += (double)x; }
    __device__ __forceinline__ double get() const { return s; }
};

// 2^t on the FMA pipe, for the accurate product form: t = m + f with m = round(t)
// (rounded by adding and subtracting 1.5 * 2^23), |f| <= 1/2 exact, and
// 2^f = e^(f ln 2) = sum_k (ln 2)^k f^k / k! truncated after k = 7 (the first dropped
// term is below 0.35^8 / 8! = 5.2e-9 relative), in Horner form; the result is scaled by
// 2^m through its exponent bits.  Arguments below -125 give 0 (the products use t <= 0,
// and such terms are below FP32 resolution of any sum they enter).
__device__ __forceinline__ float exp2_poly(float t) {
    const float magic = 12582912.0f;
    const float tm = __fadd_rn(t, magic);
    const float m = __fsub_rn(tm, magic);
    const float f = __fsub_rn(t, m);
    float p = 1.5252733804059838e-05f;          // (ln 2)^7 / 7!
    p = fmaf(p, f, 1.5403530393381606e-04f);    // (ln 2)^6 / 6!
    p = fmaf(p, f, 1.3333558146428441e-03f);    // (ln 2)^5 / 5!
    p = fmaf(p, f, 9.6181291076284770e-03f);    // (ln 2)^4 / 4!
    p = fmaf(p, f, 5.5504108664821576e-02f);    // (ln 2)^3 / 3!
    p = fmaf(p, f, 2.4022650695910071e-01f);    // (ln 2)^2 / 2!
    p = fmaf(p, f, 6.9314718055994531e-01f);    // ln 2
    p = fmaf(p, f, 1.0f);
    const int mi = __float_as_int(tm) - __float_as_int(magic);
    const float r = __int_as_float(__float_as_int(p) + (mi << 23));
    return t < -125.f ? 0.f : r;
}

// The hardware approximation on a reduced argument: 2^t = 2^m * 2^f with m = round(t) and
// f = t - m in [-1/2, 1/2] (exact), the hardware ex2 on f and the power of two through the
// exponent bits; arguments below -125 give 0.
__device__ __forceinline__ float ex2_reduced(float t) {
    const float magic = 12582912.0f;
    const float tm = __fadd_rn(t, magic);
    const float f = __fsub_rn(t, __fsub_rn(tm, magic));
    const int mi = __float_as_int(tm) - __float_as_int(magic);
    const float r = __int_as_float(__float_as_int(ex2f(f)) + (mi << 23));
    return t < -125.f ? 0.f : r;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

inline unsigned ceil_div(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory cap to the device maximum (less the kernel's
// static shared memory), once per kernel and process.  Setting it per launch to that launch's size races when several host threads
// launch the same kernel with different sizes (batched solves).
int allow_max_dynamic_smem(krr_ctx* ctx, const void* fn);

// ---------------------------------------------------------------- launchers
// kmvm.cu
int launch_mean(krr_ctx* ctx, const float* X, long long n, int d, double* mu_dev);
int launch_pack(krr_ctx* ctx, const float* X, long long n, int d, const double* mu_dev, double s,
                float* P);
int launch_gather_pack(krr_ctx* ctx, const float* P, int ps, const float* X, int d, const int* idx,
                       int m, float* Pout, float* Xout);
// Q = K(Pr, Pc) V + beta V (RHS-major, V: nc x nrhs, Q: nr x nrhs).  raw_nsc = 0: Pr, Pc
// are packed [xh, a] points (expansion form); raw_nsc = -s: they are the raw coordinates
// packed with mu = 0 and s = 1 and the exponent is raw_nsc * ||x_i - x_j||^2.
// With Q64 non-null (split mode): V holds nrhs / 2 FP64 columns as hi/lo FP32 column pairs
// (2q, 2q + 1), nr == nc, and Q64 = K (V_hi + V_lo) + beta V64 in FP64 (nrhs / 2 columns).
// In split mode with raw_nsc != 0 (exact differences), raw_nsc + raw_nsc_lo is -s as a
// float pair, used by the compensated kernels.
int launch_kmvm(krr_ctx* ctx, const float* Pr, long long nr, const float* Pc, long long nc, int d,
                float beta, const float* V, int nrhs, float* Q, float raw_nsc = 0.f,
                const double* V64 = nullptr, double* Q64 = nullptr, float raw_nsc_lo = 0.f);
// R = Y - (K + beta I) A in FP64 (Y float, A/R double)
int launch_residual_hp(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                       const float* Y, const double* A, int nrhs, double* R);

int launch_kmvm_reduce(krr_ctx* ctx, const double* part, int splits, int nr, int nrhs, const float* V,
                       int ldv, float beta, float* Q, int ldq);
// Q = (dK/dlog sigma)(Pr, Pc) v, one column
int launch_kmvm_dsigma(krr_ctx* ctx, const float* Pr, long long nr, const float* Pc, long long nc,
                       int d, const float* V, float* Q);

// tune.cu: tuned work splits.  Key of a product configuration; the table entry for it
// (only with opts.autotune and outside tuning); the split count to use (forced, tuned or
// the cost model's `analytic`, clamped to [1, ntiles]; also recorded in ctx->last_splits).
struct TuneEntry {
    int splits, pv;
    double ms;
};
std::string tune_key(int form, int width, int nrhs, long long n);
bool tune_lookup(const krr_ctx* ctx, const std::string& key, TuneEntry* out);
int tuned_splits(krr_ctx* ctx, const std::string& key, int analytic, int ntiles);

// One problem of a (possibly grouped) tensor-core product with P.V on the tensor cores:
// its features, V tiles, per-column scales, partial sums and work split.  Its items are
// item0 .. item0 + items - 1 of the launch, item li = (row block li / splits, column
// split li % splits); tps column tiles per split.
struct PvProb {
    const unsigned char* FA;
    const unsigned char* FB;
    const unsigned char* Vt;
    const double* vsc;
    double* part;
    int nr, nc, Kp, splits, tps, items, item0, pad;
};
// One problem of the grouped V preparation: V (n entries per column, ldv apart) into the
// tiles Vt (ncp columns), scale exponents vexp and factors vsc; its blocks start at blk0.
struct PvPrep {
    const float* V;
    unsigned char* Vt;
    int* vexp;
    double* vsc;
    int ldv, n, ncp, blk0;
};
int pv_tile_bytes(int nrhs);
int launch_pv_prep_grouped(krr_ctx* ctx, const PvPrep* tab_dev, int nprob, int nblk, int nrhs);
int launch_kmvm_tcpv_table(krr_ctx* ctx, const PvProb* table_dev, int nprob, int items, int nrhs,
                           int* err);
// (K + beta I) V for the built point set in product form 0, 1 or 2 (api.cu)
int square_product(krr_ctx* ctx, const float* V, int nrhs, float* Q, int form);
// A replacement whose true residual norm exceeds twice the recursive one restarts the
// recurrence (squared norms compared).
constexpr double kGapRestart2 = 4.0;

// tc_kmvm.cu: BF16x3 tcgen05 product (d <= 16).  Features: role 0 rows, 1 columns.
int tc_feature_kp(int d);
size_t tc_feature_bytes(long long n, int d);
int launch_tc_features(krr_ctx* ctx, const float* P, long long n, int d, int role, unsigned char* out);
int launch_kmvm_tc(krr_ctx* ctx, const unsigned char* FA, long long nr, const unsigned char* FB,
                   long long nc, int d, float beta, const float* V, int nrhs, float* Q,
                   const double* V64 = nullptr, double* Q64 = nullptr);
int launch_sketch_tc(krr_ctx* ctx, const unsigned char* FA, const unsigned char* FB, long long n, int d,
                     const void* Om, int l, int njc_alloc, float* Y, int ldy);
int launch_omega_bf16_tiled(krr_ctx* ctx, unsigned long long seed, int l, long long n, int nab,
                            int njc, void* out);

// residual_ff.cu: same contract in float-float on the FP32 pipe (d <= 16; else FP64)
int launch_residual_ff(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                       const float* Y, const double* A, int nrhs, double* R);

// out = K(Xr, Xc) a (mode 0) or (dK/dlog sigma) a (mode 1) in float-float (d <= 16)
int launch_rect_ff(krr_ctx* ctx, const float* Xr, long long nr, const float* Xc, long long nc, int d,
                   double sigma, const double* a, int mode, double* out);

// sketch.cu
int launch_omega(krr_ctx* ctx, unsigned long long seed, int l, long long n, int ld, float* OmT);
// Algorithm 2: index/sign draws (l x r each) and Y = sum over drawn columns (n x ldy)
int launch_sparse_draw(krr_ctx* ctx, unsigned long long seed, int l, int r, long long n, int* R, float* S);
int launch_sparse_sketch(krr_ctx* ctx, const float* P, long long n, int d, const int* R, const float* S,
                         int l, int r, float* Y, int ldy);
// Out[i*ldo + a] = sum_j K(Pr_i, Pc_j) V[j*ldv + a], a < ncol (FP32 SIMT contraction)
int launch_kgemm(krr_ctx* ctx, const float* Pr, long long nr, const float* Pc, long long nc, int d,
                 const float* V, int ldv, int ncol, float* Out, int ldo);
// G = beta I + F^T F (FP64 k x k, full), F: n x ldF
int launch_gram(krr_ctx* ctx, const float* F, long long n, int k, int ldF, double beta, double* G);

// qrcp.cu, rrqr.cu
int launch_qrcp(krr_ctx* ctx, float* Y, long long n, int l, int ldy, int k, int* piv, float* rdiag);
int launch_strong_rrqr(krr_ctx* ctx, float* Y, long long n, int l, int ldy, int k, double f, int max_swaps,
                       int* piv, float* rdiag, int* swaps_out, double* rho_out);

// dense64.cu
int launch_kss(krr_ctx* ctx, const float* XS, int k, int d, double sigma, double* A);
// In-place lower Cholesky of the k x k row-major A (upper part ignored).  Sets *info
// (host) to 0 or to 1 + the first column whose pivot is <= tau (or not finite); the
// columns before it are final.
int launch_potrf(krr_ctx* ctx, double* A, int k, int* info, double tau = 0.0);
// Solve L X = B in place (B k x k row-major), L lower k x k row-major.
int launch_trsm_lower(krr_ctx* ctx, const double* L, double* B, int k);
int launch_transpose64(krr_ctx* ctx, const double* A, double* At, int k);
int launch_to_float_transposed(krr_ctx* ctx, const double* A, int k, float* Out, int ldo);
int launch_set_identity(krr_ctx* ctx, double* A, int k);
int launch_add_diag(krr_ctx* ctx, double* A, int k, double v);

// cg.cu
int launch_apply_precond(krr_ctx* ctx, const float* R, int nrhs, float* Z, double* rz_part_out);
// b = (float) a; b = (double) a; y += x (tot elements)
int launch_convert(krr_ctx* ctx, const double* a, float* b, long long tot);
int launch_convert_up(krr_ctx* ctx, const float* a, double* b, long long tot);
int launch_accumulate(krr_ctx* ctx, const float* x, double* y, long long tot);
// cg64.cu: FP64 recurrence (split product input, FP64 apply and CG updates)
int launch_split_hilo(krr_ctx* ctx, const double* a, long long n, int nrhs, float* out);
int launch_apply_precond64(krr_ctx* ctx, const double* R, int nrhs, double* Z, double* rz_part);
int cg64_vec_blocks(krr_ctx* ctx);
int launch_cg64_start(krr_ctx* ctx, const double* r, int nrhs, double* rz_part, double* rr_part);
int launch_cg64_alpha(krr_ctx* ctx, const double* p, const double* q, int nrhs, double* part);
int launch_cg64_update_xr(krr_ctx* ctx, double* x, double* r, const double* p, const double* q, int nrhs,
                          double* part);
int launch_cg64_beta_p(krr_ctx* ctx, double* p, const double* z, int nrhs, const double* rz_part);
int launch_add64(krr_ctx* ctx, const double* x, double* y, long long tot);
int launch_dot(krr_ctx* ctx, const float* A, const float* B, long long n, int nrhs, double* out);
int launch_dot64(krr_ctx* ctx, const double* A, const double* B, long long n, int nrhs, double* out);

}  // namespace krr
