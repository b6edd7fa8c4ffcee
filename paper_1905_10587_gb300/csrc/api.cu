// extern "C" entry points of libkrr (declared in include/krr.h) and the host-side
// drivers: the preconditioner build (Algorithm 5 steps 1-2 = Algorithms 1 and 3)
// and the refined PCG solve (Algorithm 5 step 3 inside FP64 iterative refinement).
#include "internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

namespace krr {

int fail(krr_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int allow_max_dynamic_smem(krr_ctx* ctx, const void* fn) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(fn)) return KRR_OK;
    int dev = 0, optin = 0;
    KRR_TRY_CUDA(cudaGetDevice(&dev));
    KRR_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    // the dynamic allowance is what the opt-in maximum leaves after the static arrays
    cudaFuncAttributes fa{};
    KRR_TRY_CUDA(cudaFuncGetAttributes(&fa, fn));
    KRR_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      optin - (int)fa.sharedSizeBytes));
    done[fn] = 1;
    return KRR_OK;
}

const char* const kPhaseNames[PH_COUNT] = {"kmvm", "sketch", "omega", "qrcp", "fgemm", "gram",
                                           "chol", "apply", "resid_hp", "cgvec", "prep"};

static cudaEvent_t pool_event(krr_ctx* ctx) {
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

Phase::Phase(krr_ctx* ctx, int id) : ctx_(ctx), id_(id) {
    if (!ctx_->prof) return;
    start_ = pool_event(ctx_);
    if (start_) cudaEventRecord(start_, ctx_->stream);
}

Phase::~Phase() {
    if (!ctx_->prof || !start_) return;
    cudaEvent_t stop = pool_event(ctx_);
    if (!stop) return;
    cudaEventRecord(stop, ctx_->stream);
    ctx_->prof_recs.push_back(PhaseRec{start_, stop, id_});
}

int buf(krr_ctx* ctx, const char* name, size_t bytes, void** out) {
    Buf& b = ctx->bufs[name];
    if (bytes == 0) bytes = 16;
    if (b.bytes < bytes) {
        if (b.p) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
        }
        const size_t want = (bytes + 255) / 256 * 256;
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return fail(ctx, KRR_E_NOMEM, std::string("workspace '") + name + "': " +
                                              cudaGetErrorString(e));
        }
        b.bytes = want;
    }
    *out = b.p;
    return KRR_OK;
}

// launchers implemented in cg.cu that only the drivers use
int cg_vec_blocks(krr_ctx* ctx);
int launch_cg_start(krr_ctx* ctx, const float* r, const float* z, int nrhs, double* rz_part,
                    double* rr_part);
int launch_cg_alpha(krr_ctx* ctx, const float* p, const float* q, int nrhs, double* part);
int launch_cg_update_xr(krr_ctx* ctx, float* x, float* r, const float* p, const float* q, int nrhs,
                        double* part, double tol2);
int launch_cg_beta_p(krr_ctx* ctx, float* p, const float* z, int nrhs, const double* rz_part);
int launch_cg_set_active(krr_ctx* ctx, const int* act_host, int nrhs);
int launch_identity_apply(krr_ctx* ctx, const float* R, int nrhs, float* Z, double* rz_part);
int launch_identity_apply64(krr_ctx* ctx, const double* R, int nrhs, double* Z, double* rz_part);

// Extreme eigenvalues of the symmetric tridiagonal with diagonal d and off-diagonal e
// (e[j] couples j-1 and j, e[0] unused) by bisection on Sturm counts: the number of
// negative pivots of the LDL^T factorisation of T - x I is the number of eigenvalues below x.
static int sturm_below(const std::vector<double>& d, const std::vector<double>& e, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t j = 0; j < d.size(); ++j) {
        q = (d[j] - x) - (j ? e[j] * e[j] / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}
static void tridiag_extremes(const std::vector<double>& d, const std::vector<double>& e, double* lo,
                             double* hi) {
    const int m = (int)d.size();
    double a = HUGE_VAL, b = -HUGE_VAL;   // Gershgorin bracket
    for (int j = 0; j < m; ++j) {
        const double r = (j ? std::fabs(e[j]) : 0.0) + (j + 1 < m ? std::fabs(e[j + 1]) : 0.0);
        a = std::min(a, d[j] - r);
        b = std::max(b, d[j] + r);
    }
    auto kth = [&](int k) {   // the k-th smallest eigenvalue (1-based)
        double l = a, h = b;
        for (int it = 0; it < 200 && h - l > 1e-15 * std::max(std::fabs(l), std::fabs(h)); ++it) {
            const double mid = 0.5 * (l + h);
            if (sturm_below(d, e, mid) >= k) h = mid;
            else l = mid;
        }
        return 0.5 * (l + h);
    };
    *lo = kth(1);
    *hi = kth(m);
}

static const double LOG2E = 1.4426950408889634;

// g = 2 (f - yv) / m and per-block partial sums of (f - yv)^2, all FP64
__global__ void k_val_grad64(const double* __restrict__ f, const float* __restrict__ yv, long long m,
                             double* __restrict__ g, double* __restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = f[i] - (double)yv[i];
        g[i] = 2.0 * r / (double)m;
        s += r * r;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// g = 2 (f - yv) / m and per-block partial sums of (f - yv)^2 (FP64)
__global__ void k_val_grad(const float* __restrict__ f, const float* __restrict__ yv, long long m,
                           float* __restrict__ g, double* __restrict__ part) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = (double)f[i] - (double)yv[i];
        g[i] = (float)(2.0 * r / (double)m);
        s += r * r;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

static int check_points(krr_ctx* ctx, const void* X, long long n, int d) {
    if (!X) return fail(ctx, KRR_E_INVAL, "null point array");
    if (n < 1) return fail(ctx, KRR_E_INVAL, "n must be >= 1");
    if (n > 0x7fffffffLL) return fail(ctx, KRR_E_INVAL, "n must be < 2^31");
    if (d < 1 || d > KRR_MAX_DIM) return fail(ctx, KRR_E_INVAL, "d must be in [1, 64]");
    return KRR_OK;
}

static int check_sigma_beta(krr_ctx* ctx, double sigma, double beta, bool need_beta) {
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(ctx, KRR_E_INVAL, "sigma must be > 0");
    if (need_beta && (!(beta > 0.0) || !std::isfinite(beta)))
        return fail(ctx, KRR_E_INVAL, "beta must be > 0");
    if (!need_beta && (!(beta >= 0.0) || !std::isfinite(beta)))
        return fail(ctx, KRR_E_INVAL, "beta must be >= 0");
    return KRR_OK;
}

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------- preconditioner build
static int build_from_anchors(krr_ctx* ctx, const int* S_dev, int k_eff) {
    const long long n = ctx->n;
    const int d = ctx->d, ps = ctx->ps;
    ctx->k_eff = k_eff;
    KRR_RET(bufT(ctx, "S", (size_t)k_eff, &ctx->S));
    if (S_dev != ctx->S)
        KRR_TRY_CUDA(cudaMemcpyAsync(ctx->S, S_dev, sizeof(int) * k_eff, cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    KRR_RET(bufT(ctx, "PS", (size_t)k_eff * ps, &ctx->PS));
    KRR_RET(bufT(ctx, "XS", (size_t)k_eff * d, &ctx->XS));
    {
        Phase ph(ctx, PH_PREP);
        KRR_RET(launch_gather_pack(ctx, ctx->P, ps, ctx->X, d, ctx->S, k_eff, ctx->PS, ctx->XS));
    }

    // L1 L1^T = K_SS (FP64), anchors in pivot order.  K_SS has a unit diagonal, so the
    // Cholesky pivot of anchor j is its conditional variance given the anchors before it;
    // where it falls below opts.pivot_tol the anchor adds nothing FP32 arithmetic can
    // resolve and only inflates L1^{-1}, so the anchor set ends there (the columns before
    // the failing one are final; the factor is recomputed for the kept prefix).
    double *L1, *L1inv;
    KRR_RET(bufT(ctx, "L1", (size_t)k_eff * k_eff, &L1));
    KRR_RET(bufT(ctx, "L1inv", (size_t)k_eff * k_eff, &L1inv));
    int info = 0;
    {
        Phase ph_chol(ctx, PH_CHOL);
        KRR_RET(launch_kss(ctx, ctx->XS, k_eff, d, ctx->sigma, L1));
        KRR_RET(launch_potrf(ctx, L1, k_eff, &info, ctx->opts.pivot_tol));
        if (info != 0) {
            const int keep = info - 1;
            if (keep < 1) return fail(ctx, KRR_E_NONFINITE, "first anchor pivot is not positive");
            k_eff = keep;
            ctx->k_eff = keep;
            KRR_RET(launch_kss(ctx, ctx->XS, k_eff, d, ctx->sigma, L1));   // prefix of the same S
            KRR_RET(launch_potrf(ctx, L1, k_eff, &info, 0.0));
            if (info != 0) return fail(ctx, KRR_E_NOTSPD, "Cholesky of K_SS failed");
        }
        KRR_RET(launch_set_identity(ctx, L1inv, k_eff));
        KRR_RET(launch_trsm_lower(ctx, L1, L1inv, k_eff));
    }

    // F = K(X, X_S) L1^{-T}  (n x ldF)
    ctx->ldF = (k_eff + 3) / 4 * 4;
    float* W32;
    KRR_RET(bufT(ctx, "W32", (size_t)k_eff * ctx->ldF, &W32));
    KRR_RET(launch_to_float_transposed(ctx, L1inv, k_eff, W32, ctx->ldF));
    KRR_RET(bufT(ctx, "F", (size_t)n * ctx->ldF, &ctx->F));
    {
        Phase ph(ctx, PH_FGEMM);
        KRR_TRY_CUDA(cudaMemsetAsync(ctx->F, 0, sizeof(float) * n * ctx->ldF, ctx->stream));
        KRR_RET(launch_kgemm(ctx, ctx->P, n, ctx->PS, k_eff, d, W32, ctx->ldF, k_eff, ctx->F,
                             ctx->ldF));
    }

    // G = beta I + F^T F = L2 L2^T;  T2 = L2^{-1}
    double* G;
    KRR_RET(bufT(ctx, "G", (size_t)k_eff * k_eff, &G));
    {
        Phase ph(ctx, PH_GRAM);
        KRR_RET(launch_gram(ctx, ctx->F, n, k_eff, ctx->ldF, ctx->beta, G));
    }
    Phase ph_chol2(ctx, PH_CHOL);   // until the end of the build
    KRR_RET(launch_potrf(ctx, G, k_eff, &info));
    if (info != 0) return fail(ctx, KRR_E_NOTSPD, "Cholesky of beta I + F^T F failed");
    KRR_RET(bufT(ctx, "T2", (size_t)k_eff * k_eff, &ctx->T2));
    KRR_RET(bufT(ctx, "T2t", (size_t)k_eff * k_eff, &ctx->T2t));
    KRR_RET(launch_set_identity(ctx, ctx->T2, k_eff));
    KRR_RET(launch_trsm_lower(ctx, G, ctx->T2, k_eff));
    KRR_RET(launch_transpose64(ctx, ctx->T2, ctx->T2t, k_eff));
    return KRR_OK;
}

static bool use_tc(const krr_ctx* ctx, int d) { return ctx->opts.precision == 1 && kernel_dim(d) <= 16; }

// Raw coordinates of the built point set in the packed layout (mu = 0, s = 1), made once.
static int ensure_raw_points(krr_ctx* ctx) {
    if (ctx->Praw) return KRR_OK;
    double* mu0;
    KRR_RET(bufT(ctx, "mu0", (size_t)ctx->d, &mu0));
    KRR_TRY_CUDA(cudaMemsetAsync(mu0, 0, sizeof(double) * ctx->d, ctx->stream));
    KRR_RET(bufT(ctx, "Praw", (size_t)ctx->n * ctx->ps, &ctx->Praw));
    return launch_pack(ctx, ctx->X, ctx->n, ctx->d, mu0, 1.0, ctx->Praw);
}

// (K + beta I) V for the built point set in product form 0 (FP32 expansion), 1 (tensor
// cores, when built) or 2 (FP32 on raw coordinate differences).
int square_product(krr_ctx* ctx, const float* V, int nrhs, float* Q, int form) {
    if (form == 1 && ctx->FA)
        return launch_kmvm_tc(ctx, ctx->FA, ctx->n, ctx->FB, ctx->n, ctx->d, (float)ctx->beta, V, nrhs, Q);
    if (form == 2) {
        KRR_RET(ensure_raw_points(ctx));
        return launch_kmvm(ctx, ctx->Praw, ctx->n, ctx->Praw, ctx->n, ctx->d, (float)ctx->beta, V, nrhs,
                           Q, (float)(-ctx->s));
    }
    return launch_kmvm(ctx, ctx->P, ctx->n, ctx->P, ctx->n, ctx->d, (float)ctx->beta, V, nrhs, Q);
}

static int build_common(krr_ctx* ctx, const float* X, long long n, int d, double sigma,
                        double beta) {
    ctx->built = false;
    ctx->X = X;
    ctx->n = n;
    ctx->d = d;
    ctx->ps = packed_stride(d);
    ctx->sigma = sigma;
    ctx->beta = beta;
    ctx->s = LOG2E / (2.0 * sigma * sigma);
    double* mu;
    KRR_RET(bufT(ctx, "mu", (size_t)d, &mu));
    KRR_RET(bufT(ctx, "P", (size_t)n * ctx->ps, &ctx->P));
    Phase ph(ctx, PH_PREP);
    KRR_RET(launch_mean(ctx, X, n, d, mu));
    KRR_RET(launch_pack(ctx, X, n, d, mu, ctx->s, ctx->P));
    ctx->FA = ctx->FB = nullptr;
    ctx->Praw = nullptr;
    if (use_tc(ctx, d)) {
        KRR_RET(bufT(ctx, "tc_FA", tc_feature_bytes(n, d), &ctx->FA));
        KRR_RET(bufT(ctx, "tc_FB", tc_feature_bytes(n, d), &ctx->FB));
        KRR_RET(launch_tc_features(ctx, ctx->P, n, d, 0, ctx->FA));
        KRR_RET(launch_tc_features(ctx, ctx->P, n, d, 1, ctx->FB));
    }
    return KRR_OK;
}

}  // namespace krr

using namespace krr;

extern "C" {

int krr_default_opts(krr_opts* o) {
    if (!o) return KRR_E_INVAL;
    std::memset(o, 0, sizeof(*o));
    o->max_iter = 5000;
    o->refine_max = 40;
    o->oversample = 5;
    o->check_every = 1;
    o->inner_tol = 1e-2;
    o->anchor_rtol = 1e-5;
    o->pivot_tol = 1e-6;
    o->precision = 0;
    o->escalate = 1;
    o->recurrence = 0;
    o->ex2_correct = 1;
    o->tc_pv = 1;
    o->tc_vfold = 1;
    return KRR_OK;
}

int krr_create(krr_ctx** out, const krr_opts* opts, void* stream) {
    if (!out) return KRR_E_INVAL;
    *out = nullptr;
    krr_ctx* ctx = new krr_ctx();
    if (opts) ctx->opts = *opts;
    else krr_default_opts(&ctx->opts);
    if (ctx->opts.max_iter < 1 || ctx->opts.refine_max < 1 || ctx->opts.oversample < 0 ||
        ctx->opts.check_every < 1 || !(ctx->opts.inner_tol > 0.0) || ctx->opts.inner_tol >= 1.0 ||
        ctx->opts.residual < 0 || ctx->opts.residual > 1 || ctx->opts.precision < 0 ||
        ctx->opts.precision > 2 || ctx->opts.escalate < 0 || ctx->opts.escalate > 1 ||
        ctx->opts.sparse_r < 0 || ctx->opts.sparse_r > 1024 ||
        (ctx->opts.wait_limit_log2 != 0 &&
         (ctx->opts.wait_limit_log2 < 10 || ctx->opts.wait_limit_log2 > 40)) ||
        ctx->opts.test_stall_copies < 0 || ctx->opts.test_stall_copies > 1 ||
        ctx->opts.recurrence < 0 || ctx->opts.recurrence > 2 ||
        ctx->opts.no_precond < 0 || ctx->opts.no_precond > 1 ||
        ctx->opts.ex2_correct < 0 || ctx->opts.ex2_correct > 1 || ctx->opts.tc_pv < 0 ||
        ctx->opts.tc_pv > 2 || ctx->opts.autotune < 0 || ctx->opts.autotune > 1 ||
        ctx->opts.tc_vfold < 0 || ctx->opts.tc_vfold > 1 ||
        !(ctx->opts.strong_f == 0.0 || ctx->opts.strong_f > 1.0) || ctx->opts.strong_swaps < 0 ||
        !(ctx->opts.anchor_rtol >= 0.0) || !(ctx->opts.pivot_tol >= 0.0) || ctx->opts.pivot_tol >= 1.0) {
        delete ctx;
        return KRR_E_INVAL;
    }
    ctx->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return KRR_E_CUDA;
    }
    if (cudaMalloc(&ctx->cg, sizeof(CGScalars)) != cudaSuccess ||
        cudaMallocHost(&ctx->cg_host, sizeof(CGScalars)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->cg) cudaFree(ctx->cg);
        delete ctx;
        return KRR_E_NOMEM;
    }
    *out = ctx;
    return KRR_OK;
}

void krr_destroy(krr_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->prof_recs) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (auto e : ctx->prof_pool) cudaEventDestroy(e);
    for (auto& kv : ctx->bufs)
        if (kv.second.p) cudaFree(kv.second.p);
    if (ctx->cg) cudaFree(ctx->cg);
    if (ctx->cg_host) cudaFreeHost(ctx->cg_host);
    delete ctx;
}

const char* krr_last_error(const krr_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int krr_profile_enable(krr_ctx* ctx, int on) {
    if (!ctx) return KRR_E_INVAL;
    cudaStreamSynchronize(ctx->stream);
    for (auto& r : ctx->prof_recs) {
        ctx->prof_pool.push_back(r.start);
        ctx->prof_pool.push_back(r.stop);
    }
    ctx->prof_recs.clear();
    ctx->prof = on != 0;
    return KRR_OK;
}

int krr_profile_read(krr_ctx* ctx, const char* phase, double* total_ms, long long* count) {
    if (!ctx || !phase || !total_ms || !count) return KRR_E_INVAL;
    int id = -1;
    for (int i = 0; i < PH_COUNT; ++i)
        if (std::strcmp(phase, kPhaseNames[i]) == 0) id = i;
    if (id < 0) return fail(ctx, KRR_E_INVAL, std::string("unknown phase ") + phase);
    double tot = 0.0;
    long long cnt = 0;
    for (auto& r : ctx->prof_recs) {
        if (r.phase != id) continue;
        float ms = 0.f;
        if (cudaEventSynchronize(r.stop) != cudaSuccess ||
            cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, KRR_E_CUDA, "profile event read failed");
        }
        tot += ms;
        ++cnt;
    }
    *total_ms = tot;
    *count = cnt;
    return KRR_OK;
}

long long krr_launch_count(const krr_ctx* ctx) { return ctx ? ctx->launches : 0; }

int krr_kmvm(krr_ctx* ctx, const float* Xr, long long nr, const float* Xc, long long nc, int d,
             double sigma, double beta, const float* V, int nrhs, float* Q) {
    if (!ctx) return KRR_E_INVAL;
    KRR_RET(check_points(ctx, Xr, nr, d));
    KRR_RET(check_points(ctx, Xc, nc, d));
    KRR_RET(check_sigma_beta(ctx, sigma, beta, false));
    if (!V || !Q) return fail(ctx, KRR_E_INVAL, "null V or Q");
    if (nrhs < 1 || nrhs > KRR_MAX_RHS) return fail(ctx, KRR_E_INVAL, "nrhs must be in [1, 16]");
    if (beta != 0.0 && nr != nc) return fail(ctx, KRR_E_INVAL, "beta needs a square product");
    const int ps = packed_stride(d);
    const double s = LOG2E / (2.0 * sigma * sigma);
    const bool raw = ctx->opts.precision == 2;
    double* mu;
    float *Pc, *Pr;
    KRR_RET(bufT(ctx, "kmvm_mu", (size_t)d, &mu));
    KRR_RET(bufT(ctx, "kmvm_Pc", (size_t)nc * ps, &Pc));
    if (raw) {
        // exact-difference form: raw coordinates (mu = 0, unit scale)
        KRR_TRY_CUDA(cudaMemsetAsync(mu, 0, sizeof(double) * d, ctx->stream));
        KRR_RET(launch_pack(ctx, Xc, nc, d, mu, 1.0, Pc));
        Pr = Pc;
        if (!(Xr == Xc && nr == nc)) {
            KRR_RET(bufT(ctx, "kmvm_Pr", (size_t)nr * ps, &Pr));
            KRR_RET(launch_pack(ctx, Xr, nr, d, mu, 1.0, Pr));
        }
        return launch_kmvm(ctx, Pr, nr, Pc, nc, d, (float)beta, V, nrhs, Q, (float)(-s));
    }
    KRR_RET(launch_mean(ctx, Xc, nc, d, mu));
    KRR_RET(launch_pack(ctx, Xc, nc, d, mu, s, Pc));
    if (Xr == Xc && nr == nc) {
        Pr = Pc;
    } else {
        KRR_RET(bufT(ctx, "kmvm_Pr", (size_t)nr * ps, &Pr));
        KRR_RET(launch_pack(ctx, Xr, nr, d, mu, s, Pr));
    }
    if (use_tc(ctx, d)) {
        unsigned char *FA, *FB;
        KRR_RET(bufT(ctx, "kmvm_FA", tc_feature_bytes(nr, d), &FA));
        KRR_RET(bufT(ctx, "kmvm_FB", tc_feature_bytes(nc, d), &FB));
        KRR_RET(launch_tc_features(ctx, Pr, nr, d, 0, FA));
        KRR_RET(launch_tc_features(ctx, Pc, nc, d, 1, FB));
        int* err;
        int herr = 0;
        KRR_RET(bufT(ctx, "tc_err", 1, &err));
        KRR_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
        KRR_RET(launch_kmvm_tc(ctx, FA, nr, FB, nc, d, (float)beta, V, nrhs, Q));
        KRR_TRY_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
        if (herr) return fail(ctx, KRR_E_TIMEOUT, "tensor-core product: a bounded wait timed out");
        return KRR_OK;
    }
    KRR_RET(launch_kmvm(ctx, Pr, nr, Pc, nc, d, (float)beta, V, nrhs, Q));
    return KRR_OK;
}

int krr_residual_hp(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                    const float* Y, const double* A, int nrhs, double* R) {
    if (!ctx) return KRR_E_INVAL;
    KRR_RET(check_points(ctx, X, n, d));
    KRR_RET(check_sigma_beta(ctx, sigma, beta, false));
    if (!Y || !A || !R) return fail(ctx, KRR_E_INVAL, "null Y, A or R");
    if (nrhs < 1 || nrhs > KRR_MAX_RHS) return fail(ctx, KRR_E_INVAL, "nrhs must be in [1, 16]");
    return launch_residual_hp(ctx, X, n, d, sigma, beta, Y, A, nrhs, R);
}

int krr_residual_ff(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                    const float* Y, const double* A, int nrhs, double* R) {
    if (!ctx) return KRR_E_INVAL;
    KRR_RET(check_points(ctx, X, n, d));
    KRR_RET(check_sigma_beta(ctx, sigma, beta, false));
    if (!Y || !A || !R) return fail(ctx, KRR_E_INVAL, "null Y, A or R");
    if (nrhs < 1 || nrhs > KRR_MAX_RHS) return fail(ctx, KRR_E_INVAL, "nrhs must be in [1, 16]");
    return launch_residual_ff(ctx, X, n, d, sigma, beta, Y, A, nrhs, R);
}

int krr_omega(krr_ctx* ctx, unsigned long long seed, int l, long long n, float* OmT) {
    if (!ctx) return KRR_E_INVAL;
    if (!OmT || l < 1 || n < 1) return fail(ctx, KRR_E_INVAL, "bad omega arguments");
    return launch_omega(ctx, seed, l, n, l, OmT);
}

static int sketch_internal(krr_ctx* ctx, long long n, int l, unsigned long long seed, float** Yout,
                           int* ldy, bool tensor_cores) {
    const int ld = (l + 3) / 4 * 4;
    float* Y;
    KRR_RET(bufT(ctx, "sketch", (size_t)n * ld, &Y));
    if (tensor_cores && ctx->FA) {
        // BF16 Omega in tensor-core tiles and the two-MMA sketch
        const long long npad = (n + 255) / 256 * 256;
        const int nab = (l + 255) / 256, njc_alloc = (int)(npad / 64);
        void* Om;
        KRR_RET(buf(ctx, "omega_bf16", (size_t)nab * 256 * npad * 2, &Om));
        {
            Phase ph(ctx, PH_OMEGA);
            KRR_RET(launch_omega_bf16_tiled(ctx, seed, l, n, nab, njc_alloc, Om));
        }
        Phase ph(ctx, PH_SKETCH);
        KRR_RET(launch_sketch_tc(ctx, ctx->FA, ctx->FB, n, ctx->d, Om, l, njc_alloc, Y, ld));
    } else {
        float* Om;
        KRR_RET(bufT(ctx, "omega", (size_t)n * ld, &Om));
        {
            Phase ph(ctx, PH_OMEGA);
            KRR_RET(launch_omega(ctx, seed, l, n, ld, Om));
        }
        Phase ph(ctx, PH_SKETCH);
        KRR_RET(launch_kgemm(ctx, ctx->P, n, ctx->P, n, ctx->d, Om, ld, ld, Y, ld));
    }
    *Yout = Y;
    *ldy = ld;
    return KRR_OK;
}

int krr_sketch(krr_ctx* ctx, const float* X, long long n, int d, double sigma, int l,
               unsigned long long seed, float* Y) {
    if (!ctx) return KRR_E_INVAL;
    KRR_RET(check_points(ctx, X, n, d));
    KRR_RET(check_sigma_beta(ctx, sigma, 0.0, false));
    if (!Y || l < 1) return fail(ctx, KRR_E_INVAL, "bad sketch arguments");
    // uses the build state's packed points; the build state is reset
    KRR_RET(build_common(ctx, X, n, d, sigma, 1.0));
    float* Yi;
    int ld;
    KRR_RET(sketch_internal(ctx, n, l, seed, &Yi, &ld, true));
    KRR_TRY_CUDA(cudaMemcpy2DAsync(Y, sizeof(float) * l, Yi, sizeof(float) * ld, sizeof(float) * l,
                                   n, cudaMemcpyDeviceToDevice, ctx->stream));
    return KRR_OK;
}

int krr_sparse_draw(krr_ctx* ctx, unsigned long long seed, int l, int r, long long n, int* R, float* S) {
    if (!ctx) return KRR_E_INVAL;
    if (!R || !S || l < 1 || r < 1 || n < 1 || n > 0x7fffffffLL)
        return fail(ctx, KRR_E_INVAL, "bad sparse draw arguments");
    return launch_sparse_draw(ctx, seed, l, r, n, R, S);
}

int krr_sparse_sketch(krr_ctx* ctx, const float* X, long long n, int d, double sigma, int l, int r,
                      unsigned long long seed, float* Y) {
    if (!ctx) return KRR_E_INVAL;
    KRR_RET(check_points(ctx, X, n, d));
    KRR_RET(check_sigma_beta(ctx, sigma, 0.0, false));
    if (!Y || l < 1 || r < 1) return fail(ctx, KRR_E_INVAL, "bad sparse sketch arguments");
    KRR_RET(build_common(ctx, X, n, d, sigma, 1.0));   // packed points; the build state is reset
    int* R;
    float* S;
    KRR_RET(bufT(ctx, "sp_R", (size_t)l * r, &R));
    KRR_RET(bufT(ctx, "sp_S", (size_t)l * r, &S));
    KRR_RET(launch_sparse_draw(ctx, seed, l, r, n, R, S));
    Phase ph(ctx, PH_SKETCH);
    return launch_sparse_sketch(ctx, ctx->P, n, d, R, S, l, r, Y, l);
}

int krr_qrcp(krr_ctx* ctx, float* Y, long long n, int l, int k, int* piv, float* rdiag) {
    if (!ctx) return KRR_E_INVAL;
    if (!Y || !piv || !rdiag || n < 1 || l < 1 || k < 1 || k > n)
        return fail(ctx, KRR_E_INVAL, "bad qrcp arguments");
    return launch_qrcp(ctx, Y, n, l, l, k, piv, rdiag);
}

int krr_build_precond(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                      int k, unsigned long long seed) {
    if (!ctx) return KRR_E_INVAL;
    KRR_RET(check_points(ctx, X, n, d));
    KRR_RET(check_sigma_beta(ctx, sigma, beta, true));
    if (k < 1 || k > n) return fail(ctx, KRR_E_INVAL, "k must be in [1, n]");
    const double t0 = now_ms();
    KRR_RET(build_common(ctx, X, n, d, sigma, beta));
    const int l = (int)std::min<long long>(n, (long long)k + ctx->opts.oversample);
    if (l > 4096) return fail(ctx, KRR_E_INVAL, "k + oversample must be <= 4096");
    ctx->k = k;
    ctx->l = l;
    float* Y;
    int ld;
    if (ctx->opts.sparse_r > 0) {
        // Algorithm 2: l projections with sparse_r nonzeros each
        const int r = ctx->opts.sparse_r;
        int* R;
        float* S;
        ld = (l + 3) / 4 * 4;
        KRR_RET(bufT(ctx, "sketch", (size_t)n * ld, &Y));
        KRR_RET(bufT(ctx, "sp_R", (size_t)l * r, &R));
        KRR_RET(bufT(ctx, "sp_S", (size_t)l * r, &S));
        {
            Phase ph(ctx, PH_OMEGA);
            KRR_RET(launch_sparse_draw(ctx, seed, l, r, n, R, S));
        }
        Phase ph(ctx, PH_SKETCH);
        KRR_RET(launch_sparse_sketch(ctx, ctx->P, n, d, R, S, l, r, Y, ld));
    } else {
        KRR_RET(sketch_internal(ctx, n, l, seed, &Y, &ld, true));
    }
    int* piv;
    float* rdiag;
    KRR_RET(bufT(ctx, "piv", (size_t)k, &piv));
    KRR_RET(bufT(ctx, "rdiag", (size_t)k, &rdiag));
    ctx->rrqr_swaps = 0;
    ctx->rrqr_rho = 0.0;
    {
        Phase ph(ctx, PH_QRCP);
        if (ctx->opts.strong_f > 1.0 && k < n)
            KRR_RET(launch_strong_rrqr(ctx, Y, n, l, ld, k, ctx->opts.strong_f,
                                       ctx->opts.strong_swaps > 0 ? ctx->opts.strong_swaps : 64, piv, rdiag,
                                       &ctx->rrqr_swaps, &ctx->rrqr_rho));
        else
            KRR_RET(launch_qrcp(ctx, Y, n, l, ld, k, piv, rdiag));
    }
    std::vector<float> rd(k);
    KRR_TRY_CUDA(cudaMemcpyAsync(rd.data(), rdiag, sizeof(float) * k, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    int tc_err = 0;
    if (ctx->FA && ctx->opts.sparse_r == 0) {   // the tensor-core sketch ran
        int* err;
        KRR_RET(bufT(ctx, "tc_err", 1, &err));
        KRR_TRY_CUDA(cudaMemcpyAsync(&tc_err, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    }
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    if (tc_err) return fail(ctx, KRR_E_TIMEOUT, "tensor-core sketch: a bounded wait timed out");
    int k_eff = 0;
    const float thr = (float)(ctx->opts.anchor_rtol * rd[0]);
    while (k_eff < k && rd[k_eff] > thr && std::isfinite(rd[k_eff])) ++k_eff;
    if (k_eff < 1) return fail(ctx, KRR_E_NONFINITE, "sketch has no nonzero pivot");
    KRR_RET(build_from_anchors(ctx, piv, k_eff));
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->build_ms = now_ms() - t0;
    ctx->built = true;
    return KRR_OK;
}

int krr_build_precond_anchors(krr_ctx* ctx, const float* X, long long n, int d, double sigma,
                              double beta, const int* S, int k) {
    if (!ctx) return KRR_E_INVAL;
    KRR_RET(check_points(ctx, X, n, d));
    KRR_RET(check_sigma_beta(ctx, sigma, beta, true));
    if (!S || k < 1 || k > n) return fail(ctx, KRR_E_INVAL, "bad anchors");
    std::vector<int> hs(k);
    KRR_TRY_CUDA(cudaMemcpyAsync(hs.data(), S, sizeof(int) * k, cudaMemcpyDeviceToHost, ctx->stream));
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int a = 0; a < k; ++a)
        if (hs[a] < 0 || hs[a] >= n) return fail(ctx, KRR_E_INVAL, "anchor index out of range");
    const double t0 = now_ms();
    KRR_RET(build_common(ctx, X, n, d, sigma, beta));
    ctx->k = k;
    ctx->l = 0;
    KRR_RET(build_from_anchors(ctx, S, k));
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->build_ms = now_ms() - t0;
    ctx->built = true;
    return KRR_OK;
}

int krr_anchor_stats(krr_ctx* ctx, int* rrqr_swaps, double* rrqr_rho) {
    if (!ctx || !rrqr_swaps || !rrqr_rho) return KRR_E_INVAL;
    if (!ctx->built) return fail(ctx, KRR_E_STATE, "no preconditioner built");
    *rrqr_swaps = ctx->rrqr_swaps;
    *rrqr_rho = ctx->rrqr_rho;
    return KRR_OK;
}

int krr_get_anchors(krr_ctx* ctx, int* S, int* k_eff) {
    if (!ctx || !k_eff) return KRR_E_INVAL;
    if (!ctx->built) return fail(ctx, KRR_E_STATE, "no preconditioner built");
    *k_eff = ctx->k_eff;
    if (S)
        KRR_TRY_CUDA(cudaMemcpyAsync(S, ctx->S, sizeof(int) * ctx->k_eff, cudaMemcpyDeviceToDevice,
                                     ctx->stream));
    return KRR_OK;
}

int krr_precond_apply(krr_ctx* ctx, const float* In, int nrhs, float* Out) {
    if (!ctx) return KRR_E_INVAL;
    if (!ctx->built) return fail(ctx, KRR_E_STATE, "no preconditioner built");
    if (!In || !Out || nrhs < 1 || nrhs > KRR_MAX_RHS) return fail(ctx, KRR_E_INVAL, "bad apply arguments");
    return launch_apply_precond(ctx, In, nrhs, Out, nullptr);
}


// (K + beta I) p for FP64 p (n x nrhs): p split into FP32 hi/lo column pairs, FP64 sums out.
static int square_product64(krr_ctx* ctx, const double* p64, int nrhs, float* psplit, double* q64,
                            int form) {
    KRR_RET(launch_split_hilo(ctx, p64, ctx->n, nrhs, psplit));
    if (form == 1 && ctx->FA)
        return launch_kmvm_tc(ctx, ctx->FA, ctx->n, ctx->FB, ctx->n, ctx->d, (float)ctx->beta, psplit,
                              2 * nrhs, nullptr, p64, q64);
    if (form == 2) {
        KRR_RET(ensure_raw_points(ctx));
        const float nsc = (float)(-ctx->s);
        return launch_kmvm(ctx, ctx->Praw, ctx->n, ctx->Praw, ctx->n, ctx->d, (float)ctx->beta, psplit,
                           2 * nrhs, nullptr, nsc, p64, q64, (float)(-ctx->s - (double)nsc));
    }
    return launch_kmvm(ctx, ctx->P, ctx->n, ctx->P, ctx->n, ctx->d, (float)ctx->beta, psplit, 2 * nrhs,
                       nullptr, 0.f, p64, q64);
}

int krr_solve(krr_ctx* ctx, const float* X, const float* Y, int nrhs, double tol, double* alpha,
              krr_solve_info* info) {
    if (!ctx) return KRR_E_INVAL;
    if (!ctx->built) return fail(ctx, KRR_E_STATE, "krr_solve before krr_build_precond");
    if (X != ctx->X) return fail(ctx, KRR_E_INVAL, "X differs from the built point set");
    if (!Y || !alpha) return fail(ctx, KRR_E_INVAL, "null Y or alpha");
    if (nrhs < 1 || nrhs > KRR_MAX_RHS) return fail(ctx, KRR_E_INVAL, "nrhs must be in [1, 16]");
    if (!(tol > 0.0) || !(tol < 1.0)) return fail(ctx, KRR_E_INVAL, "tol must be in (0, 1)");
    const double t0 = now_ms();
    const long long n = ctx->n;
    const long long tot = n * nrhs;
    const int nb = cg_vec_blocks(ctx);
    if (nb != cg64_vec_blocks(ctx)) return fail(ctx, KRR_E_STATE, "vector block counts differ");
    double *r64, *ynorm2, *rnorm2;
    float *x, *r, *z, *p, *q;
    double *part1, *part2, *part3;
    KRR_RET(bufT(ctx, "sv_r64", (size_t)tot, &r64));
    KRR_RET(bufT(ctx, "sv_yn", (size_t)KRR_MAX_RHS, &ynorm2));
    KRR_RET(bufT(ctx, "sv_rn", (size_t)KRR_MAX_RHS, &rnorm2));
    KRR_RET(bufT(ctx, "sv_x", (size_t)tot, &x));
    KRR_RET(bufT(ctx, "sv_r", (size_t)tot, &r));
    KRR_RET(bufT(ctx, "sv_z", (size_t)tot, &z));
    KRR_RET(bufT(ctx, "sv_p", (size_t)tot, &p));
    KRR_RET(bufT(ctx, "sv_q", (size_t)tot, &q));
    KRR_RET(bufT(ctx, "sv_part1", (size_t)nb * nrhs, &part1));
    KRR_RET(bufT(ctx, "sv_part2", (size_t)nb * nrhs, &part2));
    KRR_RET(bufT(ctx, "sv_part3", (size_t)nb * nrhs, &part3));

    // FP64 recurrence vectors (opts.recurrence 1, or 2 after an escalation), made on demand
    bool hp = false;
    double *x64 = nullptr, *rr64 = nullptr, *z64 = nullptr, *p64 = nullptr, *q64 = nullptr;
    float* psplit = nullptr;
    auto enter_hp = [&]() -> int {
        KRR_RET(bufT(ctx, "sv_x64", (size_t)tot, &x64));
        KRR_RET(bufT(ctx, "sv_rr64", (size_t)tot, &rr64));
        KRR_RET(bufT(ctx, "sv_z64", (size_t)tot, &z64));
        KRR_RET(bufT(ctx, "sv_p64", (size_t)tot, &p64));
        KRR_RET(bufT(ctx, "sv_q64", (size_t)tot, &q64));
        KRR_RET(bufT(ctx, "sv_psplit", (size_t)2 * tot, &psplit));
        KRR_TRY_CUDA(cudaMemsetAsync(x64, 0, sizeof(double) * tot, ctx->stream));
        hp = true;
        return KRR_OK;
    };
    if (ctx->opts.recurrence == 1) KRR_RET(enter_hp());

    std::vector<double> yn(nrhs), rn(nrhs);
    KRR_RET(launch_dot(ctx, Y, Y, n, nrhs, ynorm2));
    KRR_TRY_CUDA(cudaMemcpyAsync(yn.data(), ynorm2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    KRR_TRY_CUDA(cudaMemsetAsync(alpha, 0, sizeof(double) * tot, ctx->stream));
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int c = 0; c < nrhs; ++c)
        if (!std::isfinite(yn[c])) return fail(ctx, KRR_E_NONFINITE, "non-finite right-hand side");

    krr_solve_info inf;
    std::memset(&inf, 0, sizeof(inf));
    inf.k_eff = ctx->k_eff;
    inf.build_ms = ctx->build_ms;
    int status = KRR_E_NOCONV;
    std::vector<double> lz_alpha, lz_beta;   // CG step lengths and direction updates

    // One preconditioned CG recurrence with reliable updates: whenever the recursive
    // residual of a column has fallen by the factor opts.inner_tol since the last true
    // residual (or looks converged), the correction x is folded into the FP64 alpha and
    // the recursive residual is replaced by y - (K + beta I) alpha evaluated in
    // float-float.  With FP32 vectors the search direction is kept, so the Krylov space
    // is not thrown away; with FP64 vectors (precision-limited problems) the recurrence
    // restarts from each replaced residual.
    const double delta2 = ctx->opts.inner_tol * ctx->opts.inner_tol;
    std::vector<double> rtrue(nrhs);
    std::vector<int> act(nrhs);
    // per column, the alpha with the smallest true residual so far: a solve that ends
    // without reaching tol returns that one, never a worse later iterate
    double* abest;
    KRR_RET(bufT(ctx, "sv_abest", (size_t)tot, &abest));
    std::vector<double> best_rel(nrhs, HUGE_VAL);
    auto zero_x = [&]() -> int {
        KRR_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * tot, ctx->stream));
        if (x64) KRR_TRY_CUDA(cudaMemsetAsync(x64, 0, sizeof(double) * tot, ctx->stream));
        return KRR_OK;
    };
    auto true_residual = [&](bool first) -> int {
        if (first) {
            KRR_RET(launch_convert_up(ctx, Y, r64, tot));
            for (int c = 0; c < nrhs; ++c) rn[c] = yn[c];
        } else {
            KRR_RET(launch_accumulate(ctx, x, alpha, tot));
            if (x64) KRR_RET(launch_add64(ctx, x64, alpha, tot));
            KRR_RET(zero_x());
            {
                Phase ph(ctx, PH_RESID);
                if (ctx->opts.residual == 1)
                    KRR_RET(launch_residual_hp(ctx, ctx->X, n, ctx->d, ctx->sigma, ctx->beta, Y,
                                               alpha, nrhs, r64));
                else
                    KRR_RET(launch_residual_ff(ctx, ctx->X, n, ctx->d, ctx->sigma, ctx->beta, Y,
                                               alpha, nrhs, r64));
            }
            KRR_RET(launch_dot64(ctx, r64, r64, n, nrhs, rnorm2));
            KRR_TRY_CUDA(cudaMemcpyAsync(rn.data(), rnorm2, sizeof(double) * nrhs,
                                         cudaMemcpyDeviceToHost, ctx->stream));
            KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
        }
        double worst = 0.0;
        for (int c = 0; c < nrhs; ++c) {
            const double rel = yn[c] > 0.0 ? std::sqrt(rn[c] / yn[c]) : 0.0;
            if (!std::isfinite(rel)) return fail(ctx, KRR_E_NONFINITE, "non-finite residual");
            inf.rel_residual[c] = rel;
            rtrue[c] = rn[c];
            act[c] = rel > tol ? 1 : 0;
            worst = std::max(worst, rel);
        }
        if (inf.sweeps < 8) inf.sweep_residual[inf.sweeps] = worst;
        for (int c = 0; c < nrhs; ++c)
            if (inf.rel_residual[c] < best_rel[c]) {
                best_rel[c] = inf.rel_residual[c];
                KRR_TRY_CUDA(cudaMemcpyAsync(abest + (size_t)c * n, alpha + (size_t)c * n, sizeof(double) * n,
                                             cudaMemcpyDeviceToDevice, ctx->stream));
            }
        // the recursive residual of either recurrence starts from the true one
        KRR_RET(launch_convert(ctx, r64, r, tot));
        if (hp)
            KRR_TRY_CUDA(cudaMemcpyAsync(rr64, r64, sizeof(double) * tot, cudaMemcpyDeviceToDevice,
                                         ctx->stream));
        return KRR_OK;
    };
    auto any_active = [&]() {
        for (int c = 0; c < nrhs; ++c)
            if (act[c]) return true;
        return false;
    };

    // Product form: the requested one, and the exact-difference FP32 form after an
    // escalation.  The expansion forms (0, 1) round a_i + a_j + 2 x_i.x_j, which costs
    // about eps (|a_i| + |a_j|) per entry; when lambda_max(K) / beta approaches 1/eps that
    // perturbation is as large as beta I: the FP32 operator then meets non-positive
    // curvature, or stops reducing the true residual, and form 2 takes over.
    int form = ctx->opts.precision == 1 ? (ctx->FA ? 1 : 0) : ctx->opts.precision;
    // (Re)start the recurrence from the current recursive residual: z = M^-1 r, p = z.
    auto restart_cg = [&]() -> int {
        if (hp) {
            {
                Phase ph(ctx, PH_APPLY);
                if (ctx->opts.no_precond)
                    KRR_RET(launch_identity_apply64(ctx, rr64, nrhs, z64, part1));
                else
                    KRR_RET(launch_apply_precond64(ctx, rr64, nrhs, z64, part1));
            }
            KRR_RET(launch_cg64_start(ctx, rr64, nrhs, part1, part2));
            KRR_RET(launch_cg_set_active(ctx, act.data(), nrhs));
            KRR_TRY_CUDA(cudaMemcpyAsync(p64, z64, sizeof(double) * tot, cudaMemcpyDeviceToDevice,
                                         ctx->stream));
            return KRR_OK;
        }
        {
            Phase ph(ctx, PH_APPLY);
            if (ctx->opts.no_precond)
                KRR_RET(launch_identity_apply(ctx, r, nrhs, z, part1));
            else
                KRR_RET(launch_apply_precond(ctx, r, nrhs, z, part1));
        }
        KRR_RET(launch_cg_start(ctx, r, z, nrhs, part1, part2));
        KRR_RET(launch_cg_set_active(ctx, act.data(), nrhs));
        KRR_TRY_CUDA(cudaMemcpyAsync(p, z, sizeof(float) * tot, cudaMemcpyDeviceToDevice, ctx->stream));
        return KRR_OK;
    };
    // error word of the tensor-core product (set when one of its bounded waits ran out);
    // read with the CG scalars, into the pinned tail of the scalar mirror
    int* tc_err_dev = nullptr;
    KRR_RET(bufT(ctx, "tc_err", 1, &tc_err_dev));
    int* tc_err_host = &ctx->cg_host->tc_err;
    *tc_err_host = 0;
    KRR_TRY_CUDA(cudaMemsetAsync(tc_err_dev, 0, sizeof(int), ctx->stream));
    KRR_RET(zero_x());
    KRR_RET(true_residual(true));
    if (!any_active()) {
        status = KRR_OK;
    } else {
        KRR_RET(restart_cg());
        int it = 0, since = 0, gapped = 0;
        // Stall watch: `window` = 3x the length of the first cycle (at least 100; 500 until
        // the first cycle ends, which also bounds that cycle before a true residual); if the
        // worst column's true residual has not halved within a window, the product's
        // error is what limits the solve.  A replacement is forced once per window so
        // that a stalled column is measured even when no column triggers one.
        // (plain CG for the condition-number experiment runs its first cycle unforced)
        int window = ctx->opts.no_precond ? ctx->opts.max_iter : 500, it_best = 0;
        double best = 1.0;
        std::vector<double> rec(nrhs);
        bool lanczos_on = true;
        while (true) {
            {
                Phase ph(ctx, PH_KMVM);
                if (hp)
                    KRR_RET(square_product64(ctx, p64, nrhs, psplit, q64, form));
                else
                    KRR_RET(square_product(ctx, p, nrhs, q, form));
            }
            inf.mvm_count++;
            {
                Phase ph(ctx, PH_CGVEC);
                if (hp) {
                    KRR_RET(launch_cg64_alpha(ctx, p64, q64, nrhs, part1));
                    KRR_RET(launch_cg64_update_xr(ctx, x64, rr64, p64, q64, nrhs, part2));
                } else {
                    KRR_RET(launch_cg_alpha(ctx, p, q, nrhs, part1));
                    KRR_RET(launch_cg_update_xr(ctx, x, r, p, q, nrhs, part2, 0.0));
                }
            }
            ++it;
            ++since;
            const bool last = it >= ctx->opts.max_iter;
            if (it % ctx->opts.check_every == 0 || last) {
                KRR_TRY_CUDA(cudaMemcpyAsync(ctx->cg_host, ctx->cg, sizeof(CGScalars),
                                             cudaMemcpyDeviceToHost, ctx->stream));
                if (form == 1)
                    KRR_TRY_CUDA(cudaMemcpyAsync(tc_err_host, tc_err_dev, sizeof(int),
                                                 cudaMemcpyDeviceToHost, ctx->stream));
                KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
                if (form == 1 && *tc_err_host) {
                    status = KRR_E_TIMEOUT;
                    fail(ctx, status, "tensor-core product: a bounded wait timed out");
                    break;
                }
                // column 0's CG coefficients while its first cycle runs uninterrupted
                if (lanczos_on && act[0] && ctx->opts.check_every == 1 && !ctx->cg_host->bad &&
                    ctx->cg_host->a[0] > 0.0 && lz_alpha.size() < 20000) {
                    lz_alpha.push_back(ctx->cg_host->a[0]);
                    lz_beta.push_back(ctx->cg_host->b[0]);   // the previous step's beta
                }
                bool escalate = false;
                if (ctx->cg_host->bad) {
                    if (!ctx->opts.escalate || form == 2 || last) {
                        status = KRR_E_NONFINITE;
                        fail(ctx, status, "non-positive curvature or non-finite value in PCG");
                        break;
                    }
                    // The correction x was built on an operator that is not positive
                    // definite in FP32: it is unverified and is discarded, and the solve
                    // goes on from the best verified alpha of every column.
                    escalate = true;
                    KRR_RET(zero_x());
                    KRR_TRY_CUDA(cudaMemcpyAsync(alpha, abest, sizeof(double) * tot,
                                                 cudaMemcpyDeviceToDevice, ctx->stream));
                }
                bool update = last || escalate || since >= window;
                for (int c = 0; c < nrhs; ++c) {
                    if (!act[c]) continue;
                    const double rr = ctx->cg_host->rr[c];
                    rec[c] = rr;
                    if (rr <= delta2 * rtrue[c] || rr <= 0.25 * tol * tol * yn[c]) update = true;
                }
                if (update) {
                    lanczos_on = false;
                    if (inf.sweeps < 8) inf.sweep_iters[inf.sweeps] = since;
                    if (inf.sweeps == 0) window = std::max(100, 3 * since);
                    inf.sweeps++;
                    since = 0;
                    std::vector<int> was(act);
                    KRR_RET(true_residual(false));
                    if (!any_active()) {
                        status = KRR_OK;
                        break;
                    }
                    if (last || inf.sweeps >= ctx->opts.refine_max) break;
                    // A true residual well above the recursive one means the FP32 operator,
                    // not rounding in the recurrence, set the gap: the old direction is then
                    // no longer conjugate for this residual, so the recurrence restarts.
                    // FP64 vectors restart at every replacement.
                    bool restart = escalate || hp;
                    for (int c = 0; c < nrhs; ++c)
                        if (was[c] && act[c] && !escalate && rtrue[c] > kGapRestart2 * rec[c])
                            restart = true;
                    // two gapped replacements in a row, or a stall: the product's own error,
                    // not the recurrence, limits the solve; move to the exact-difference form
                    gapped = restart && !hp ? gapped + 1 : 0;
                    double w = 0.0;
                    for (int c = 0; c < nrhs; ++c) w = std::max(w, inf.rel_residual[c]);
                    if (w < 0.5 * best) {
                        best = w;
                        it_best = it;
                    }
                    const bool stalled = it - it_best > window;
                    if (ctx->opts.escalate && form != 2 && (gapped >= 2 || escalate || stalled)) {
                        form = 2;
                        restart = true;
                        gapped = 0;
                        it_best = it;
                        best = w;
                        if (ctx->opts.recurrence == 2 && !hp) {
                            // FP64 vectors from here on, starting from the true residual
                            KRR_RET(enter_hp());
                            KRR_TRY_CUDA(cudaMemcpyAsync(rr64, r64, sizeof(double) * tot,
                                                         cudaMemcpyDeviceToDevice, ctx->stream));
                        }
                    } else if (stalled) {
                        restart = true;   // already exact differences: fresh direction
                        it_best = it;
                        best = w;
                    }
                    if (restart) {
                        inf.restarts++;
                        KRR_RET(restart_cg());
                        continue;
                    }
                    KRR_RET(launch_cg_set_active(ctx, act.data(), nrhs));
                }
            }
            {
                Phase ph(ctx, PH_APPLY);
                if (ctx->opts.no_precond)
                    KRR_RET(hp ? launch_identity_apply64(ctx, rr64, nrhs, z64, part3)
                               : launch_identity_apply(ctx, r, nrhs, z, part3));
                else if (hp)
                    KRR_RET(launch_apply_precond64(ctx, rr64, nrhs, z64, part3));
                else
                    KRR_RET(launch_apply_precond(ctx, r, nrhs, z, part3));
            }
            {
                Phase ph(ctx, PH_CGVEC);
                if (hp)
                    KRR_RET(launch_cg64_beta_p(ctx, p64, z64, nrhs, part3));
                else
                    KRR_RET(launch_cg_beta_p(ctx, p, z, nrhs, part3));
            }
        }
        inf.iters = it;
        if (status != KRR_OK) {
            // the last partial correction (if any) is unverified: return each column's best
            for (int c = 0; c < nrhs; ++c)
                if (since > 0 || inf.rel_residual[c] > best_rel[c]) {
                    KRR_TRY_CUDA(cudaMemcpyAsync(alpha + (size_t)c * n, abest + (size_t)c * n,
                                                 sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
                    inf.rel_residual[c] = best_rel[c];
                }
        }
    }
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    // Lanczos tridiagonal of the CG coefficients (alpha_j, beta_j): diagonal
    // 1/alpha_0 and 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal sqrt(beta_{j-1})/alpha_{j-1};
    // its eigenvalues are Ritz values of the preconditioned operator
    if (lz_alpha.size() >= 2) {
        const size_t m = lz_alpha.size();
        std::vector<double> dg(m), of(m, 0.0);
        for (size_t j = 0; j < m; ++j) {
            dg[j] = 1.0 / lz_alpha[j];
            if (j) {
                const double bj = lz_beta[j];   // beta_{j-1}, read with alpha_j
                dg[j] += bj / lz_alpha[j - 1];
                of[j] = std::sqrt(std::max(bj, 0.0)) / lz_alpha[j - 1];
            }
        }
        double lo = 0.0, hi = 0.0;
        tridiag_extremes(dg, of, &lo, &hi);
        inf.lanczos_steps = (int)m;
        inf.cond_estimate = lo > 0.0 ? hi / lo : HUGE_VAL;
    }
    inf.status = status;
    inf.product_form = form;
    inf.recurrence64 = hp ? 1 : 0;
    inf.solve_ms = now_ms() - t0;
    if (info) *info = inf;
    if (status == KRR_E_NOCONV) fail(ctx, status, "tolerance not reached");
    return status;
}

int krr_kmvm_dsigma(krr_ctx* ctx, const float* Xr, long long nr, const float* Xc, long long nc, int d,
                    double sigma, const float* V, float* Q) {
    if (!ctx) return KRR_E_INVAL;
    KRR_RET(check_points(ctx, Xr, nr, d));
    KRR_RET(check_points(ctx, Xc, nc, d));
    KRR_RET(check_sigma_beta(ctx, sigma, 0.0, false));
    if (!V || !Q) return fail(ctx, KRR_E_INVAL, "null V or Q");
    const int ps = packed_stride(d);
    const double s = LOG2E / (2.0 * sigma * sigma);
    double* mu;
    float *Pc, *Pr;
    KRR_RET(bufT(ctx, "kmvm_mu", (size_t)d, &mu));
    KRR_RET(bufT(ctx, "kmvm_Pc", (size_t)nc * ps, &Pc));
    KRR_RET(bufT(ctx, "kmvm_Pr", (size_t)nr * ps, &Pr));
    KRR_RET(launch_mean(ctx, Xc, nc, d, mu));
    KRR_RET(launch_pack(ctx, Xc, nc, d, mu, s, Pc));
    KRR_RET(launch_pack(ctx, Xr, nr, d, mu, s, Pr));
    return launch_kmvm_dsigma(ctx, Pr, nr, Pc, nc, d, V, Q);
}

int krr_grad(krr_ctx* ctx, const float* Y, const float* Xval, long long m, const float* yval, double tol,
             double* loss, double* dlogsigma, double* dlogbeta, double* dy) {
    if (!ctx) return KRR_E_INVAL;
    if (!ctx->built) return fail(ctx, KRR_E_STATE, "krr_grad before krr_build_precond");
    KRR_RET(check_points(ctx, Xval, m, ctx->d));
    if (!Y || !yval || !loss || !dlogsigma || !dlogbeta || !dy)
        return fail(ctx, KRR_E_INVAL, "null argument");
    if (!(tol > 0.0) || !(tol < 1.0)) return fail(ctx, KRR_E_INVAL, "tol must be in (0, 1)");
    if (ctx->d > 16) return fail(ctx, KRR_E_INVAL, "krr_grad needs d <= 16");
    const long long n = ctx->n;
    const int d = ctx->d;
    double *a64, *lam64, *f64, *g64, *b64, *u1, *u2, *sc;
    float* b32;
    KRR_RET(bufT(ctx, "gr_a64", (size_t)n, &a64));
    KRR_RET(bufT(ctx, "gr_lam64", (size_t)n, &lam64));
    KRR_RET(bufT(ctx, "gr_f64", (size_t)m, &f64));
    KRR_RET(bufT(ctx, "gr_g64", (size_t)m, &g64));
    KRR_RET(bufT(ctx, "gr_b64", (size_t)n, &b64));
    KRR_RET(bufT(ctx, "gr_u1", (size_t)m, &u1));
    KRR_RET(bufT(ctx, "gr_u2", (size_t)n, &u2));
    KRR_RET(bufT(ctx, "gr_sc", 8, &sc));
    KRR_RET(bufT(ctx, "gr_b32", (size_t)n, &b32));
    const int nbv = (int)std::min<long long>(2LL * ctx->num_sms, ceil_div(m, 256));
    double* vpart;
    KRR_RET(bufT(ctx, "gr_vpart", (size_t)nbv, &vpart));

    // Every kernel product here is evaluated in float-float: the sigma gradient is a
    // difference of two products that cancel, and finite differences of the loss need it
    // far below FP32 noise.
    // alpha = (K + beta I)^{-1} y
    int rc = krr_solve(ctx, ctx->X, Y, 1, tol, a64, nullptr);
    if (rc != KRR_OK) return rc;
    // f = K(Xval, X) alpha;  g = 2 (f - yval) / m
    KRR_RET(launch_rect_ff(ctx, Xval, m, ctx->X, n, d, ctx->sigma, a64, 0, f64));
    k_val_grad64<<<nbv, 256, 0, ctx->stream>>>(f64, yval, m, g64, vpart);
    KRR_CHECK_LAUNCH();
    // lambda = (K + beta I)^{-1} K(X, Xval) g  (adjoint solve, same preconditioner)
    KRR_RET(launch_rect_ff(ctx, ctx->X, n, Xval, m, d, ctx->sigma, g64, 0, b64));
    KRR_RET(launch_convert(ctx, b64, b32, n));
    rc = krr_solve(ctx, ctx->X, b32, 1, tol, lam64, nullptr);
    if (rc != KRR_OK) return rc;
    KRR_TRY_CUDA(cudaMemcpyAsync(dy, lam64, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    // dL/dlog beta = -beta lambda . alpha
    KRR_RET(launch_dot64(ctx, lam64, a64, n, 1, sc + 0));
    // dL/dlog sigma = g . dK(Xval, X) alpha - lambda . dK(X, X) alpha
    KRR_RET(launch_rect_ff(ctx, Xval, m, ctx->X, n, d, ctx->sigma, a64, 1, u1));
    KRR_RET(launch_dot64(ctx, g64, u1, m, 1, sc + 1));
    KRR_RET(launch_rect_ff(ctx, ctx->X, n, ctx->X, n, d, ctx->sigma, a64, 1, u2));
    KRR_RET(launch_dot64(ctx, lam64, u2, n, 1, sc + 2));
    double h[3];
    std::vector<double> vp(nbv);
    KRR_TRY_CUDA(cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    KRR_TRY_CUDA(cudaMemcpyAsync(vp.data(), vpart, sizeof(double) * nbv, cudaMemcpyDeviceToHost,
                                 ctx->stream));
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    double ssq = 0.0;
    for (double v : vp) ssq += v;
    *loss = ssq / (double)m;
    *dlogbeta = -ctx->beta * h[0];
    *dlogsigma = h[1] - h[2];
    return KRR_OK;
}

int krr_predict(krr_ctx* ctx, const float* Xtest, long long m, const float* alpha, int nrhs,
                float* f) {
    if (!ctx) return KRR_E_INVAL;
    if (!ctx->built) return fail(ctx, KRR_E_STATE, "krr_predict before krr_build_precond");
    KRR_RET(check_points(ctx, Xtest, m, ctx->d));
    if (!alpha || !f) return fail(ctx, KRR_E_INVAL, "null alpha or f");
    if (nrhs < 1 || nrhs > KRR_MAX_RHS) return fail(ctx, KRR_E_INVAL, "nrhs must be in [1, 16]");
    float* Pt;
    double* mu;
    KRR_RET(bufT(ctx, "pred_P", (size_t)m * ctx->ps, &Pt));
    if (ctx->opts.precision == 2) {
        KRR_RET(ensure_raw_points(ctx));
        KRR_RET(bufT(ctx, "mu0", (size_t)ctx->d, &mu));
        KRR_RET(launch_pack(ctx, Xtest, m, ctx->d, mu, 1.0, Pt));
        return launch_kmvm(ctx, Pt, m, ctx->Praw, ctx->n, ctx->d, 0.f, alpha, nrhs, f, (float)(-ctx->s));
    }
    KRR_RET(bufT(ctx, "mu", (size_t)ctx->d, &mu));
    KRR_RET(launch_pack(ctx, Xtest, m, ctx->d, mu, ctx->s, Pt));
    return launch_kmvm(ctx, Pt, m, ctx->P, ctx->n, ctx->d, 0.f, alpha, nrhs, f);
}

}  // extern "C"
