// FP64 recurrence vectors for precision-limited solves (Algorithm 5 step 3).
//
// When lambda_max(K) / beta approaches 1 / eps32 (the 10^6-point cube: lambda_max ~ 8e3,
// beta = 1e-4), a CG recurrence whose x, r and p are rounded to FP32 every iteration loses
// its convergence rate long before the tolerance.  In this mode the recurrence keeps
// x, r, p, z in FP64 and the operators are applied so that rounding does not depend on
// the iteration:
//   * the kernel product takes p as two FP32 columns p = p_hi + p_lo (exact to about
//     2^-48) and returns q = K^ (p_hi + p_lo) + beta p in FP64 (the FP64 tile sums of the
//     product kernels, never rounded to FP32);
//   * the Woodbury apply z = (r - F G^{-1} F^T r) / beta uses the stored FP32 F and the
//     FP64 factor of G = beta I + F^T F, with F^T r and F v summed in float-float from the
//     split r and v, so it is the exact inverse of F F^T + beta I for the stored F up to
//     FP64 rounding: a fixed SPD operator.
#include "internal.cuh"

#include <algorithm>

namespace krr {

constexpr int V64T = 256;

static int vec_blocks64(krr_ctx* ctx, long long n) {
    return (int)std::max<long long>(1, std::min<long long>(4LL * ctx->num_sms, ceil_div(n, 64)));
}

// a = hi + lo with hi = fl32(a), lo = fl32(a - hi): columns 2q (hi) and 2q + 1 (lo) of out
__global__ void k_split_hilo(const double* __restrict__ a, long long n, int nrhs, float* __restrict__ out) {
    const long long tot = n * nrhs;
    for (long long e = (long long)blockIdx.x * V64T + threadIdx.x; e < tot; e += (long long)gridDim.x * V64T) {
        const int q = (int)(e / n);
        const long long i = e - (long long)q * n;
        const double v = a[e];
        const float hi = (float)v;
        out[(size_t)(2 * q) * n + i] = hi;
        out[(size_t)(2 * q + 1) * n + i] = (float)(v - (double)hi);
    }
}

// Q64[q][i] = sum over the partials of columns 2q and 2q + 1 + beta V64[q][i]
__global__ void k_kmvm_reduce64(const double* __restrict__ part, int nparts, int nr, int nrhs2,
                                const double* __restrict__ V64, double beta, double* __restrict__ Q64,
                                double ksc) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int nrhs = nrhs2 / 2;
    if (e >= (long long)nr * nrhs) return;
    const int q = (int)(e / nr);
    const int i = (int)(e - (long long)q * nr);
    double s = 0.0;
    for (int sp = 0; sp < nparts; ++sp)
        s += part[((size_t)sp * nrhs2 + 2 * q) * nr + i] + part[((size_t)sp * nrhs2 + 2 * q + 1) * nr + i];
    Q64[(size_t)q * nr + i] = ksc * s + beta * V64[(size_t)q * nr + i];
}

int launch_split_hilo(krr_ctx* ctx, const double* a, long long n, int nrhs, float* out) {
    k_split_hilo<<<vec_blocks64(ctx, n * nrhs), V64T, 0, ctx->stream>>>(a, n, nrhs, out);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

int launch_kmvm_reduce64(krr_ctx* ctx, const double* part, int nparts, int nr, int nrhs2,
                         const double* V64, double beta, double* Q64, double ksc) {
    const long long tot = (long long)nr * (nrhs2 / 2);
    k_kmvm_reduce64<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(part, nparts, nr, nrhs2, V64, beta, Q64,
                                                                 ksc);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// ------------------------------------------------------------------ Woodbury apply, FP64 in/out
__device__ __forceinline__ void c64_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// (h, l) += f * r exactly up to the final float-float rounding
__device__ __forceinline__ void c64_acc(float& h, float& l, float f, float r) {
    const float p = __fmul_rn(f, r);
    const float pe = fmaf(f, r, -p);
    float s, e;
    c64_two_sum(h, p, s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, pe));
}

constexpr int G64_ROWS = 128;

// upart[blk][q][a] = sum_{i in chunk(blk)} F[i, a] r[q][i] with r split hi + lo, float-float
// sums; thread t owns the float4 columns 4t.. (stride 4 V64T).
template <int NQ>
__global__ void __launch_bounds__(V64T)
k_gemv_t64(const float* __restrict__ F, long long n, int ldF, const double* __restrict__ R,
           long long rows_per, double* __restrict__ upart) {
    __shared__ float sh[NQ][G64_ROWS], sl[NQ][G64_ROWS];
    const long long r0 = (long long)blockIdx.x * rows_per;
    const long long r1 = min(n, r0 + rows_per);
    const int ld4 = ldF >> 2;
    const float4* F4 = reinterpret_cast<const float4*>(F);
    for (int c0 = 0; c0 < ld4; c0 += V64T) {
        const int c4 = c0 + threadIdx.x;
        float h[NQ][4], l[NQ][4];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) h[q][w] = l[q][w] = 0.f;
        for (long long b0 = r0; b0 < r1; b0 += G64_ROWS) {
            const int nb = (int)min((long long)G64_ROWS, r1 - b0);
            __syncthreads();
            for (int e = threadIdx.x; e < NQ * G64_ROWS; e += V64T) {
                const int q = e / G64_ROWS, i = e - q * G64_ROWS;
                const double v = (i < nb) ? R[(size_t)q * n + b0 + i] : 0.0;
                const float hi = (float)v;
                sh[q][i] = hi;
                sl[q][i] = (float)(v - (double)hi);
            }
            __syncthreads();
            if (c4 < ld4) {
                const float4* fp = F4 + b0 * ld4 + c4;
                for (int i = 0; i < nb; ++i) {
                    const float4 f = fp[(size_t)i * ld4];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float a = sh[q][i], b = sl[q][i];
                        c64_acc(h[q][0], l[q][0], f.x, a); c64_acc(h[q][0], l[q][0], f.x, b);
                        c64_acc(h[q][1], l[q][1], f.y, a); c64_acc(h[q][1], l[q][1], f.y, b);
                        c64_acc(h[q][2], l[q][2], f.z, a); c64_acc(h[q][2], l[q][2], f.z, b);
                        c64_acc(h[q][3], l[q][3], f.w, a); c64_acc(h[q][3], l[q][3], f.w, b);
                    }
                }
            }
        }
        if (c4 < ld4) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                double* o = upart + ((size_t)blockIdx.x * NQ + q) * ldF + 4 * c4;
#pragma unroll
                for (int w = 0; w < 4; ++w) o[w] = (double)h[q][w] + (double)l[q][w];
            }
        }
    }
}

// z[q][i] = (r[q][i] - sum_a F[i, a] v[q][a]) / beta in FP64, the sum in float-float from
// v = v_hi + v_lo; one warp per row; optional per-block partial sums of r.z.
template <int NQ>
__global__ void __launch_bounds__(V64T)
k_gemv_n_apply64(const float* __restrict__ F, long long n, int k, int ldF, const double* __restrict__ v,
                 const double* __restrict__ R, double inv_beta, double* __restrict__ Z,
                 double* __restrict__ rz_part) {
    extern __shared__ float4 sv64[];   // [NQ][2][ld4]: hi then lo
    const int ld4 = ldF >> 2;
    for (int e = threadIdx.x; e < NQ * ld4; e += V64T) {
        const int q = e / ld4, c4 = e - q * ld4;
        float th[4], tl[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int a = 4 * c4 + w;
            const double x = (a < k) ? v[(size_t)q * k + a] : 0.0;
            th[w] = (float)x;
            tl[w] = (float)(x - (double)th[w]);
        }
        sv64[(2 * q) * ld4 + c4] = make_float4(th[0], th[1], th[2], th[3]);
        sv64[(2 * q + 1) * ld4 + c4] = make_float4(tl[0], tl[1], tl[2], tl[3]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float4* F4 = reinterpret_cast<const float4*>(F);
    double rz[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) rz[q] = 0.0;
    const long long wstride = (long long)gridDim.x * (V64T / 32);
    for (long long i = (long long)blockIdx.x * (V64T / 32) + w; i < n; i += wstride) {
        float h[NQ], l[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) h[q] = l[q] = 0.f;
        const float4* f0 = F4 + i * ld4;
        for (int c = lane; c < ld4; c += 32) {
            const float4 a = f0[c];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const float4 vh = sv64[(2 * q) * ld4 + c], vl = sv64[(2 * q + 1) * ld4 + c];
                c64_acc(h[q], l[q], a.x, vh.x); c64_acc(h[q], l[q], a.x, vl.x);
                c64_acc(h[q], l[q], a.y, vh.y); c64_acc(h[q], l[q], a.y, vl.y);
                c64_acc(h[q], l[q], a.z, vh.z); c64_acc(h[q], l[q], a.z, vl.z);
                c64_acc(h[q], l[q], a.w, vh.w); c64_acc(h[q], l[q], a.w, vl.w);
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double t = warp_sum((double)h[q] + (double)l[q]);
            if (lane == 0) {
                const double r = R[(size_t)q * n + i];
                const double z = (r - t) * inv_beta;
                Z[(size_t)q * n + i] = z;
                rz[q] += r * z;
            }
        }
    }
    if (rz_part) {
        __shared__ double red[V64T / 32];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const double s = warp_sum(lane == 0 ? rz[q] : 0.0);
            __syncthreads();
            if (lane == 0) red[w] = s;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int j = 0; j < V64T / 32; ++j) t += red[j];
                rz_part[(size_t)q * gridDim.x + blockIdx.x] = t;
            }
        }
    }
}

// defined in cg.cu
int launch_gemv_t_reduce(krr_ctx* ctx, const double* upart, int nblk, int nq, int k, int ldF, double* u);
int launch_tri_gemv(krr_ctx* ctx, const double* T, int k, const double* x, int nq, bool lower, double* y);

typedef void (*gt64_fn)(const float*, long long, int, const double*, long long, double*);
typedef void (*gn64_fn)(const float*, long long, int, int, const double*, const double*, double, double*,
                        double*);

// Z = M^{-1} R (FP64 in and out, n x nrhs RHS-major).  rz_part (optional) receives per-block
// partial sums of R.Z laid out [q][blk] with the vector block count of the CG kernels.
int launch_apply_precond64(krr_ctx* ctx, const double* R, int nrhs, double* Z, double* rz_part) {
    const long long n = ctx->n;
    const int k = ctx->k_eff, ldF = ctx->ldF;
    const int nb = vec_blocks64(ctx, n);
    const long long rows_per = ceil_div(n, nb);
    double *upart, *u, *u1, *v;
    KRR_RET(bufT(ctx, "ap_upart", (size_t)nb * 4 * ldF, &upart));
    KRR_RET(bufT(ctx, "ap_u", (size_t)4 * k, &u));
    KRR_RET(bufT(ctx, "ap_u1", (size_t)4 * k, &u1));
    KRR_RET(bufT(ctx, "ap_v", (size_t)4 * k, &v));
    for (int q0 = 0; q0 < nrhs; q0 += 4) {
        const int nq = std::min(4, nrhs - q0);
        gt64_fn gt = nq == 1 ? &k_gemv_t64<1> : nq == 2 ? &k_gemv_t64<2> : nq == 3 ? &k_gemv_t64<3>
                   : &k_gemv_t64<4>;
        gn64_fn gn = nq == 1 ? &k_gemv_n_apply64<1> : nq == 2 ? &k_gemv_n_apply64<2>
                   : nq == 3 ? &k_gemv_n_apply64<3> : &k_gemv_n_apply64<4>;
        const double* Rq = R + (size_t)q0 * n;
        double* Zq = Z + (size_t)q0 * n;
        gt<<<nb, V64T, 0, ctx->stream>>>(ctx->F, n, ldF, Rq, rows_per, upart);
        KRR_CHECK_LAUNCH();
        KRR_RET(launch_gemv_t_reduce(ctx, upart, nb, nq, k, ldF, u));
        KRR_RET(launch_tri_gemv(ctx, ctx->T2, k, u, nq, true, u1));
        KRR_RET(launch_tri_gemv(ctx, ctx->T2t, k, u1, nq, false, v));
        const size_t smem = sizeof(float4) * 2 * nq * (ldF / 4);
        if (smem > 48 * 1024) KRR_RET(allow_max_dynamic_smem(ctx, (const void*)gn));
        gn<<<nb, V64T, smem, ctx->stream>>>(ctx->F, n, k, ldF, v, Rq, 1.0 / ctx->beta, Zq,
                                            rz_part ? rz_part + (size_t)q0 * nb : nullptr);
        KRR_CHECK_LAUNCH();
    }
    return KRR_OK;
}

// ------------------------------------------------------------------ FP64 recurrences
__device__ __forceinline__ void block_sum_store64(double v, double* part, int q) {
    __shared__ double red[V64T / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < V64T / 32; ++i) s += red[i];
        part[(size_t)q * gridDim.x + blockIdx.x] = s;
    }
}

// x += a p; r -= a q; partial r.r
__global__ void __launch_bounds__(V64T)
k_cg_update_xr64(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                 const double* __restrict__ qv, long long n, int nrhs, const CGScalars* __restrict__ cg,
                 double* __restrict__ part) {
    for (int q = 0; q < nrhs; ++q) {
        const double a = cg->a[q];
        double s = 0.0;
        for (long long i = (long long)blockIdx.x * V64T + threadIdx.x; i < n; i += (long long)gridDim.x * V64T) {
            const long long e = q * n + i;
            const double rv = fma(-a, qv[e], r[e]);
            x[e] = fma(a, p[e], x[e]);
            r[e] = rv;
            s = fma(rv, rv, s);
        }
        block_sum_store64(s, part, q);
    }
}

// p = z + b p
__global__ void __launch_bounds__(V64T)
k_cg_update_p64(double* __restrict__ p, const double* __restrict__ z, long long n, int nrhs,
                const CGScalars* __restrict__ cg) {
    const long long tot = n * nrhs;
    for (long long e = (long long)blockIdx.x * V64T + threadIdx.x; e < tot; e += (long long)gridDim.x * V64T) {
        const int q = (int)(e / n);
        p[e] = fma(cg->b[q], p[e], z[e]);
    }
}

// y += x (FP64)
__global__ void k_add64(const double* __restrict__ x, double* __restrict__ y, long long tot) {
    for (long long e = (long long)blockIdx.x * V64T + threadIdx.x; e < tot; e += (long long)gridDim.x * V64T)
        y[e] += x[e];
}

// defined in cg.cu
int launch_cg_scalars_init(krr_ctx* ctx, const double* rz_part, const double* rr_part, int nb, int nrhs);
int launch_cg_scalars_alpha(krr_ctx* ctx, const double* part, int nb, int nrhs);
int launch_cg_scalars_check(krr_ctx* ctx, const double* part, int nb, int nrhs, double tol2);
int launch_cg_scalars_beta(krr_ctx* ctx, const double* rz_part, int nb, int nrhs);
int launch_dot64_parts(krr_ctx* ctx, const double* A, const double* B, long long n, int nrhs, int nb,
                       double* part);

int cg64_vec_blocks(krr_ctx* ctx) { return vec_blocks64(ctx, ctx->n); }

int launch_cg64_start(krr_ctx* ctx, const double* r, int nrhs, double* rz_part, double* rr_part) {
    const int nb = vec_blocks64(ctx, ctx->n);
    KRR_RET(launch_dot64_parts(ctx, r, r, ctx->n, nrhs, nb, rr_part));
    return launch_cg_scalars_init(ctx, rz_part, rr_part, nb, nrhs);
}

int launch_cg64_alpha(krr_ctx* ctx, const double* p, const double* q, int nrhs, double* part) {
    const int nb = vec_blocks64(ctx, ctx->n);
    KRR_RET(launch_dot64_parts(ctx, p, q, ctx->n, nrhs, nb, part));
    return launch_cg_scalars_alpha(ctx, part, nb, nrhs);
}

int launch_cg64_update_xr(krr_ctx* ctx, double* x, double* r, const double* p, const double* q, int nrhs,
                          double* part) {
    const int nb = vec_blocks64(ctx, ctx->n);
    k_cg_update_xr64<<<nb, V64T, 0, ctx->stream>>>(x, r, p, q, ctx->n, nrhs, ctx->cg, part);
    KRR_CHECK_LAUNCH();
    return launch_cg_scalars_check(ctx, part, nb, nrhs, 0.0);
}

int launch_cg64_beta_p(krr_ctx* ctx, double* p, const double* z, int nrhs, const double* rz_part) {
    const int nb = vec_blocks64(ctx, ctx->n);
    KRR_RET(launch_cg_scalars_beta(ctx, rz_part, nb, nrhs));
    k_cg_update_p64<<<nb, V64T, 0, ctx->stream>>>(p, z, ctx->n, nrhs, ctx->cg);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

int launch_add64(krr_ctx* ctx, const double* x, double* y, long long tot) {
    k_add64<<<vec_blocks64(ctx, tot), V64T, 0, ctx->stream>>>(x, y, tot);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

}  // namespace krr
