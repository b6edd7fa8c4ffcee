// Conjugate-gradient vector kernels (Algorithm 5 step 3) and the Woodbury
// application of the preconditioner (Algorithm 4, Eq. (7)).
//
// Vectors are FP32, RHS-major (column q of an n x nrhs block at q*n); every dot
// product is accumulated in FP64 and the CG scalars live in a small device struct,
// so the recurrences run without host round trips.  The preconditioner is
//     M^{-1} r = (r - F G^{-1} F^T r) / beta,   G = beta I + F^T F = L2 L2^T,
// with F = K(X, X_S) L1^{-T} stored (n x ldF) and T2 = L2^{-1} held explicitly,
// so one application is two streaming passes over F and two k x k triangular
// products in FP64.
#include "internal.cuh"

#include <algorithm>
#include <cstring>

namespace krr {

constexpr int VT = 256;   // threads of the streaming kernels

// Blocks of the streaming kernels: four per SM where n allows (the Woodbury GEMVs are
// latency bound with fewer loads in flight), at least 64 rows per block.
static int vec_blocks(krr_ctx* ctx, long long n) {
    return (int)std::max<long long>(1, std::min<long long>(4LL * ctx->num_sms, ceil_div(n, 64)));
}

// Block-wide FP64 sum into part[q * gridDim.x + blockIdx.x].
__device__ __forceinline__ void block_sum_store(double v, double* part, int q) {
    __shared__ double red[VT / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < VT / 32; ++i) s += red[i];
        part[(size_t)q * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(VT)
k_dot_part(const float* __restrict__ A, const float* __restrict__ B, long long n, int nrhs,
           double* __restrict__ part) {
    for (int q = 0; q < nrhs; ++q) {
        double s = 0.0;
        for (long long i = (long long)blockIdx.x * VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
            s += (double)A[q * n + i] * (double)B[q * n + i];
        block_sum_store(s, part, q);
    }
}

__global__ void __launch_bounds__(VT)
k_dot64_part(const double* __restrict__ A, const double* __restrict__ B, long long n, int nrhs,
             double* __restrict__ part) {
    for (int q = 0; q < nrhs; ++q) {
        double s = 0.0;
        for (long long i = (long long)blockIdx.x * VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT)
            s = fma(A[q * n + i], B[q * n + i], s);
        block_sum_store(s, part, q);
    }
}

__global__ void k_sum_parts(const double* __restrict__ part, int nblk, int nrhs, double* out) {
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (q >= nrhs) return;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[(size_t)q * nblk + b];
    s = warp_sum(s);
    if (lane == 0) out[q] = s;
}

int launch_dot(krr_ctx* ctx, const float* A, const float* B, long long n, int nrhs, double* out) {
    const int nb = vec_blocks(ctx, n);
    double* part;
    KRR_RET(bufT(ctx, "dot_part", (size_t)nb * nrhs, &part));
    k_dot_part<<<nb, VT, 0, ctx->stream>>>(A, B, n, nrhs, part);
    KRR_CHECK_LAUNCH();
    k_sum_parts<<<1, 32 * nrhs, 0, ctx->stream>>>(part, nb, nrhs, out);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

int launch_dot64(krr_ctx* ctx, const double* A, const double* B, long long n, int nrhs, double* out) {
    const int nb = vec_blocks(ctx, n);
    double* part;
    KRR_RET(bufT(ctx, "dot_part", (size_t)nb * nrhs, &part));
    k_dot64_part<<<nb, VT, 0, ctx->stream>>>(A, B, n, nrhs, part);
    KRR_CHECK_LAUNCH();
    k_sum_parts<<<1, 32 * nrhs, 0, ctx->stream>>>(part, nb, nrhs, out);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// ------------------------------------------------------------------ Woodbury apply
constexpr int GT_ROWS = 256;   // rows of R staged in shared memory per batch

// Error-free transformations (Knuth two-sum, FMA two-product) for compensated sums.
__device__ __forceinline__ void cg_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
__device__ __forceinline__ void ff_acc(float& h, float& l, float f, float r) {
    const float p = __fmul_rn(f, r);
    const float pe = fmaf(f, r, -p);
    float s, e;
    cg_two_sum(h, p, s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, pe));
}

// u_part[blk][q][a] = sum_{i in chunk(blk)} F[i, a] R[q, i], as FP64.  Thread t owns the
// float4 columns 4t.. (stride 4*VT), so one CTA streams whole rows of F with 16-byte
// loads.  Products are exact and the sums compensated (float-float): F^T r carries the
// cancellation of the preconditioner, and a plain FP32 sum costs PCG iterations.
template <int NQ>
__global__ void __launch_bounds__(VT)
k_gemv_t(const float* __restrict__ F, long long n, int ldF, const float* __restrict__ R,
         long long ldr, long long rows_per, double* __restrict__ upart) {
    __shared__ float sr[NQ][GT_ROWS];
    const long long r0 = (long long)blockIdx.x * rows_per;
    const long long r1 = min(n, r0 + rows_per);
    const int ld4 = ldF >> 2;
    const float4* F4 = reinterpret_cast<const float4*>(F);
    for (int c0 = 0; c0 < ld4; c0 += VT) {
        const int c4 = c0 + threadIdx.x;
        float hx[NQ], hy[NQ], hz[NQ], hw[NQ], lx[NQ], ly[NQ], lz[NQ], lw[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) hx[q] = hy[q] = hz[q] = hw[q] = lx[q] = ly[q] = lz[q] = lw[q] = 0.f;
        for (long long b0 = r0; b0 < r1; b0 += GT_ROWS) {
            const int nb = (int)min((long long)GT_ROWS, r1 - b0);
            __syncthreads();
            for (int e = threadIdx.x; e < NQ * GT_ROWS; e += VT) {
                const int q = e / GT_ROWS, i = e - q * GT_ROWS;
                sr[q][i] = (i < nb) ? R[q * ldr + b0 + i] : 0.f;
            }
            __syncthreads();
            if (c4 < ld4) {
                const float4* fp = F4 + b0 * ld4 + c4;
                constexpr int U = 8;   // rows whose loads are in flight together
                int i = 0;
                for (; i + U <= nb; i += U) {
                    float4 f[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) f[u] = fp[(size_t)(i + u) * ld4];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            const float a = sr[q][i + u];
                            ff_acc(hx[q], lx[q], f[u].x, a); ff_acc(hy[q], ly[q], f[u].y, a);
                            ff_acc(hz[q], lz[q], f[u].z, a); ff_acc(hw[q], lw[q], f[u].w, a);
                        }
                    }
                }
                for (; i < nb; ++i) {
                    const float4 f = fp[(size_t)i * ld4];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const float a = sr[q][i];
                        ff_acc(hx[q], lx[q], f.x, a); ff_acc(hy[q], ly[q], f.y, a);
                        ff_acc(hz[q], lz[q], f.z, a); ff_acc(hw[q], lw[q], f.w, a);
                    }
                }
            }
        }
        if (c4 < ld4) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                double* o = upart + ((size_t)blockIdx.x * NQ + q) * ldF + 4 * c4;
                o[0] = (double)hx[q] + (double)lx[q];
                o[1] = (double)hy[q] + (double)ly[q];
                o[2] = (double)hz[q] + (double)lz[q];
                o[3] = (double)hw[q] + (double)lw[q];
            }
        }
    }
}

// u[q][a] = sum_blk upart (FP64), a < k.  A CTA covers 8 columns with 32 groups of 8
// threads: each group sums every 32nd partial (8 consecutive columns = one 64-byte
// segment per load), and the groups combine through shared memory.  k / 8 CTAs keep
// enough loads in flight for the 4 x SMs partials of the F^T r pass.
__global__ void __launch_bounds__(256)
k_gemv_t_reduce(const double* __restrict__ upart, int nblk, int nq, int k, int ldF,
                double* __restrict__ u) {
    __shared__ double red[32][9];
    const int c = threadIdx.x & 7, g = threadIdx.x >> 3;
    const int a = blockIdx.x * 8 + c;
    const int q = blockIdx.y;
    double s = 0.0;
    if (a < k)
        for (int b = g; b < nblk; b += 32) s += upart[((size_t)b * nq + q) * ldF + a];
    red[g][c] = s;
    __syncthreads();
    if (threadIdx.x < 8 && a < k) {
        double t = 0.0;
#pragma unroll 8
        for (int i = 0; i < 32; ++i) t += red[i][c];
        u[(size_t)q * k + a] = t;
    }
}

// y[q][a] = sum_b T[a][b] x[q][b] over b <= a (lower) or b >= a (upper).  One 128-thread
// block per row a: every thread has at most a few independent loads of the row, so the
// k x k factor streams at memory rate instead of one dependent chain per warp.
constexpr int TG_T = 128;
__global__ void __launch_bounds__(TG_T) k_tri_gemv(const double* __restrict__ T, int k,
                                                   const double* __restrict__ x, int nq, bool lower,
                                                   double* __restrict__ y) {
    __shared__ double red[TG_T / 32];
    const int a = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b0 = lower ? 0 : a, b1 = lower ? a + 1 : k;
    for (int q = 0; q < nq; ++q) {
        double s = 0.0;
        for (int b = b0 + threadIdx.x; b < b1; b += TG_T) s = fma(T[(size_t)a * k + b], x[(size_t)q * k + b], s);
        s = warp_sum(s);
        __syncthreads();
        if (lane == 0) red[w] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
#pragma unroll
            for (int i = 0; i < TG_T / 32; ++i) t += red[i];
            y[(size_t)q * k + a] = t;
        }
    }
}

// Z[q][i] = (R[q][i] - sum_a F[i, a] v[q][a]) / beta; one warp per row with float4 loads.
// Optional per-block partial sums of R.Z.
template <int NQ>
__global__ void __launch_bounds__(VT)
k_gemv_n_apply(const float* __restrict__ F, long long n, int k, int ldF, const double* __restrict__ v,
               const float* __restrict__ R, long long ldr, float inv_beta, float* __restrict__ Z,
               double* __restrict__ rz_part) {
    extern __shared__ float4 sv4[];   // NQ x ld4
    const int ld4 = ldF >> 2;
    for (int e = threadIdx.x; e < NQ * ld4; e += VT) {
        const int q = e / ld4, c4 = e - q * ld4;
        float t[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int a = 4 * c4 + w;
            t[w] = (a < k) ? (float)v[(size_t)q * k + a] : 0.f;
        }
        sv4[e] = make_float4(t[0], t[1], t[2], t[3]);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float4* F4 = reinterpret_cast<const float4*>(F);
    double rz[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) rz[q] = 0.0;
    // each warp takes two rows at a time and issues all of their loads before the FMAs
    const long long wstride = (long long)gridDim.x * (VT / 32);
    for (long long i0 = (long long)blockIdx.x * (VT / 32) + w; i0 < n; i0 += 2 * wstride) {
        const long long i1 = i0 + wstride;
        const bool has1 = i1 < n;
        float s0[NQ], s1[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) s0[q] = s1[q] = 0.f;
        const float4* f0 = F4 + i0 * ld4;
        const float4* f1 = F4 + (has1 ? i1 : i0) * ld4;
        for (int c0 = lane; c0 < ld4; c0 += 32 * 4) {
            float4 a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + 32 * u;
                a[u] = c < ld4 ? f0[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                b[u] = (c < ld4 && has1) ? f1[c] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + 32 * u;
                if (c >= ld4) break;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 vv = sv4[q * ld4 + c];
                    s0[q] = fmaf(a[u].x, vv.x, fmaf(a[u].y, vv.y, fmaf(a[u].z, vv.z, fmaf(a[u].w, vv.w, s0[q]))));
                    s1[q] = fmaf(b[u].x, vv.x, fmaf(b[u].y, vv.y, fmaf(b[u].z, vv.z, fmaf(b[u].w, vv.w, s1[q]))));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float t0 = warp_sum(s0[q]);
            const float t1 = warp_sum(s1[q]);
            if (lane == 0) {
                const float r0 = R[q * ldr + i0];
                const float z0 = (r0 - t0) * inv_beta;
                Z[q * ldr + i0] = z0;
                rz[q] += (double)r0 * (double)z0;
                if (has1) {
                    const float r1 = R[q * ldr + i1];
                    const float z1 = (r1 - t1) * inv_beta;
                    Z[q * ldr + i1] = z1;
                    rz[q] += (double)r1 * (double)z1;
                }
            }
        }
    }
    if (rz_part) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) block_sum_store(lane == 0 ? rz[q] : 0.0, rz_part, q);
    }
}

typedef void (*gemv_t_fn)(const float*, long long, int, const float*, long long, long long, double*);
typedef void (*gemv_n_fn)(const float*, long long, int, int, const double*, const float*, long long,
                          float, float*, double*);

// Z = M^{-1} R for nrhs columns.  When rz_part is non-null it receives per-block partial
// sums of R.Z laid out [q][blk] with vec_blocks(n) blocks per column.
int launch_apply_precond(krr_ctx* ctx, const float* R, int nrhs, float* Z, double* rz_part) {
    const long long n = ctx->n;
    const int k = ctx->k_eff, ldF = ctx->ldF;
    const int nb = vec_blocks(ctx, n);
    const long long rows_per = ceil_div(n, nb);
    double *upart, *u, *u1, *v;
    KRR_RET(bufT(ctx, "ap_upart", (size_t)nb * 4 * ldF, &upart));
    KRR_RET(bufT(ctx, "ap_u", (size_t)4 * k, &u));
    KRR_RET(bufT(ctx, "ap_u1", (size_t)4 * k, &u1));
    KRR_RET(bufT(ctx, "ap_v", (size_t)4 * k, &v));
    const float inv_beta = (float)(1.0 / ctx->beta);
    for (int q0 = 0; q0 < nrhs; q0 += 4) {
        const int nq = std::min(4, nrhs - q0);
        gemv_t_fn gt = nq == 1 ? &k_gemv_t<1> : nq == 2 ? &k_gemv_t<2> : nq == 3 ? &k_gemv_t<3> : &k_gemv_t<4>;
        gemv_n_fn gn = nq == 1 ? &k_gemv_n_apply<1> : nq == 2 ? &k_gemv_n_apply<2>
                     : nq == 3 ? &k_gemv_n_apply<3> : &k_gemv_n_apply<4>;
        const float* Rq = R + (size_t)q0 * n;
        float* Zq = Z + (size_t)q0 * n;
        gt<<<nb, VT, 0, ctx->stream>>>(ctx->F, n, ldF, Rq, n, rows_per, upart);
        KRR_CHECK_LAUNCH();
        k_gemv_t_reduce<<<dim3(ceil_div(k, 8), nq), 256, 0, ctx->stream>>>(upart, nb, nq, k, ldF, u);
        KRR_CHECK_LAUNCH();
        k_tri_gemv<<<k, TG_T, 0, ctx->stream>>>(ctx->T2, k, u, nq, true, u1);
        KRR_CHECK_LAUNCH();
        k_tri_gemv<<<k, TG_T, 0, ctx->stream>>>(ctx->T2t, k, u1, nq, false, v);
        KRR_CHECK_LAUNCH();
        const size_t smem = sizeof(float4) * nq * (ldF / 4);
        if (smem > 48 * 1024) {
            KRR_RET(allow_max_dynamic_smem(ctx, (const void*)gn));
        }
        gn<<<nb, VT, smem, ctx->stream>>>(ctx->F, n, k, ldF, v, Rq, n, inv_beta, Zq,
                                          rz_part ? rz_part + (size_t)q0 * nb : nullptr);
        KRR_CHECK_LAUNCH();
    }
    return KRR_OK;
}

// ------------------------------------------------------------------ PCG recurrences
// The scalar kernels run one warp per right-hand side: the warp sums that column's
// per-block partials (FP64) and lane 0 applies the recurrence.
__device__ __forceinline__ double warp_sum_parts(const double* __restrict__ part, int nblk, int q) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[(size_t)q * nblk + b];
    return warp_sum(s);
}

// a_q = rz_q / (p_q . q_q) for active columns; zero otherwise.
__global__ void k_cg_alpha(CGScalars* cg, const double* __restrict__ part, int nblk, int nrhs) {
    const int q = threadIdx.x >> 5;
    if (q >= nrhs) return;
    const double s = warp_sum_parts(part, nblk, q);
    if ((threadIdx.x & 31) != 0) return;
    cg->pq[q] = s;
    double a = 0.0;
    if (cg->active[q]) {
        if (!(s > 0.0) || !isfinite(s) || !isfinite(cg->rz[q])) {
            cg->bad = 1;
            cg->active[q] = 0;
        } else {
            a = cg->rz[q] / s;
        }
    }
    cg->a[q] = a;
}

// x += a p; r -= a q; partial r.r
__global__ void __launch_bounds__(VT)
k_cg_update_xr(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ p,
               const float* __restrict__ qv, long long n, int nrhs, const CGScalars* __restrict__ cg,
               double* __restrict__ part) {
    for (int q = 0; q < nrhs; ++q) {
        const float a = (float)cg->a[q];
        double s = 0.0;
        for (long long i = (long long)blockIdx.x * VT + threadIdx.x; i < n; i += (long long)gridDim.x * VT) {
            const long long e = q * n + i;
            const float rv = fmaf(-a, qv[e], r[e]);
            x[e] = fmaf(a, p[e], x[e]);
            r[e] = rv;
            s += (double)rv * (double)rv;
        }
        block_sum_store(s, part, q);
    }
}

// rr_q = sum part (recursive residual); columns with tol2 > 0 stop once rr_q <= tol2 rr0_q.
__global__ void k_cg_check(CGScalars* cg, const double* __restrict__ part, int nblk, int nrhs,
                           double tol2) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const int q = threadIdx.x >> 5;
    if (q < nrhs) {
        const double s = warp_sum_parts(part, nblk, q);
        if ((threadIdx.x & 31) == 0) {
            cg->rr[q] = s;
            if (!isfinite(s)) {
                cg->bad = 1;
                cg->active[q] = 0;
            }
            if (tol2 > 0.0 && cg->active[q] && !(s > tol2 * cg->rr0[q])) cg->active[q] = 0;
            if (cg->active[q]) atomicOr(&any, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) cg->all_done = any ? 0 : 1;
}

// b_q = rz_new / rz; rz = rz_new (b = 0 for finished columns: p restarts from z)
__global__ void k_cg_beta(CGScalars* cg, const double* __restrict__ part, int nblk, int nrhs) {
    const int q = threadIdx.x >> 5;
    if (q >= nrhs) return;
    const double s = warp_sum_parts(part, nblk, q);
    if ((threadIdx.x & 31) != 0) return;
    const double rz = cg->rz[q];
    cg->b[q] = (cg->active[q] && rz != 0.0 && isfinite(s)) ? s / rz : 0.0;
    cg->rz[q] = s;
}

// p = z + b p
__global__ void __launch_bounds__(VT)
k_cg_update_p(float* __restrict__ p, const float* __restrict__ z, long long n, int nrhs,
              const CGScalars* __restrict__ cg) {
    const long long tot = n * nrhs;
    for (long long e = (long long)blockIdx.x * VT + threadIdx.x; e < tot; e += (long long)gridDim.x * VT) {
        const int q = (int)(e / n);
        p[e] = fmaf((float)cg->b[q], p[e], z[e]);
    }
}

// start: rz = part sum (r.z), rr0 = r.r given in rr0_part, active = rr0 > 0
__global__ void k_cg_init(CGScalars* cg, const double* __restrict__ rz_part,
                          const double* __restrict__ rr_part, int nblk, int nrhs) {
    const int q = threadIdx.x;
    if (threadIdx.x == 0) {
        cg->all_done = 0;
        cg->bad = 0;
    }
    if (q >= nrhs) return;
    double s = 0.0, t = 0.0;
    for (int b = 0; b < nblk; ++b) {
        s += rz_part[(size_t)q * nblk + b];
        t += rr_part[(size_t)q * nblk + b];
    }
    cg->rz[q] = s;
    cg->rr0[q] = t;
    cg->rr[q] = t;
    cg->active[q] = (t > 0.0 && isfinite(t) && isfinite(s)) ? 1 : 0;
    cg->a[q] = 0.0;
    cg->b[q] = 0.0;
}

// out32 = (float) in64 ; and alpha64 += x32
__global__ void k_f64_to_f32(const double* __restrict__ a, float* __restrict__ b, long long tot) {
    for (long long e = (long long)blockIdx.x * VT + threadIdx.x; e < tot; e += (long long)gridDim.x * VT)
        b[e] = (float)a[e];
}
__global__ void k_f32_to_f64(const float* __restrict__ a, double* __restrict__ b, long long tot) {
    for (long long e = (long long)blockIdx.x * VT + threadIdx.x; e < tot; e += (long long)gridDim.x * VT)
        b[e] = (double)a[e];
}
__global__ void k_axpy_f32_into_f64(const float* __restrict__ x, double* __restrict__ y, long long tot) {
    for (long long e = (long long)blockIdx.x * VT + threadIdx.x; e < tot; e += (long long)gridDim.x * VT)
        y[e] += (double)x[e];
}

// ---- host drivers for the recurrences (launch sequences; no host sync inside)
int launch_cg_set_active(krr_ctx* ctx, const int* act_host, int nrhs) {
    // staged through the pinned mirror so the copy is asynchronous
    std::memcpy(ctx->cg_host->active, act_host, sizeof(int) * nrhs);
    KRR_TRY_CUDA(cudaMemcpyAsync(ctx->cg->active, ctx->cg_host->active, sizeof(int) * nrhs,
                                 cudaMemcpyHostToDevice, ctx->stream));
    return KRR_OK;
}

int cg_vec_blocks(krr_ctx* ctx) { return vec_blocks(ctx, ctx->n); }

int launch_cg_start(krr_ctx* ctx, const float* r, const float* z, int nrhs, double* rz_part,
                    double* rr_part) {
    const int nb = vec_blocks(ctx, ctx->n);
    k_dot_part<<<nb, VT, 0, ctx->stream>>>(r, r, ctx->n, nrhs, rr_part);
    KRR_CHECK_LAUNCH();
    k_cg_init<<<1, 32, 0, ctx->stream>>>(ctx->cg, rz_part, rr_part, nb, nrhs);
    KRR_CHECK_LAUNCH();
    (void)z;
    return KRR_OK;
}

int launch_cg_alpha(krr_ctx* ctx, const float* p, const float* q, int nrhs, double* part) {
    const int nb = vec_blocks(ctx, ctx->n);
    k_dot_part<<<nb, VT, 0, ctx->stream>>>(p, q, ctx->n, nrhs, part);
    KRR_CHECK_LAUNCH();
    k_cg_alpha<<<1, 32 * nrhs, 0, ctx->stream>>>(ctx->cg, part, nb, nrhs);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

int launch_cg_update_xr(krr_ctx* ctx, float* x, float* r, const float* p, const float* q, int nrhs,
                        double* part, double tol2) {
    const int nb = vec_blocks(ctx, ctx->n);
    k_cg_update_xr<<<nb, VT, 0, ctx->stream>>>(x, r, p, q, ctx->n, nrhs, ctx->cg, part);
    KRR_CHECK_LAUNCH();
    k_cg_check<<<1, 32 * nrhs, 0, ctx->stream>>>(ctx->cg, part, nb, nrhs, tol2);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

int launch_cg_beta_p(krr_ctx* ctx, float* p, const float* z, int nrhs, const double* rz_part) {
    const int nb = vec_blocks(ctx, ctx->n);
    k_cg_beta<<<1, 32 * nrhs, 0, ctx->stream>>>(ctx->cg, rz_part, nb, nrhs);
    KRR_CHECK_LAUNCH();
    k_cg_update_p<<<nb, VT, 0, ctx->stream>>>(p, z, ctx->n, nrhs, ctx->cg);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// The identity in place of the preconditioner (plain CG): Z = R and per-block partial
// sums of R.R in the layout of launch_apply_precond's rz_part.
int launch_identity_apply(krr_ctx* ctx, const float* R, int nrhs, float* Z, double* rz_part) {
    const long long n = ctx->n;
    if (Z != R)
        KRR_TRY_CUDA(cudaMemcpyAsync(Z, R, sizeof(float) * n * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
    if (rz_part) {
        k_dot_part<<<vec_blocks(ctx, n), VT, 0, ctx->stream>>>(R, R, n, nrhs, rz_part);
        KRR_CHECK_LAUNCH();
    }
    return KRR_OK;
}
int launch_identity_apply64(krr_ctx* ctx, const double* R, int nrhs, double* Z, double* rz_part) {
    const long long n = ctx->n;
    if (Z != R)
        KRR_TRY_CUDA(cudaMemcpyAsync(Z, R, sizeof(double) * n * nrhs, cudaMemcpyDeviceToDevice, ctx->stream));
    if (rz_part) {
        k_dot64_part<<<vec_blocks(ctx, n), VT, 0, ctx->stream>>>(R, R, n, nrhs, rz_part);
        KRR_CHECK_LAUNCH();
    }
    return KRR_OK;
}

// pieces used by the FP64 recurrence (cg64.cu)
int launch_gemv_t_reduce(krr_ctx* ctx, const double* upart, int nblk, int nq, int k, int ldF, double* u) {
    k_gemv_t_reduce<<<dim3(ceil_div(k, 8), nq), 256, 0, ctx->stream>>>(upart, nblk, nq, k, ldF, u);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}
int launch_tri_gemv(krr_ctx* ctx, const double* T, int k, const double* x, int nq, bool lower, double* y) {
    k_tri_gemv<<<k, TG_T, 0, ctx->stream>>>(T, k, x, nq, lower, y);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}
int launch_dot64_parts(krr_ctx* ctx, const double* A, const double* B, long long n, int nrhs, int nb,
                       double* part) {
    k_dot64_part<<<nb, VT, 0, ctx->stream>>>(A, B, n, nrhs, part);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}
int launch_cg_scalars_init(krr_ctx* ctx, const double* rz_part, const double* rr_part, int nb, int nrhs) {
    k_cg_init<<<1, 32, 0, ctx->stream>>>(ctx->cg, rz_part, rr_part, nb, nrhs);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}
int launch_cg_scalars_alpha(krr_ctx* ctx, const double* part, int nb, int nrhs) {
    k_cg_alpha<<<1, 32 * nrhs, 0, ctx->stream>>>(ctx->cg, part, nb, nrhs);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}
int launch_cg_scalars_check(krr_ctx* ctx, const double* part, int nb, int nrhs, double tol2) {
    k_cg_check<<<1, 32 * nrhs, 0, ctx->stream>>>(ctx->cg, part, nb, nrhs, tol2);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}
int launch_cg_scalars_beta(krr_ctx* ctx, const double* rz_part, int nb, int nrhs) {
    k_cg_beta<<<1, 32 * nrhs, 0, ctx->stream>>>(ctx->cg, rz_part, nb, nrhs);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

int launch_convert(krr_ctx* ctx, const double* a, float* b, long long tot) {
    k_f64_to_f32<<<vec_blocks(ctx, tot), VT, 0, ctx->stream>>>(a, b, tot);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}
int launch_convert_up(krr_ctx* ctx, const float* a, double* b, long long tot) {
    k_f32_to_f64<<<vec_blocks(ctx, tot), VT, 0, ctx->stream>>>(a, b, tot);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}
int launch_accumulate(krr_ctx* ctx, const float* x, double* y, long long tot) {
    k_axpy_f32_into_f64<<<vec_blocks(ctx, tot), VT, 0, ctx->stream>>>(x, y, tot);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

}  // namespace krr
