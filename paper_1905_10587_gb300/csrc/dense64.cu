// FP64 k x k linear algebra of the preconditioner build (Algorithm 3, Eq. (10)):
// the anchor kernel block K_SS, blocked right-looking Cholesky, triangular
// inversion by blocked forward substitution, and small helpers.  All matrices are
// row-major k x k.  k is at most a few thousand, so these run a few hundred
// small launches; GB300's FP64 rate, not memory, bounds them.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace krr {

constexpr int NB = 32;

__global__ void k_kss(const float* __restrict__ XS, int k, int d, double inv2s2,
                      double* __restrict__ A) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (b >= k) return;
    double d2 = 0.0;
    for (int c = 0; c < d; ++c) {
        const double df = (double)XS[(size_t)a * d + c] - (double)XS[(size_t)b * d + c];
        d2 = fma(df, df, d2);
    }
    A[(size_t)a * k + b] = exp(-d2 * inv2s2);
}

int launch_kss(krr_ctx* ctx, const float* XS, int k, int d, double sigma, double* A) {
    dim3 grid(ceil_div(k, 128), k);
    k_kss<<<grid, 128, 0, ctx->stream>>>(XS, k, d, 1.0 / (2.0 * sigma * sigma), A);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// ---- unblocked Cholesky of the nb x nb diagonal block at (j0, j0); one CTA of NB x NB threads.
__global__ void __launch_bounds__(NB * NB)
k_potf2(double* __restrict__ A, int k, int j0, int nb, double tau, int* __restrict__ info) {
    __shared__ double s[NB][NB + 1];
    const int r = threadIdx.y, c = threadIdx.x;
    s[r][c] = (r < nb && c < nb) ? A[(size_t)(j0 + r) * k + j0 + c] : 0.0;
    __syncthreads();
    for (int m = 0; m < nb; ++m) {
        const double piv = s[m][m];
        const bool bad = !(piv > tau) || !isfinite(piv);
        if (bad) {
            if (r == 0 && c == 0) atomicCAS(info, 0, j0 + m + 1);
            return;   // uniform: every thread sees the same s[m][m]
        }
        const double dm = sqrt(piv);
        __syncthreads();
        if (c == m && r >= m) s[r][m] = (r == m) ? dm : s[r][m] / dm;
        __syncthreads();
        if (r > m && c > m && c <= r) s[r][c] -= s[r][m] * s[c][m];
        __syncthreads();
    }
    if (r < nb && c < nb) A[(size_t)(j0 + r) * k + j0 + c] = (c <= r) ? s[r][c] : 0.0;
}

// ---- panel solve: rows i >= j0+nb, A[i, j0:j0+nb] <- A[i, j0:j0+nb] L_jj^{-T}
__global__ void __launch_bounds__(128)
k_potrf_panel(double* __restrict__ A, int k, int j0, int nb) {
    __shared__ double L[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e - r * NB;
        L[r][c] = (r < nb && c < nb) ? A[(size_t)(j0 + r) * k + j0 + c] : 0.0;
    }
    __syncthreads();
    const int i = j0 + nb + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    double x[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) x[c] = (c < nb) ? A[(size_t)i * k + j0 + c] : 0.0;
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        if (c < nb) {
            double v = x[c];
#pragma unroll
            for (int m = 0; m < c; ++m) v -= x[m] * L[c][m];
            x[c] = v / L[c][c];
        }
    }
#pragma unroll
    for (int c = 0; c < NB; ++c)
        if (c < nb) A[(size_t)i * k + j0 + c] = x[c];
}

// ---- trailing update: A[i, j] -= sum_m A[i, j0+m] A[j, j0+m]  for blocks (bi >= bj) past j0+nb
__global__ void __launch_bounds__(256)
k_potrf_update(double* __restrict__ A, int k, int j0, int nb, int t0) {
    // blockIdx.x enumerates lower-triangular block pairs of the trailing matrix
    int p = blockIdx.x, bi = 0;
    while ((bi + 1) * (bi + 2) / 2 <= p) ++bi;
    const int bj = p - bi * (bi + 1) / 2;
    const int r0 = t0 + bi * NB, c0 = t0 + bj * NB;
    __shared__ double sa[NB][NB + 1];
    __shared__ double sb[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, m = e - r * NB;
        sa[r][m] = (r0 + r < k && m < nb) ? A[(size_t)(r0 + r) * k + j0 + m] : 0.0;
        sb[r][m] = (c0 + r < k && m < nb) ? A[(size_t)(c0 + r) * k + j0 + m] : 0.0;
    }
    __syncthreads();
    const int c = threadIdx.x & 31, rq = threadIdx.x >> 5;   // 8 row groups of 4
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
        const int r = rq * 4 + rr;
        const int gi = r0 + r, gj = c0 + c;
        if (gi >= k || gj >= k || gj > gi) continue;
        double s = 0.0;
#pragma unroll 8
        for (int m = 0; m < NB; ++m) s = fma(sa[r][m], sb[c][m], s);
        A[(size_t)gi * k + gj] -= s;
    }
}

__global__ void k_zero_upper(double* A, int k) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)k * k) return;
    const int r = (int)(e / k), c = (int)(e - (long long)r * k);
    if (c > r) A[e] = 0.0;
}

int launch_potrf(krr_ctx* ctx, double* A, int k, int* info_host, double tau) {
    int* info;
    KRR_RET(bufT(ctx, "potrf_info", 1, &info));
    KRR_TRY_CUDA(cudaMemsetAsync(info, 0, sizeof(int), ctx->stream));
    for (int j0 = 0; j0 < k; j0 += NB) {
        const int nb = std::min(NB, k - j0);
        k_potf2<<<1, dim3(NB, NB), 0, ctx->stream>>>(A, k, j0, nb, tau, info);
        KRR_CHECK_LAUNCH();
        const int rest = k - j0 - nb;
        if (rest <= 0) break;
        k_potrf_panel<<<ceil_div(rest, 128), 128, 0, ctx->stream>>>(A, k, j0, nb);
        KRR_CHECK_LAUNCH();
        const int tb = (rest + NB - 1) / NB;
        k_potrf_update<<<tb * (tb + 1) / 2, 256, 0, ctx->stream>>>(A, k, j0, nb, j0 + nb);
        KRR_CHECK_LAUNCH();
    }
    k_zero_upper<<<ceil_div((long long)k * k, 256), 256, 0, ctx->stream>>>(A, k);
    KRR_CHECK_LAUNCH();
    KRR_TRY_CUDA(cudaMemcpyAsync(info_host, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    return KRR_OK;
}

// ---- solve L X = B in place, right-looking by 32-row blocks.  B = I gives X = L^{-1}
// (lower triangular), so only columns < j0 + nb carry nonzeros at step j0.
__global__ void __launch_bounds__(128)
k_trsm_diag(const double* __restrict__ L, double* __restrict__ B, int k, int j0, int nb,
            int ncols) {
    __shared__ double sl[NB][NB + 1];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, c = e - r * NB;
        sl[r][c] = (r < nb && c < nb) ? L[(size_t)(j0 + r) * k + j0 + c] : 0.0;
    }
    __syncthreads();
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= ncols) return;
    double x[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) x[r] = (r < nb) ? B[(size_t)(j0 + r) * k + col] : 0.0;
#pragma unroll
    for (int r = 0; r < NB; ++r) {
        if (r < nb) {
            double v = x[r];
#pragma unroll
            for (int m = 0; m < r; ++m) v -= sl[r][m] * x[m];
            x[r] = v / sl[r][r];
        }
    }
#pragma unroll
    for (int r = 0; r < NB; ++r)
        if (r < nb) B[(size_t)(j0 + r) * k + col] = x[r];
}

// B[i, c] -= sum_m L[i, j0+m] B[j0+m, c]  for i >= j0+nb, c < ncols.  CTA: 32 rows x 64 cols.
__global__ void __launch_bounds__(256)
k_trsm_update(const double* __restrict__ L, double* __restrict__ B, int k, int j0, int nb,
              int ncols) {
    __shared__ double sl[NB][NB + 1];
    __shared__ double sx[NB][64 + 1];
    const int r0 = j0 + nb + blockIdx.y * NB;
    const int c0 = blockIdx.x * 64;
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e / NB, m = e - r * NB;
        sl[r][m] = (r0 + r < k && m < nb) ? L[(size_t)(r0 + r) * k + j0 + m] : 0.0;
    }
    for (int e = threadIdx.x; e < NB * 64; e += blockDim.x) {
        const int m = e / 64, c = e - m * 64;
        sx[m][c] = (m < nb && c0 + c < ncols) ? B[(size_t)(j0 + m) * k + c0 + c] : 0.0;
    }
    __syncthreads();
    const int c = threadIdx.x & 63, rq = threadIdx.x >> 6;   // 4 groups of 8 rows
    if (c0 + c >= ncols) return;
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
        const int r = rq * 8 + rr;
        if (r0 + r >= k) break;
        double s = 0.0;
#pragma unroll 8
        for (int m = 0; m < NB; ++m) s = fma(sl[r][m], sx[m][c], s);
        B[(size_t)(r0 + r) * k + c0 + c] -= s;
    }
}

int launch_trsm_lower(krr_ctx* ctx, const double* L, double* B, int k) {
    for (int j0 = 0; j0 < k; j0 += NB) {
        const int nb = std::min(NB, k - j0);
        const int ncols = j0 + nb;   // B = I: columns >= j0+nb are still zero in these rows
        k_trsm_diag<<<ceil_div(ncols, 128), 128, 0, ctx->stream>>>(L, B, k, j0, nb, ncols);
        KRR_CHECK_LAUNCH();
        const int rest = k - j0 - nb;
        if (rest <= 0) break;
        dim3 grid(ceil_div(ncols, 64), ceil_div(rest, NB));
        k_trsm_update<<<grid, 256, 0, ctx->stream>>>(L, B, k, j0, nb, ncols);
        KRR_CHECK_LAUNCH();
    }
    return KRR_OK;
}

__global__ void k_set_identity(double* A, int k) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)k * k) return;
    const int r = (int)(e / k), c = (int)(e - (long long)r * k);
    A[e] = (r == c) ? 1.0 : 0.0;
}

int launch_set_identity(krr_ctx* ctx, double* A, int k) {
    k_set_identity<<<ceil_div((long long)k * k, 256), 256, 0, ctx->stream>>>(A, k);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

__global__ void k_add_diag(double* A, int k, double v) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a < k) A[(size_t)a * k + a] += v;
}

int launch_add_diag(krr_ctx* ctx, double* A, int k, double v) {
    k_add_diag<<<ceil_div(k, 256), 256, 0, ctx->stream>>>(A, k, v);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

__global__ void k_transpose64(const double* __restrict__ A, double* __restrict__ At, int k) {
    __shared__ double t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int gr = by + r, gc = bx + threadIdx.x;
        t[r][threadIdx.x] = (gr < k && gc < k) ? A[(size_t)gr * k + gc] : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int gr = bx + r, gc = by + threadIdx.x;
        if (gr < k && gc < k) At[(size_t)gr * k + gc] = t[threadIdx.x][r];
    }
}

int launch_transpose64(krr_ctx* ctx, const double* A, double* At, int k) {
    dim3 grid(ceil_div(k, 32), ceil_div(k, 32));
    k_transpose64<<<grid, dim3(32, 8), 0, ctx->stream>>>(A, At, k);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// Out[a * ldo + b] = (float) A[b * k + a]   (zero for b >= k up to ldo)
__global__ void k_to_float_t(const double* __restrict__ A, int k, float* __restrict__ Out, int ldo) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)k * ldo) return;
    const int a = (int)(e / ldo), b = (int)(e - (long long)a * ldo);
    Out[e] = (b < k) ? (float)A[(size_t)b * k + a] : 0.f;
}

int launch_to_float_transposed(krr_ctx* ctx, const double* A, int k, float* Out, int ldo) {
    k_to_float_t<<<ceil_div((long long)k * ldo, 256), 256, 0, ctx->stream>>>(A, k, Out, ldo);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

}  // namespace krr
