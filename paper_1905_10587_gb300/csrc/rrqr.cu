// Strong rank-revealing QR (Gu and Eisenstat, 1996) on the GPU: the factorization the
// interpolative-decomposition bound of Section 2.3 (Eq. (4)) assumes, where Algorithm 1 and
// Section 3's remarks use plain pivoted QR.
//
// After k pivots with the rows of R kept (Rout, k x n), the factorization is a strong RRQR
// with bound f when every entry of R11^{-1} R12 and every ratio gamma_j / omega_i stay within
// f in the combined measure
//     rho_ij = (R11^{-1} R12)_ij^2 + gamma_j^2 ||row i of R11^{-1}||^2 <= f^2
// (gamma_j: residual norm of column j after the k pivots, 1 / omega_i: norm of row i of
// R11^{-1}).  A pair breaking it is swapped and the pivoted QR recomputed with the new pivot
// list; every such swap raises |det R11| by more than f, so the loop ends.  The measure is one
// fused pass: T = R11^{-1} R12 in 64 x 64 tiles (FP32 FMA from shared memory) with the block's
// largest rho and its position.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace krr {

int qrcp_core(krr_ctx* ctx, float* Y, long long n, int l, int ldy, int k, int* piv, float* rdiag,
              const int* forced, float* Rout, double** nrm_out);
int launch_set_identity(krr_ctx* ctx, double* A, int k);
int launch_trsm_lower(krr_ctx* ctx, const double* L, double* B, int k);
int launch_transpose64(krr_ctx* ctx, const double* A, double* At, int k);

// R11[a][b] = R_a,piv[b] (upper triangular, FP64, row-major)
__global__ void k_gather_r11(const float* __restrict__ Rout, long long n, const int* __restrict__ piv, int k,
                             double* __restrict__ R11) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)k * k) return;
    const int a = (int)(e / k), b = (int)(e - (long long)a * k);
    R11[e] = b >= a ? (double)Rout[(size_t)a * n + piv[b]] : 0.0;
}

// W32 = R11^{-1} in FP32 from Linv = (R11^T)^{-1} (W[i][b] = Linv[b][i]); wn[i] = ||row i of W||^2
__global__ void k_rrqr_w(const double* __restrict__ Linv, int k, float* __restrict__ W32, double* __restrict__ wn) {
    __shared__ double red[8];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < k; b += blockDim.x) {
        const double w = Linv[(size_t)b * k + i];
        W32[(size_t)i * k + b] = (float)w;
        s = fma(w, w, s);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        wn[i] = t;
    }
}

constexpr int RT = 64, RK = 16;

// rho over a 64 x 64 tile of (pivot position i, column j); columns already chosen (nrm < 0)
// are skipped; writes the block's largest rho and its (i, j).
__global__ void __launch_bounds__(256)
k_rrqr_rho(const float* __restrict__ W32, int k, const float* __restrict__ Rout, long long n,
           const double* __restrict__ nrm, const double* __restrict__ wn, float* __restrict__ bval,
           int* __restrict__ bi, int* __restrict__ bj) {
    __shared__ float As[RK][RT + 4], Bs[RK][RT + 4];
    __shared__ float rv[256];
    __shared__ int ri[256], rj[256];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * RT;
    const long long j0 = (long long)blockIdx.x * RT;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int m0 = 0; m0 < k; m0 += RK) {
        for (int e = threadIdx.x; e < RK * RT; e += 256) {
            const int mm = e / RT, c = e - mm * RT;
            As[mm][c] = (i0 + c < k && m0 + mm < k) ? W32[(size_t)(i0 + c) * k + m0 + mm] : 0.f;
            Bs[mm][c] = (m0 + mm < k && j0 + c < n) ? Rout[(size_t)(m0 + mm) * n + j0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int mm = 0; mm < RK; ++mm) {
            float av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[mm][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[mm][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
    float best = -1.f;
    int besti = -1, bestj = -1;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = i0 + ty * 4 + a;
            const long long j = j0 + tx * 4 + b;
            if (i >= k || j >= n) continue;
            const double g2 = nrm[j];
            if (g2 < 0.0) continue;
            const float rho = (float)((double)acc[a][b] * acc[a][b] + g2 * wn[i]);
            if (rho > best) {
                best = rho;
                besti = i;
                bestj = (int)j;
            }
        }
    rv[threadIdx.x] = best;
    ri[threadIdx.x] = besti;
    rj[threadIdx.x] = bestj;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o && rv[threadIdx.x + o] > rv[threadIdx.x]) {
            rv[threadIdx.x] = rv[threadIdx.x + o];
            ri[threadIdx.x] = ri[threadIdx.x + o];
            rj[threadIdx.x] = rj[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        bval[b] = rv[0];
        bi[b] = ri[0];
        bj[b] = rj[0];
    }
}

// Largest sqrt(rho) of the current factorization and its (position in the pivot list, column).
static int rrqr_measure(krr_ctx* ctx, const float* Rout, long long n, int k, const int* piv, const double* nrm,
                        double* rho_max, int* pos, int* col) {
    double *R11, *L, *Linv, *wn;
    float *W32, *bval;
    int *bi, *bj;
    KRR_RET(bufT(ctx, "srq_r11", (size_t)k * k, &R11));
    KRR_RET(bufT(ctx, "srq_l", (size_t)k * k, &L));
    KRR_RET(bufT(ctx, "srq_linv", (size_t)k * k, &Linv));
    KRR_RET(bufT(ctx, "srq_wn", (size_t)k, &wn));
    KRR_RET(bufT(ctx, "srq_w32", (size_t)k * k, &W32));
    const dim3 grid((unsigned)ceil_div(n, RT), (unsigned)ceil_div(k, RT));
    const size_t nb = (size_t)grid.x * grid.y;
    KRR_RET(bufT(ctx, "srq_bval", nb, &bval));
    KRR_RET(bufT(ctx, "srq_bi", nb, &bi));
    KRR_RET(bufT(ctx, "srq_bj", nb, &bj));
    k_gather_r11<<<ceil_div((long long)k * k, 256), 256, 0, ctx->stream>>>(Rout, n, piv, k, R11);
    KRR_CHECK_LAUNCH();
    KRR_RET(launch_transpose64(ctx, R11, L, k));   // L = R11^T, lower
    KRR_RET(launch_set_identity(ctx, Linv, k));
    KRR_RET(launch_trsm_lower(ctx, L, Linv, k));   // Linv = R11^{-T}
    k_rrqr_w<<<k, 256, 0, ctx->stream>>>(Linv, k, W32, wn);
    KRR_CHECK_LAUNCH();
    k_rrqr_rho<<<grid, 256, 0, ctx->stream>>>(W32, k, Rout, n, nrm, wn, bval, bi, bj);
    KRR_CHECK_LAUNCH();
    std::vector<float> hv(nb);
    std::vector<int> hi(nb), hj(nb);
    KRR_TRY_CUDA(cudaMemcpyAsync(hv.data(), bval, sizeof(float) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    KRR_TRY_CUDA(cudaMemcpyAsync(hi.data(), bi, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    KRR_TRY_CUDA(cudaMemcpyAsync(hj.data(), bj, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream));
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    double best = -1.0;
    *pos = *col = -1;
    for (size_t b = 0; b < nb; ++b)
        if (hv[b] > best && hi[b] >= 0) {
            best = hv[b];
            *pos = hi[b];
            *col = hj[b];
        }
    *rho_max = best > 0.0 ? std::sqrt(best) : 0.0;
    return KRR_OK;
}

int launch_strong_rrqr(krr_ctx* ctx, float* Y, long long n, int l, int ldy, int k, double f, int max_swaps,
                       int* piv, float* rdiag, int* swaps_out, double* rho_out) {
    if (!(f > 1.0)) return fail(ctx, KRR_E_INVAL, "strong RRQR needs f > 1");
    if (k >= n) return fail(ctx, KRR_E_INVAL, "strong RRQR needs k < n");
    float *Ycopy, *Rout;
    int* forced;
    KRR_RET(bufT(ctx, "srq_y", (size_t)n * ldy, &Ycopy));
    KRR_RET(bufT(ctx, "srq_rout", (size_t)k * n, &Rout));
    KRR_RET(bufT(ctx, "srq_forced", (size_t)k, &forced));
    KRR_TRY_CUDA(cudaMemcpyAsync(Ycopy, Y, sizeof(float) * n * ldy, cudaMemcpyDeviceToDevice, ctx->stream));
    std::vector<int> order(k);
    int swaps = 0;
    double rho = 0.0;
    for (int s = 0;; ++s) {
        if (s > 0)
            KRR_TRY_CUDA(cudaMemcpyAsync(Y, Ycopy, sizeof(float) * n * ldy, cudaMemcpyDeviceToDevice, ctx->stream));
        KRR_TRY_CUDA(cudaMemsetAsync(Rout, 0, sizeof(float) * k * n, ctx->stream));
        double* nrm = nullptr;
        KRR_RET(qrcp_core(ctx, Y, n, l, ldy, k, piv, rdiag, s > 0 ? forced : nullptr, Rout, &nrm));
        int pos = -1, col = -1;
        KRR_RET(rrqr_measure(ctx, Rout, n, k, piv, nrm, &rho, &pos, &col));
        // a small slack keeps FP32 rounding of a boundary case from swapping back and forth
        if (rho <= f * (1.0 + 1e-3) || pos < 0 || s >= max_swaps) break;
        KRR_TRY_CUDA(cudaMemcpyAsync(order.data(), piv, sizeof(int) * k, cudaMemcpyDeviceToHost, ctx->stream));
        KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
        order[pos] = col;   // column col takes the place of pivot pos
        KRR_TRY_CUDA(cudaMemcpyAsync(forced, order.data(), sizeof(int) * k, cudaMemcpyHostToDevice, ctx->stream));
        ++swaps;
    }
    if (swaps_out) *swaps_out = swaps;
    if (rho_out) *rho_out = rho;
    return KRR_OK;
}

}  // namespace krr

using namespace krr;

extern "C" int krr_strong_rrqr(krr_ctx* ctx, float* Y, long long n, int l, int k, double f, int max_swaps,
                               int* piv, float* rdiag, int* swaps, double* rho_max) {
    if (!ctx) return KRR_E_INVAL;
    if (!Y || !piv || !rdiag || n < 2 || l < 1 || k < 1 || k > l || k >= n || max_swaps < 0)
        return fail(ctx, KRR_E_INVAL, "bad strong RRQR arguments");
    return launch_strong_rrqr(ctx, Y, n, l, l, k, f, max_swaps, piv, rdiag, swaps, rho_max);
}
