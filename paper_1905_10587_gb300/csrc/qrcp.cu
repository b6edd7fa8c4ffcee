// Column-pivoted QR pivot selection (Algorithm 1, steps 3-4) on Y^T.
//
// The columns of Y^T are the rows of the n x l sketch Y.  Step j takes the row p
// with the largest residual norm (lowest index on ties), forms q = y_p / ||y_p||
// and projects q out of every remaining row (modified Gram-Schmidt); this is the
// Businger-Golub pivot sequence.  Each launch handles one step: a warp owns a
// row, keeps it in registers between the dot product and the update, writes it
// back and recomputes its norm exactly (no norm downdating), and the next pivot
// is found with a 64-bit atomicMax on (norm bits, ~index).
#include "internal.cuh"

#include <algorithm>

namespace krr {

constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;

__device__ __forceinline__ unsigned long long pivot_key(float nrm2, long long i) {
    return ((unsigned long long)__float_as_uint(nrm2) << 32) |
           (unsigned long long)(0xffffffffu - (unsigned)i);
}

template <int NPL>
__global__ void __launch_bounds__(QR_THREADS)
k_qr_norms(const float* __restrict__ Y, long long n, int l, int ldy, float* __restrict__ nrm,
           unsigned long long* __restrict__ key0) {
    const int lane = threadIdx.x & 31;
    const long long w0 = (long long)blockIdx.x * QR_WARPS + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * QR_WARPS;
    unsigned long long best = 0;
    for (long long i = w0; i < n; i += nw) {
        float s = 0.f;
        for (int c = lane; c < l; c += 32) {
            const float v = Y[i * ldy + c];
            s = fmaf(v, v, s);
        }
        s = warp_sum(s);
        if (lane == 0) nrm[i] = s;
        best = max(best, pivot_key(s, i));
    }
    if (lane == 0) atomicMax(key0, best);
}

// One pivot step j.  Rows already chosen carry nrm < 0.
template <int NPL>
__global__ void __launch_bounds__(QR_THREADS)
k_qr_step(float* __restrict__ Y, long long n, int l, int ldy, float* __restrict__ nrm,
          unsigned long long* __restrict__ keys, int j, int* __restrict__ piv,
          float* __restrict__ rdiag) {
    extern __shared__ float sq[];
    __shared__ unsigned long long sbest[QR_WARPS];
    const unsigned long long kj = keys[j];
    const long long p = (long long)(0xffffffffu - (unsigned)(kj & 0xffffffffu));
    const float pn2 = __uint_as_float((unsigned)(kj >> 32));
    const float inv = pn2 > 1e-30f ? rsqrtf(pn2) : 0.f;
    for (int c = threadIdx.x; c < l; c += QR_THREADS) sq[c] = Y[p * ldy + c] * inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        piv[j] = (int)p;
        rdiag[j] = sqrtf(fmaxf(pn2, 0.f));
        nrm[p] = -1.f;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long w0 = (long long)blockIdx.x * QR_WARPS + wid;
    const long long nw = (long long)gridDim.x * QR_WARPS;
    unsigned long long best = 0;
    for (long long i = w0; i < n; i += nw) {
        if (i == p) continue;
        if (nrm[i] < 0.f) continue;   // chosen earlier (uniform across the warp)
        float y[NPL];
        float t = 0.f;
#pragma unroll
        for (int m = 0; m < NPL; ++m) {
            const int c = lane + 32 * m;
            y[m] = (c < l) ? Y[i * ldy + c] : 0.f;
            if (c < l) t = fmaf(y[m], sq[c], t);
        }
        t = warp_sum(t);
        float s = 0.f;
#pragma unroll
        for (int m = 0; m < NPL; ++m) {
            const int c = lane + 32 * m;
            if (c < l) {
                y[m] = fmaf(-t, sq[c], y[m]);
                Y[i * ldy + c] = y[m];
                s = fmaf(y[m], y[m], s);
            }
        }
        s = warp_sum(s);
        if (lane == 0) nrm[i] = s;
        best = max(best, pivot_key(s, i));
    }
    if (lane == 0) sbest[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < QR_WARPS; ++w) b = max(b, sbest[w]);
        if (b) atomicMax(&keys[j + 1], b);
    }
}

typedef void (*qr_step_fn)(float*, long long, int, int, float*, unsigned long long*, int, int*,
                           float*);

int launch_qrcp(krr_ctx* ctx, float* Y, long long n, int l, int ldy, int k, int* piv,
                float* rdiag) {
    if (l > 4096) return fail(ctx, KRR_E_INVAL, "qrcp: more than 4096 projections");
    if (n >= 0xffffffffLL) return fail(ctx, KRR_E_INVAL, "qrcp: too many points");
    qr_step_fn step;
    const int npl = (l + 31) / 32;
    if (npl <= 4) step = &k_qr_step<4>;
    else if (npl <= 8) step = &k_qr_step<8>;
    else if (npl <= 16) step = &k_qr_step<16>;
    else if (npl <= 32) step = &k_qr_step<32>;
    else if (npl <= 64) step = &k_qr_step<64>;
    else step = &k_qr_step<128>;
    float* nrm;
    unsigned long long* keys;
    KRR_RET(bufT(ctx, "qr_nrm", (size_t)n, &nrm));
    KRR_RET(bufT(ctx, "qr_keys", (size_t)k + 1, &keys));
    KRR_TRY_CUDA(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * (k + 1), ctx->stream));
    int occ = 1;
    const size_t smem = sizeof(float) * l;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)step, QR_THREADS, smem);
    occ = std::max(occ, 1);
    const int grid = (int)std::min<long long>((long long)ctx->num_sms * occ,
                                              ceil_div(n, QR_WARPS));
    k_qr_norms<1><<<grid, QR_THREADS, 0, ctx->stream>>>(Y, n, l, ldy, nrm, keys);
    KRR_CHECK_LAUNCH();
    for (int j = 0; j < k; ++j) {
        step<<<grid, QR_THREADS, smem, ctx->stream>>>(Y, n, l, ldy, nrm, keys, j, piv, rdiag);
        KRR_CHECK_LAUNCH();
    }
    return KRR_OK;
}

}  // namespace krr
