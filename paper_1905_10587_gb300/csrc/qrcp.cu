// Column-pivoted QR pivot selection (Algorithm 1, steps 3-4) on Y^T.
//
// The columns of Y^T are the rows of the n x l sketch Y.  Step m takes the row p whose
// residual (its part orthogonal to the rows chosen before) has the largest norm, lowest
// index on ties: the Businger-Golub pivot sequence.  The residuals are kept by
// Householder reflectors acting on the coordinates of the rows, blocked in panels of
// QH_B pivots:
//   * reflector m (coordinates m..l-1) is built from the pivot row's current residual,
//     H_m = I - tau_m v_m v_m^T with v_m[m] = 1;
//   * within a panel the rows are not rewritten: c[i][j] = tau_j v_j . y_i^(j) records
//     what reflector j does to row i, so y_i^(m) = y_i^(m0) - sum_j c[i][j] v_j, and one
//     read-only pass over the trailing coordinates m..l-1 per pivot gives c[i][m], the new
//     coordinate r_im of every row and its residual norm by downdating (FP64);
//   * at the end of a panel one pass applies the panel's reflectors to the coordinates
//     beyond it and recomputes every residual norm exactly.
// Each pivot reads n x (l - m) floats (the trailing part shrinks), and each panel reads
// and writes it once, instead of reading and writing the whole n x l sketch per pivot.
#include "internal.cuh"

#include <algorithm>

namespace krr {

constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;
constexpr int QH_B = 32;   // pivots per panel
constexpr int QR_REF_THREADS = 1024;   // the one-block reflector kernel: short dependent chains
constexpr int QR_REF_WARPS = QR_REF_THREADS / 32;

// max key = largest residual norm, then lowest index
__device__ __forceinline__ unsigned long long pivot_key(double nrm2, long long i) {
    const float f = (float)fmax(nrm2, 0.0);
    return ((unsigned long long)__float_as_uint(f) << 32) | (unsigned long long)(0xffffffffu - (unsigned)i);
}
__device__ __forceinline__ long long key_index(unsigned long long k) {
    return (long long)(0xffffffffu - (unsigned)(k & 0xffffffffu));
}

// residual norms of all rows (FP64 sums) and the key of the first pivot
__global__ void __launch_bounds__(QR_THREADS)
k_qr_norms(const float* __restrict__ Y, long long n, int l, int ldy, double* __restrict__ nrm,
           unsigned long long* __restrict__ bkeys) {
    __shared__ unsigned long long sbest[QR_WARPS];
    const int lane = threadIdx.x & 31;
    const long long w0 = (long long)blockIdx.x * QR_WARPS + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * QR_WARPS;
    unsigned long long best = 0;
    for (long long i = w0; i < n; i += nw) {
        double s = 0.0;
        for (int c = lane; c < l; c += 32) {
            const double v = Y[i * ldy + c];
            s = fma(v, v, s);
        }
        s = warp_sum(s);
        if (lane == 0) nrm[i] = s;
        best = max(best, pivot_key(s, i));
    }
    if (lane == 0) sbest[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < QR_WARPS; ++w) b = max(b, sbest[w]);
        bkeys[blockIdx.x] = b;
    }
}

// Reflector of pivot step m (panel column jm = m - m0), one block: the pivot row's
// residual z = y_p^(m0)[m:] - sum_{j<jm} c[p][j] v_j[m:], then v = z / (z_0 - alpha) with
// alpha = -sign(z_0) ||z||, tau = (alpha - z_0) / alpha (v_0 = 1), and g_j = v . v_j[m:]
// for the earlier reflectors of the panel.  Writes the pivot, |R_mm| = ||z|| and marks
// the row chosen.
__global__ void __launch_bounds__(QR_REF_THREADS)
k_qr_reflector(const float* __restrict__ Y, long long n, int l, int ldy, int m, int jm, const float* __restrict__ C,
               float* __restrict__ Vp, float* __restrict__ tau, float* __restrict__ g,
               double* __restrict__ nrm, const unsigned long long* __restrict__ bkeys, int nbk,
               int* __restrict__ piv, float* __restrict__ rdiag, const int* __restrict__ forced,
               float* __restrict__ Rout) {
    extern __shared__ double zs[];   // l - m
    __shared__ double red[QR_REF_WARPS];
    __shared__ unsigned long long kred[QR_REF_WARPS];
    __shared__ double s_alpha, s_scale;
    const int L = l - m;
    // the pivot: the largest of the previous pass's per-block keys
    {
        unsigned long long b = 0;
        for (int i = threadIdx.x; i < nbk; i += QR_REF_THREADS) b = max(b, bkeys[i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        if ((threadIdx.x & 31) == 0) kred[threadIdx.x >> 5] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (int w = 0; w < QR_REF_WARPS; ++w) t = max(t, kred[w]);
            kred[0] = t;
        }
        __syncthreads();
    }
    // the argmax, or the caller's pivot (strong RRQR re-factorizes with a given order)
    const unsigned long long km = forced ? 1ull : kred[0];
    const long long p = forced ? (long long)forced[m] : key_index(km);
    if (km == 0 || p < 0 || p >= n) {   // no candidate left (cannot happen for k <= n): stop
        if (threadIdx.x == 0) {
            piv[m] = 0;
            rdiag[m] = 0.f;
            tau[jm] = 0.f;
        }
        for (int t = threadIdx.x; t < l; t += QR_REF_THREADS) Vp[(size_t)jm * l + t] = 0.f;
        if (threadIdx.x < jm) g[threadIdx.x] = 0.f;
        return;
    }
    const float* yp = Y + p * ldy;
    const float* cp = C + p * QH_B;
    __shared__ float cps[QH_B];
    if (threadIdx.x < QH_B) cps[threadIdx.x] = threadIdx.x < jm ? cp[threadIdx.x] : 0.f;
    __syncthreads();
    double ss = 0.0;
    for (int t = threadIdx.x; t < L; t += QR_REF_THREADS) {
        double z = yp[m + t];
        const float* vt = Vp + m + t;
#pragma unroll 8
        for (int j = 0; j < jm; ++j) z -= (double)cps[j] * (double)vt[(size_t)j * l];
        zs[t] = z;
        ss = fma(z, z, ss);
    }
    ss = warp_sum(ss);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t2 = 0.0;
        for (int i = 0; i < QR_REF_WARPS; ++i) t2 += red[i];
        const double nz = sqrt(t2);
        const double z0 = zs[0];
        const double alpha = z0 >= 0.0 ? -nz : nz;
        double scale = 0.0, tu = 0.0;
        if (nz > 0.0 && z0 - alpha != 0.0) {
            scale = 1.0 / (z0 - alpha);
            tu = (alpha - z0) / alpha;
        }
        s_alpha = alpha;
        s_scale = scale;
        tau[jm] = (float)tu;
        piv[m] = (int)p;
        rdiag[m] = (float)nz;
        nrm[p] = -1.0;
        if (Rout) Rout[(size_t)m * n + p] = (float)alpha;   // R_mm
    }
    __syncthreads();
    float* vm = Vp + (size_t)jm * l;
    const double scale = s_scale;
    // g_j = v . v_j[m:] for j < jm: every thread sums its coordinates for all j at once
    // (independent loads), then one reduction per j
    float gacc[QH_B];
#pragma unroll
    for (int j = 0; j < QH_B; ++j) gacc[j] = 0.f;
    for (int t = threadIdx.x; t < l; t += QR_REF_THREADS) {
        float v = 0.f;
        if (t == m) v = 1.f;
        else if (t > m) v = (float)(zs[t - m] * scale);
        vm[t] = v;
        if (t >= m) {
#pragma unroll
            for (int j = 0; j < QH_B; ++j)
                if (j < jm) gacc[j] = fmaf(v, Vp[(size_t)j * l + t], gacc[j]);
        }
    }
    __shared__ float gred[QR_REF_WARPS][QH_B];
#pragma unroll
    for (int j = 0; j < QH_B; ++j) {
        const float sj = warp_sum(gacc[j]);
        if (lane == 0) gred[w][j] = sj;
    }
    __syncthreads();
    if (threadIdx.x < jm) {
        float t2 = 0.f;
        for (int i = 0; i < QR_REF_WARPS; ++i) t2 += gred[i][threadIdx.x];
        g[threadIdx.x] = t2;
    }
}

// Pivot step m: for every row not chosen, c[i][jm] = tau (v . y_i^(m0)[m:] - sum_j c[i][j] g_j),
// its coordinate r = y_i^(m0)[m] - sum_j c[i][j] v_j[m] - c[i][jm], and nrm_i -= r^2; the
// key of the next pivot.  One warp per row, reading the row's coordinates m..l-1 once; the
// row's loads (NPL per lane), its c values and its norm are all issued before any use.
template <int NPL>
__global__ void __launch_bounds__(QR_THREADS)
k_qr_step(const float* __restrict__ Y, long long n, int l, int ldy, int m, int jm, float* __restrict__ C,
          const float* __restrict__ Vp, const float* __restrict__ tau, const float* __restrict__ g,
          double* __restrict__ nrm, unsigned long long* __restrict__ bkeys, float* __restrict__ Rout) {
    __shared__ float vsh[NPL * 32];   // v_m[m:], zero-padded
    __shared__ float gsh[QH_B], vjm[QH_B];
    __shared__ unsigned long long sbest[QR_WARPS];
    const int L = l - m;
    const float* vm = Vp + (size_t)jm * l + m;
    for (int t = threadIdx.x; t < NPL * 32; t += QR_THREADS) vsh[t] = t < L ? vm[t] : 0.f;
    if (threadIdx.x < QH_B) {
        gsh[threadIdx.x] = threadIdx.x < jm ? g[threadIdx.x] : 0.f;
        vjm[threadIdx.x] = threadIdx.x < jm ? Vp[(size_t)threadIdx.x * l + m] : 0.f;
    }
    __syncthreads();
    const float tu = tau[jm];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long w0 = (long long)blockIdx.x * QR_WARPS + wid;
    const long long nw = (long long)gridDim.x * QR_WARPS;
    unsigned long long best = 0;
    for (long long i = w0; i < n; i += nw) {
        const float* yi = Y + i * ldy + m;
        float y[NPL];
#pragma unroll
        for (int u = 0; u < NPL; ++u) {
            const int t = lane + 32 * u;
            y[u] = t < L ? yi[t] : 0.f;
        }
        const float cij = lane < jm ? C[i * QH_B + lane] : 0.f;
        const double ni = nrm[i];
        if (ni < 0.0) continue;   // chosen (uniform across the warp)
        float dot = 0.f;
#pragma unroll
        for (int u = 0; u < NPL; ++u) dot = fmaf(y[u], vsh[lane + 32 * u], dot);
        dot = warp_sum(dot);
        const float corr = warp_sum(cij * gsh[lane]);
        const float shift = warp_sum(cij * vjm[lane]);
        if (lane == 0) {
            const float cm = tu * (dot - corr);
            C[i * QH_B + jm] = cm;
            const double r = (double)y[0] - (double)shift - (double)cm;
            if (Rout) Rout[(size_t)m * n + i] = (float)r;   // R_mi: coordinate m of row i
            const double nn = fmax(ni - r * r, 0.0);
            nrm[i] = nn;
            best = max(best, pivot_key(nn, i));
        }
    }
    if (lane == 0) sbest[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < QR_WARPS; ++w) b = max(b, sbest[w]);
        bkeys[blockIdx.x] = b;   // reduced by the next reflector (no atomic contention)
    }
}

typedef void (*qr_step_fn)(const float*, long long, int, int, int, int, float*, const float*, const float*,
                           const float*, double*, unsigned long long*, float*);

static qr_step_fn qr_step_for(int L) {
    const int npl = (L + 31) / 32;
    if (npl <= 2) return &k_qr_step<2>;
    if (npl <= 4) return &k_qr_step<4>;
    if (npl <= 8) return &k_qr_step<8>;
    if (npl <= 16) return &k_qr_step<16>;
    if (npl <= 32) return &k_qr_step<32>;
    if (npl <= 64) return &k_qr_step<64>;
    return &k_qr_step<128>;
}

// Panel end (nb reflectors, coordinates m1..l-1 with m1 = m0 + nb): y_i[m1:] -= sum_j
// c[i][j] v_j[m1:] for the rows not chosen, then their residual norms exactly (FP64) and
// the key of the next pivot.  One warp per row; the panel's reflectors in shared memory.
__global__ void __launch_bounds__(QR_THREADS)
k_qr_panel(float* __restrict__ Y, long long n, int l, int ldy, int m1, int nb, const float* __restrict__ C,
           const float* __restrict__ Vp, double* __restrict__ nrm, unsigned long long* __restrict__ bkeys) {
    extern __shared__ float vps[];   // nb x (l - m1)
    __shared__ unsigned long long sbest[QR_WARPS];
    const int L = l - m1;
    for (int e = threadIdx.x; e < nb * L; e += QR_THREADS) {
        const int j = e / L, t = e - j * L;
        vps[e] = Vp[(size_t)j * l + m1 + t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long w0 = (long long)blockIdx.x * QR_WARPS + wid;
    const long long nw = (long long)gridDim.x * QR_WARPS;
    unsigned long long best = 0;
    for (long long i = w0; i < n; i += nw) {
        if (nrm[i] < 0.0) continue;   // chosen (uniform across the warp)
        // every lane takes the row's nb coefficients into registers (lane j loads c[i][j])
        const float cl = lane < nb ? C[i * QH_B + lane] : 0.f;
        float cr[QH_B];
#pragma unroll
        for (int j = 0; j < QH_B; ++j) cr[j] = __shfl_sync(0xffffffffu, cl, j);
        float* yi = Y + i * ldy + m1;
        double s = 0.0;
        for (int t = lane; t < L; t += 32) {
            float y = yi[t];
#pragma unroll
            for (int j = 0; j < QH_B; ++j)
                if (j < nb) y = fmaf(-cr[j], vps[j * L + t], y);
            yi[t] = y;
            s = fma((double)y, (double)y, s);
        }
        s = warp_sum(s);
        if (lane == 0) {
            nrm[i] = s;
            best = max(best, pivot_key(s, i));
        }
    }
    if (lane == 0) sbest[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int w = 0; w < QR_WARPS; ++w) b = max(b, sbest[w]);
        bkeys[blockIdx.x] = b;
    }
}

// The pivoted QR of Y^T (Y n x ldy, l used columns) for k pivots.  forced (device, k) makes
// step m take pivot forced[m] instead of the argmax; Rout (device, k x n) receives row m of R
// for every column (the pivot's diagonal, the rows not yet chosen; chosen ones are left
// alone), and then the last step runs too, so that nrm ends as the squared residual norms
// after k pivots (-1 for the chosen rows).
int qrcp_core(krr_ctx* ctx, float* Y, long long n, int l, int ldy, int k, int* piv, float* rdiag,
              const int* forced, float* Rout, double** nrm_out) {
    if (l > 4096) return fail(ctx, KRR_E_INVAL, "qrcp: more than 4096 projections");
    if (n >= 0xffffffffLL) return fail(ctx, KRR_E_INVAL, "qrcp: too many points");
    if (k > l) return fail(ctx, KRR_E_INVAL, "qrcp: more pivots than projections");
    // enough warps for every row's loads to be in flight within a few waves; every pass
    // writes one key per block, which the next reflector reduces
    const int grid = (int)std::min<long long>((long long)ctx->num_sms * 8, ceil_div(n, QR_WARPS));
    double* nrm;
    float *C, *Vp, *tau, *g;
    unsigned long long* bkeys;
    KRR_RET(bufT(ctx, "qr_nrm64", (size_t)n, &nrm));
    KRR_RET(bufT(ctx, "qr_c", (size_t)n * QH_B, &C));
    KRR_RET(bufT(ctx, "qr_v", (size_t)QH_B * l, &Vp));
    KRR_RET(bufT(ctx, "qr_tau", (size_t)QH_B, &tau));
    KRR_RET(bufT(ctx, "qr_g", (size_t)QH_B, &g));
    KRR_RET(bufT(ctx, "qr_bkeys", (size_t)grid, &bkeys));
    KRR_RET(allow_max_dynamic_smem(ctx, (const void*)k_qr_panel));
    // panel width: the panel's reflectors (nb x l floats) must fit 200 KB of shared memory
    const int bmax = std::max(1, std::min(QH_B, (200 * 1024) / (4 * l)));
    k_qr_norms<<<grid, QR_THREADS, 0, ctx->stream>>>(Y, n, l, ldy, nrm, bkeys);
    KRR_CHECK_LAUNCH();
    for (int m0 = 0; m0 < k; m0 += bmax) {
        const int nb = std::min(bmax, k - m0);
        for (int jm = 0; jm < nb; ++jm) {
            const int m = m0 + jm;
            const int L = l - m;
            if (sizeof(double) * L > 48 * 1024) KRR_RET(allow_max_dynamic_smem(ctx, (const void*)k_qr_reflector));
            k_qr_reflector<<<1, QR_REF_THREADS, sizeof(double) * L, ctx->stream>>>(Y, n, l, ldy, m, jm, C, Vp,
                                                                                 tau, g, nrm, bkeys, grid,
                                                                                 piv, rdiag, forced, Rout);
            KRR_CHECK_LAUNCH();
            if (m + 1 < k || Rout) {
                qr_step_for(L)<<<grid, QR_THREADS, 0, ctx->stream>>>(Y, n, l, ldy, m, jm, C, Vp, tau, g, nrm,
                                                                    bkeys, Rout);
                KRR_CHECK_LAUNCH();
            }
        }
        const int m1 = m0 + nb;
        if (m1 < k) {
            // the panel's updates reach the coordinates beyond it; the exact norms replace
            // the downdated ones and give the next pivot
            const size_t smem = sizeof(float) * (size_t)nb * (l - m1);
            k_qr_panel<<<grid, QR_THREADS, smem, ctx->stream>>>(Y, n, l, ldy, m1, nb, C, Vp, nrm, bkeys);
            KRR_CHECK_LAUNCH();
        }
    }
    if (nrm_out) *nrm_out = nrm;
    return KRR_OK;
}

int launch_qrcp(krr_ctx* ctx, float* Y, long long n, int l, int ldy, int k, int* piv, float* rdiag) {
    return qrcp_core(ctx, Y, n, l, ldy, k, piv, rdiag, nullptr, nullptr, nullptr);
}

}  // namespace krr
