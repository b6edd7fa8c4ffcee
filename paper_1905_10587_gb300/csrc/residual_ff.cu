// Refinement residual R = Y - (K + beta I) A carried in float-float on the FP32 pipe.
//
// GB300 issues FP64 FMAs at about 1/70 of the FP32 rate, so the residual that
// drives iterative refinement keeps every quantity as an unevaluated sum of two
// floats (about 48 significant bits) instead:
//   * x_i . x_j is summed exactly term by term (FMA two-product + Knuth two-sum),
//     and ||x_i - x_j||^2 = n_i + n_j - 2 x_i . x_j with float-float norms;
//   * t = -s ||x_i - x_j||^2 with s = log2(e) / (2 sigma^2) in float-float;
//   * 2^t by the table-driven reduction of P. T. P. Tang, "Table-driven
//     implementation of the exponential function in IEEE floating-point
//     arithmetic", ACM TOMS 15(2), 1989, carried in float-float:
//     2^t = 2^m * 2^(j/64) * e^z with m = round(t), j = round(64 (t - m)) picking
//     an entry of a 65-entry float-float table of 2^(j/64) (built on the host in
//     double), and e^z with |z| <= ln2/128 evaluated as its Taylor polynomial
//     1 + z + ... + z^5/120 (truncation below 4e-17); the low word of t enters as
//     the factor (1 + ln2 t_lo);
//   * K_ij A_j is formed exactly (two-product), summed in float-float over a
//     tile of 64 columns and folded into an FP64 accumulator per tile.
// Relative error of each kernel value is a few 1e-12, against ~1e-7 for the FP32
// tile kernel.
#include "internal.cuh"

#include <algorithm>
#include <cmath>

namespace krr {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

// float-float squared norm of a point
__global__ void k_ff_norms(const float* __restrict__ X, long long n, int d, float2* __restrict__ N) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h = 0.f, l = 0.f;
    for (int c = 0; c < d; ++c) {
        const float x = X[i * d + c];
        float p, pe, s, e;
        two_prod(x, x, p, pe);
        two_sum(h, p, s, e);
        h = s;
        l = __fadd_rn(l, __fadd_rn(e, pe));
    }
    float s, e;
    fast_two_sum(h, l, s, e);
    N[i] = make_float2(s, e);
}

// A (FP64, nr columns) -> float-float pairs
__global__ void k_split64(const double* __restrict__ A, long long tot, float2* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= tot) return;
    const double a = A[e];
    const float h = (float)a;
    out[e] = make_float2(h, (float)(a - (double)h));
}

constexpr int FF_THREADS = 128;
constexpr int FF_BN = 64;
constexpr float LN2_H = 0.693147182464599609375f;          // float nearest ln 2
constexpr float LN2_L = -1.904654323148236e-09f;           // ln 2 - LN2_H

// Row block against column tiles: S_i = sum_j w_ij A_j in float-float, with w = K (mode 0)
// or w = t K, t = -s ||x_i - x_j||^2 in log2 units (mode 1, the sigma derivative up to -2 ln 2).
template <int D, int NR, int MODE>
__global__ void __launch_bounds__(FF_THREADS, 4)
k_rect_ff(const float* __restrict__ Xr, int nr, const float2* __restrict__ NR_, const float* __restrict__ Xc,
          int nc, const float2* __restrict__ NC_, float sh, float sl, const float2* __restrict__ Aff,
          const float2* __restrict__ tab, int tiles_per_split, double* __restrict__ part) {
    __shared__ float sx[FF_BN][D + 1];
    __shared__ float2 snrm[FF_BN];
    __shared__ float2 sa[NR][FF_BN];
    __shared__ float2 stab[65];
    const int tid = threadIdx.x;
    if (tid < 65) stab[tid] = tab[tid];
    const long long i = (long long)blockIdx.x * FF_THREADS + tid;
    const bool row_ok = i < nr;
    float xi[D];
#pragma unroll
    for (int c = 0; c < D; ++c) xi[c] = row_ok ? Xr[i * D + c] : 0.f;
    const float2 ni = row_ok ? NR_[i] : make_float2(0.f, 0.f);
    double acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = 0.0;

    const int ntiles = (nc + FF_BN - 1) / FF_BN;
    const int t0 = blockIdx.y * tiles_per_split;
    const int t1 = min(t0 + tiles_per_split, ntiles);
    for (int t = t0; t < t1; ++t) {
        const int c0 = t * FF_BN;
        __syncthreads();
        for (int e = tid; e < FF_BN * D; e += FF_THREADS) {
            const int j = e / D, c = e - j * D;
            sx[j][c] = (c0 + j < nc) ? Xc[(size_t)(c0 + j) * D + c] : 0.f;
        }
        for (int e = tid; e < FF_BN; e += FF_THREADS)
            snrm[e] = (c0 + e < nc) ? NC_[c0 + e] : make_float2(0.f, 0.f);
        for (int e = tid; e < NR * FF_BN; e += FF_THREADS) {
            const int q = e / FF_BN, j = e - q * FF_BN;
            sa[q][j] = (c0 + j < nc) ? Aff[(size_t)q * nc + c0 + j] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        float Sh[NR], Sl[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) Sh[q] = 0.f, Sl[q] = 0.f;
        const int jmax = min(FF_BN, nc - c0);
        for (int j = 0; j < jmax; ++j) {
            // x_i . x_j exactly up to the float-float accumulation
            float H = 0.f, L = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                float p, pe, s, e;
                two_prod(xi[c], sx[j][c], p, pe);
                two_sum(H, p, s, e);
                H = s;
                L = __fadd_rn(L, __fadd_rn(e, pe));
            }
            // D2 = n_i + n_j - 2 dot
            const float2 nj = snrm[j];
            float A, a, B, b, Dh, Dl;
            two_sum(ni.x, nj.x, A, a);
            a = __fadd_rn(a, __fadd_rn(ni.y, nj.y));
            two_sum(A, -2.f * H, B, b);
            b = __fadd_rn(b, __fsub_rn(a, 2.f * L));
            fast_two_sum(B, b, Dh, Dl);
            if (Dh <= 0.f) Dh = 0.f, Dl = 0.f;
            // t = -s D2
            float th = __fmul_rn(-sh, Dh);
            float tl = fmaf(-sh, Dh, -th);
            tl = __fsub_rn(tl, __fadd_rn(__fmul_rn(sh, Dl), __fmul_rn(sl, Dh)));
            fast_two_sum(th, tl, th, tl);
            if (th < -120.f) continue;   // K < 2^-120: below any residual that matters
            // 2^t = 2^m 2^(jj/64) e^z
            const float m = rintf(th);
            const float f64 = __fmul_rn(__fsub_rn(th, m), 64.f);
            const float jj = rintf(f64);
            const float r = __fmul_rn(__fsub_rn(f64, jj), 0.015625f);
            const float zh = __fmul_rn(r, LN2_H);
            const float zl = __fadd_rn(fmaf(r, LN2_H, -zh), __fadd_rn(__fmul_rn(r, LN2_L), __fmul_rn(tl, LN2_H)));
            const float q = __fmul_rn(__fmul_rn(zh, zh),
                                      fmaf(zh, fmaf(zh, fmaf(zh, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f));
            float Eh, El;
            fast_two_sum(1.f, zh, Eh, El);
            El = __fadd_rn(El, q);
            El = fmaf(Eh, zl, El);
            const float2 T = stab[(int)jj + 32];
            float Kh = __fmul_rn(T.x, Eh);
            float Kl = __fadd_rn(fmaf(T.x, Eh, -Kh), __fadd_rn(__fmul_rn(T.x, El), __fmul_rn(T.y, Eh)));
            fast_two_sum(Kh, Kl, Kh, Kl);
            const float sc = __int_as_float(((int)m + 127) << 23);   // 2^m, m in [-120, 0]
            Kh = __fmul_rn(Kh, sc);
            Kl = __fmul_rn(Kl, sc);
            if (MODE == 1) {   // w = t K
                const float ph = __fmul_rn(th, Kh);
                const float pl = __fadd_rn(fmaf(th, Kh, -ph), __fadd_rn(__fmul_rn(th, Kl), __fmul_rn(tl, Kh)));
                fast_two_sum(ph, pl, Kh, Kl);
            }
#pragma unroll
            for (int qq = 0; qq < NR; ++qq) {
                const float2 aj = sa[qq][j];
                float p, pe, s, e;
                two_prod(Kh, aj.x, p, pe);
                pe = __fadd_rn(pe, __fadd_rn(__fmul_rn(Kh, aj.y), __fmul_rn(Kl, aj.x)));
                two_sum(Sh[qq], p, s, e);
                Sh[qq] = s;
                Sl[qq] = __fadd_rn(Sl[qq], __fadd_rn(e, pe));
            }
        }
#pragma unroll
        for (int qq = 0; qq < NR; ++qq) acc[qq] += (double)Sh[qq] + (double)Sl[qq];
    }
    if (row_ok) {
#pragma unroll
        for (int q = 0; q < NR; ++q) part[((size_t)blockIdx.y * NR + q) * nr + i] = acc[q];
    }
}

__global__ void k_rect_ff_reduce(const double* __restrict__ part, int splits, int n, int nr,
                                 double scale, double* __restrict__ out) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nr) return;
    const int q = (int)(e / n);
    const int i = (int)(e - (long long)q * n);
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[((size_t)sp * nr + q) * n + i];
    out[(size_t)q * n + i] = scale * s;
}

__global__ void k_resid_ff_reduce(const double* __restrict__ part, int splits, int n, int nr,
                                  const float* __restrict__ Y, const double* __restrict__ A,
                                  double beta, double* __restrict__ R) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)n * nr) return;
    const int q = (int)(e / n);
    const int i = (int)(e - (long long)q * n);
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[((size_t)sp * nr + q) * n + i];
    R[(size_t)q * n + i] = (double)Y[(size_t)q * n + i] - beta * A[(size_t)q * n + i] - s;
}

typedef void (*ff_fn)(const float*, int, const float2*, const float*, int, const float2*, float, float,
                      const float2*, const float2*, int, double*);

template <int D, int MODE>
static ff_fn ff_pick1(int nr) {
    switch (nr) {
        case 1: return &k_rect_ff<D, 1, MODE>;
        case 2: return MODE == 0 ? &k_rect_ff<D, 2, MODE> : nullptr;
        case 4: return MODE == 0 ? &k_rect_ff<D, 4, MODE> : nullptr;
        case 8: return MODE == 0 ? &k_rect_ff<D, 8, MODE> : nullptr;
        case 16: return MODE == 0 ? &k_rect_ff<D, 16, MODE> : nullptr;
    }
    return nullptr;
}

static ff_fn ff_pick(int d, int nr, int mode) {
    switch (d) {
#define KRR_D(v) \
    case v: return mode == 0 ? ff_pick1<v, 0>(nr) : ff_pick1<v, 1>(nr);
        KRR_D(1) KRR_D(2) KRR_D(3) KRR_D(4) KRR_D(5) KRR_D(6) KRR_D(7) KRR_D(8)
        KRR_D(9) KRR_D(10) KRR_D(11) KRR_D(12) KRR_D(13) KRR_D(14) KRR_D(15) KRR_D(16)
#undef KRR_D
    }
    return nullptr;
}

int choose_splits_public(int nblk, int ntiles, int slots);

static int ff_table(krr_ctx* ctx, float2** tab) {
    // 2^(j/64), j = -32..32, as float-float pairs
    KRR_RET(bufT(ctx, "ff_tab", 65, tab));
    float2 h[65];
    for (int j = -32; j <= 32; ++j) {
        const double v = std::exp2(j / 64.0);
        const float hi = (float)v;
        h[j + 32] = make_float2(hi, (float)(v - (double)hi));
    }
    KRR_TRY_CUDA(cudaMemcpyAsync(*tab, h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    KRR_TRY_CUDA(cudaStreamSynchronize(ctx->stream));
    return KRR_OK;
}

// part (splits x nrhs x nr) of S_i = sum_j w_ij A_j for rows Xr and columns Xc (mode as above).
static int rect_ff_parts(krr_ctx* ctx, const float* Xr, long long nr, const float* Xc, long long nc,
                         int d, double sigma, const double* A, int nrhs_chunk, int mode,
                         double** part_out, int* splits_out) {
    float2* tab;
    KRR_RET(ff_table(ctx, &tab));
    float2 *NXr, *NXc, *Aff;
    KRR_RET(bufT(ctx, "ff_nr", (size_t)nr, &NXr));
    KRR_RET(bufT(ctx, "ff_nc", (size_t)nc, &NXc));
    KRR_RET(bufT(ctx, "ff_alpha", (size_t)nc * nrhs_chunk, &Aff));
    k_ff_norms<<<ceil_div(nr, 256), 256, 0, ctx->stream>>>(Xr, nr, d, NXr);
    KRR_CHECK_LAUNCH();
    k_ff_norms<<<ceil_div(nc, 256), 256, 0, ctx->stream>>>(Xc, nc, d, NXc);
    KRR_CHECK_LAUNCH();
    k_split64<<<ceil_div(nc * nrhs_chunk, 256), 256, 0, ctx->stream>>>(A, nc * nrhs_chunk, Aff);
    KRR_CHECK_LAUNCH();
    const double s = 1.4426950408889634 / (2.0 * sigma * sigma);
    const float sh = (float)s, sl = (float)(s - (double)sh);
    ff_fn fn = ff_pick(d, nrhs_chunk, mode);
    if (!fn) return fail(ctx, KRR_E_INVAL, "float-float product: unsupported shape");
    const int nblk = (int)ceil_div(nr, FF_THREADS);
    const int ntiles = (int)ceil_div(nc, FF_BN);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, FF_THREADS, 0);
    const int slots = ctx->num_sms * std::max(occ, 1);
    int splits = choose_splits_public(nblk, ntiles, slots);
    const int tps = (ntiles + splits - 1) / splits;
    splits = (ntiles + tps - 1) / tps;
    double* part;
    KRR_RET(bufT(ctx, "ff_part", (size_t)splits * nrhs_chunk * nr, &part));
    dim3 grid(nblk, splits);
    fn<<<grid, FF_THREADS, 0, ctx->stream>>>(Xr, (int)nr, NXr, Xc, (int)nc, NXc, sh, sl, Aff, tab, tps, part);
    KRR_CHECK_LAUNCH();
    *part_out = part;
    *splits_out = splits;
    return KRR_OK;
}

int launch_residual_ff(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                       const float* Y, const double* A, int nrhs, double* R) {
    if (n > 0x7fffffffLL) return fail(ctx, KRR_E_INVAL, "residual: more than 2^31 points");
    if (d > 16) return launch_residual_hp(ctx, X, n, d, sigma, beta, Y, A, nrhs, R);
    int done = 0;
    while (done < nrhs) {
        const int left = nrhs - done;
        const int chunk = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        double* part;
        int splits;
        KRR_RET(rect_ff_parts(ctx, X, n, X, n, d, sigma, A + (size_t)done * n, chunk, 0, &part, &splits));
        k_resid_ff_reduce<<<ceil_div(n * chunk, 256), 256, 0, ctx->stream>>>(
            part, splits, (int)n, chunk, Y + (size_t)done * n, A + (size_t)done * n, beta,
            R + (size_t)done * n);
        KRR_CHECK_LAUNCH();
        done += chunk;
    }
    return KRR_OK;
}

// out (nr) = K(Xr, Xc) a (mode 0) or (dK(Xr, Xc)/dlog sigma) a (mode 1), float-float, FP64 in/out.
int launch_rect_ff(krr_ctx* ctx, const float* Xr, long long nr, const float* Xc, long long nc, int d,
                   double sigma, const double* a, int mode, double* out) {
    if (nr > 0x7fffffffLL || nc > 0x7fffffffLL) return fail(ctx, KRR_E_INVAL, "too many points");
    if (d > 16) return fail(ctx, KRR_E_INVAL, "float-float products need d <= 16");
    double* part;
    int splits;
    KRR_RET(rect_ff_parts(ctx, Xr, nr, Xc, nc, d, sigma, a, 1, mode, &part, &splits));
    const double scale = mode == 1 ? -2.0 * 0.6931471805599453 : 1.0;
    k_rect_ff_reduce<<<ceil_div(nr, 256), 256, 0, ctx->stream>>>(part, splits, (int)nr, 1, scale, out);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

}  // namespace krr
