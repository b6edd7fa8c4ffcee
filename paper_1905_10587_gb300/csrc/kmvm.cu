// Tiled on-the-fly Gaussian kernel products (the discrete Gauss transform of
// Section 2.4, Eq. (6), evaluated exactly): K is never stored.
//
//   Q_i = sum_j exp2(a_i + a_j + 2 xh_i . xh_j) V_j  (+ beta V_i)
//
// with xh = (x - mu) sqrt(s), a = -||xh||^2 and s = log2(e) / (2 sigma^2), which
// is exp(-||x_i - x_j||^2 / (2 sigma^2)).  Each CTA holds a block of rows in
// registers and streams the column points through shared memory; the exponent is
// d+1 FP32 FMAs, the exponential is one MUFU ex2, and each right-hand side costs
// one more FMA.  Columns are split across CTAs (split-K) when the rows alone
// cannot fill the 152 SMs; the partial sums then go through a small scratch
// buffer and a deterministic reduction.
//
// Also here: the FP64 residual used by iterative refinement, which evaluates
// the kernel from exact differences of the float32 coordinates in double.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <type_traits>

namespace krr {

// ------------------------------------------------------------------ mean / pack
__global__ void k_mean_partial(const float* __restrict__ X, long long n, int d,
                               double* __restrict__ part) {
    __shared__ double red[256];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
            s += (double)X[i * d + c];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * d + c] = red[0];
        __syncthreads();
    }
}

__global__ void k_mean_final(const double* __restrict__ part, int nblk, int d, long long n,
                             double* __restrict__ mu) {
    int c = threadIdx.x;
    if (c >= d) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(size_t)b * d + c];
    mu[c] = s / (double)n;
}

int launch_mean(krr_ctx* ctx, const float* X, long long n, int d, double* mu) {
    const int nblk = (int)std::min<long long>(2 * ctx->num_sms, ceil_div(n, 256));
    double* part;
    KRR_RET(bufT(ctx, "mean_part", (size_t)nblk * d, &part));
    k_mean_partial<<<nblk, 256, 0, ctx->stream>>>(X, n, d, part);
    KRR_CHECK_LAUNCH();
    k_mean_final<<<1, 64, 0, ctx->stream>>>(part, nblk, d, n, mu);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

__global__ void k_pack(const float* __restrict__ X, long long n, int d, int dk, int ps,
                       const double* __restrict__ mu, double sq, float* __restrict__ P) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double nrm = 0.0;
    float* out = P + i * ps;
    for (int c = 0; c < ps; ++c) {
        float v = 0.f;
        if (c < d) v = (float)(((double)X[i * d + c] - mu[c]) * sq);
        if (c < dk) {
            out[c] = v;
            nrm += (double)v * (double)v;
        } else {
            out[c] = 0.f;
        }
    }
    out[dk] = (float)(-nrm);
}

int launch_pack(krr_ctx* ctx, const float* X, long long n, int d, const double* mu, double s,
                float* P) {
    const int dk = kernel_dim(d);
    const int ps = packed_stride(d);
    k_pack<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(X, n, d, dk, ps, mu, std::sqrt(s), P);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

__global__ void k_gather_pack(const float* __restrict__ P, int ps, const float* __restrict__ X,
                              int d, const int* __restrict__ idx, int m, float* __restrict__ Pout,
                              float* __restrict__ Xout) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= m) return;
    long long i = idx[a];
    for (int c = 0; c < ps; ++c) Pout[(size_t)a * ps + c] = P[i * ps + c];
    if (Xout)
        for (int c = 0; c < d; ++c) Xout[(size_t)a * d + c] = X[i * d + c];
}

int launch_gather_pack(krr_ctx* ctx, const float* P, int ps, const float* X, int d,
                       const int* idx, int m, float* Pout, float* Xout) {
    k_gather_pack<<<ceil_div(m, 128), 128, 0, ctx->stream>>>(P, ps, X, d, idx, m, Pout, Xout);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// ------------------------------------------------------------------ FP32 tile MVM
constexpr int KM_THREADS = 128;
constexpr int KM_BN = 128;

// RAW = false: packed points [xh, a] and the expansion a_i + a_j + 2 xh_i . xh_j.
// RAW = true: packed points are the caller's coordinates unchanged and the exponent is
// nsc * sum_c (x_ic - x_jc)^2 with nsc = -s: no centring, scaling or norm is rounded
// per point, so the only per-entry errors are those of the differences, the squares
// and the exponential (about eps |t|) instead of eps (|a_i| + |a_j| + 2 |xh_i . xh_j|).
template <int D, int NRHS, int R, bool RAW>
__global__ void __launch_bounds__(KM_THREADS, 4)
k_kmvm(const float* __restrict__ Pr, int nr, const float* __restrict__ Pc, int nc,
       const float* __restrict__ V, int ldv, int tiles_per_split, float beta, float nsc, float kcorr,
       float* __restrict__ Q, int ldq, double* __restrict__ part) {
    constexpr int PS = (D + 1 + 3) / 4 * 4;
    constexpr int PS4 = PS / 4;
    __shared__ float4 sP[KM_BN * PS4];
    __shared__ __align__(16) float sV[KM_BN * NRHS];

    const int tid = threadIdx.x;
    const long long row0 = (long long)blockIdx.x * (KM_THREADS * R);

    float xi[R][D];
    float ai[R];
    float acc[R][NRHS];     // one column tile, FP32
    // tiles folded float-float (FP64 for the widest rows, short of registers): smooth
    // kernels cancel heavily across tiles
    using Fold = std::conditional_t<(D <= 32), FoldFF, Fold64>;
    Fold fold[R][NRHS];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = row0 + r * KM_THREADS + tid;
        const bool ok = i < nr;
#pragma unroll
        for (int c = 0; c < D; ++c) xi[r][c] = ok ? (RAW ? 1.f : 2.f) * Pr[i * PS + c] : 0.f;
        ai[r] = (ok && !RAW) ? Pr[i * PS + D] : 0.f;
#pragma unroll
        for (int q = 0; q < NRHS; ++q) acc[r][q] = 0.f;
    }

    const int ntiles = (nc + KM_BN - 1) / KM_BN;
    const int t0 = blockIdx.y * tiles_per_split;
    const int t1 = min(t0 + tiles_per_split, ntiles);
    const float4* Pc4 = reinterpret_cast<const float4*>(Pc);

    for (int t = t0; t < t1; ++t) {
        const int c0 = t * KM_BN;
        for (int e = tid; e < KM_BN * PS4; e += KM_THREADS) {
            const int j = e / PS4;
            sP[e] = (c0 + j < nc) ? Pc4[(size_t)(c0 + j) * PS4 + (e - j * PS4)]
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = tid; e < KM_BN * NRHS; e += KM_THREADS) {
            const int q = e / KM_BN, j = e - q * KM_BN;
            sV[j * NRHS + q] = (c0 + j < nc) ? V[(size_t)q * ldv + c0 + j] : 0.f;
        }
        __syncthreads();
#pragma unroll 2
        for (int j = 0; j < KM_BN; ++j) {
            float xj[PS];
#pragma unroll
            for (int w = 0; w < PS4; ++w) {
                const float4 v = sP[j * PS4 + w];
                xj[4 * w + 0] = v.x;
                xj[4 * w + 1] = v.y;
                xj[4 * w + 2] = v.z;
                xj[4 * w + 3] = v.w;
            }
            float vj[NRHS];
            if constexpr (NRHS % 4 == 0) {
#pragma unroll
                for (int w = 0; w < NRHS / 4; ++w) {
                    const float4 v = reinterpret_cast<const float4*>(sV + j * NRHS)[w];
                    vj[4 * w + 0] = v.x;
                    vj[4 * w + 1] = v.y;
                    vj[4 * w + 2] = v.z;
                    vj[4 * w + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < NRHS; ++q) vj[q] = sV[j * NRHS + q];
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float tt;
                if constexpr (RAW) {
                    float ss = 0.f;
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        const float df = xi[r][c] - xj[c];
                        ss = fmaf(df, df, ss);
                    }
                    tt = ss * nsc;
                } else {
                    tt = ai[r] + xj[D];
#pragma unroll
                    for (int c = 0; c < D; ++c) tt = fmaf(xi[r][c], xj[c], tt);
                }
                const float e = ex2f(tt);
#pragma unroll
                for (int q = 0; q < NRHS; ++q) acc[r][q] = fmaf(e, vj[q], acc[r][q]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < NRHS; ++q) fold[r][q].add(acc[r][q]), acc[r][q] = 0.f;
    }

#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = row0 + r * KM_THREADS + tid;
        if (i >= nr) continue;
        if (part == nullptr) {
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
                Q[(size_t)q * ldq + i] =
                    (float)(fold[r][q].get() * (1.0 + (double)kcorr) +
                            (beta != 0.f ? (double)beta * V[(size_t)q * ldv + i] : 0.0));
        } else {
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
                part[((size_t)blockIdx.y * NRHS + q) * nr + i] = fold[r][q].get();
        }
    }
}

// ------------------------------------------------------------------ paired-row FP32 product
// The same products as k_kmvm for an even number of rows per thread, two rows at a time
// on the paired FP32 instructions (fma/add/sub/mul.rn.f32x2): each instruction does the
// two rows' operations with the same rounding as two scalar ones, so the result equals
// k_kmvm's bit for bit while the exponent costs half the issue slots.  The column tile
// is staged with every coordinate duplicated ((x, x) per 64-bit word) so one shared load
// feeds both halves.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// COMP (split products of the FP64 recurrence, RAW only): V holds hi/lo column pairs;
// each even (hi) column's tile sum is compensated: the products e v are formed exactly
// (FMA two-product) and summed with Kahan's compensation, so a tile sum carries an error
// of a few u |sum| instead of u times the sum of |terms| (strong cancellation across a
// tile when the direction oscillates).  The odd (lo) columns, 2^-24 smaller, are summed
// plainly.  The entries are made accurate too: t = -s d^2 with s as a float pair (the
// kernel writes partial sums only, so the `beta` argument carries the low word of -s),
// and 2^t from the FMA-pipe polynomial exp2_poly instead of the MUFU approximation.
template <int D, int NRHS, int R, bool RAW, bool COMP = false>
__global__ void __launch_bounds__(KM_THREADS, 4)
k_kmvm2(const float* __restrict__ Pr, int nr, const float* __restrict__ Pc, int nc,
        const float* __restrict__ V, int ldv, int tiles_per_split, float beta, float nsc, float kcorr,
        float* __restrict__ Q, int ldq, double* __restrict__ part) {
    static_assert(R % 2 == 0, "rows in pairs");
    static_assert(!COMP || NRHS % 2 == 0, "compensated sums take hi/lo column pairs");
    constexpr int NC = COMP ? NRHS / 2 : 1;       // compensated (hi) columns
    constexpr int PS = (D + 1 + 3) / 4 * 4;
    constexpr int PS4 = PS / 4;
    constexpr int PH = PS / 2;                     // 128-bit words per column (2 duplicated coords)
    constexpr int RP = R / 2;
    __shared__ ulonglong2 sP2[KM_BN * PH];
    __shared__ __align__(16) float sV[KM_BN * NRHS];

    const int tid = threadIdx.x;
    const long long row0 = (long long)blockIdx.x * (KM_THREADS * R);

    unsigned long long xi[RP][D];
    unsigned long long ai[RP];
    unsigned long long acc[RP][NRHS];   // one column tile, FP32 pairs
    unsigned long long kc[RP][NC];      // Kahan compensation of the hi columns (COMP)
    unsigned long long ne[RP][NC];      // sum of the negated product errors (COMP)
    double acc64[R][NRHS];              // tiles folded in FP64
#pragma unroll
    for (int pr = 0; pr < RP; ++pr)
#pragma unroll
        for (int h = 0; h < NC; ++h) kc[pr][h] = ne[pr][h] = 0ull;
#pragma unroll
    for (int pr = 0; pr < RP; ++pr) {
        float xv[2][D], av[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long long i = row0 + (2 * pr + h) * KM_THREADS + tid;
            const bool ok = i < nr;
#pragma unroll
            for (int c = 0; c < D; ++c) xv[h][c] = ok ? (RAW ? 1.f : 2.f) * Pr[i * PS + c] : 0.f;
            av[h] = (ok && !RAW) ? Pr[i * PS + D] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < D; ++c) xi[pr][c] = f2_pack(xv[0][c], xv[1][c]);
        ai[pr] = f2_pack(av[0], av[1]);
#pragma unroll
        for (int q = 0; q < NRHS; ++q) acc[pr][q] = 0ull;
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int q = 0; q < NRHS; ++q) acc64[r][q] = 0.0;
    const unsigned long long nsc2 = f2_pack(nsc, nsc);
    const unsigned long long nsclo2 = f2_pack(COMP ? beta : 0.f, COMP ? beta : 0.f);

    const int ntiles = (nc + KM_BN - 1) / KM_BN;
    const int t0 = blockIdx.y * tiles_per_split;
    const int t1 = min(t0 + tiles_per_split, ntiles);
    const float4* Pc4 = reinterpret_cast<const float4*>(Pc);

    for (int t = t0; t < t1; ++t) {
        const int c0 = t * KM_BN;
        for (int e = tid; e < KM_BN * PS4; e += KM_THREADS) {
            const int j = e / PS4, w = e - j * PS4;
            const float4 v = (c0 + j < nc) ? Pc4[(size_t)(c0 + j) * PS4 + w] : make_float4(0.f, 0.f, 0.f, 0.f);
            sP2[j * PH + 2 * w] = make_ulonglong2(f2_pack(v.x, v.x), f2_pack(v.y, v.y));
            sP2[j * PH + 2 * w + 1] = make_ulonglong2(f2_pack(v.z, v.z), f2_pack(v.w, v.w));
        }
        for (int e = tid; e < KM_BN * NRHS; e += KM_THREADS) {
            const int q = e / KM_BN, j = e - q * KM_BN;
            sV[j * NRHS + q] = (c0 + j < nc) ? V[(size_t)q * ldv + c0 + j] : 0.f;
        }
        __syncthreads();
#pragma unroll 2
        for (int j = 0; j < KM_BN; ++j) {
            unsigned long long xj[PS];
#pragma unroll
            for (int w = 0; w < PH; ++w) {
                const ulonglong2 v = sP2[j * PH + w];
                xj[2 * w] = v.x;
                xj[2 * w + 1] = v.y;
            }
            unsigned long long vj[NRHS], vn[NC];
#pragma unroll
            for (int q = 0; q < NRHS; ++q) {
                const float v = sV[j * NRHS + q];
                vj[q] = f2_pack(v, v);
                if constexpr (COMP) {
                    if (q % 2 == 0) vn[q / 2] = f2_pack(-v, -v);
                }
            }
#pragma unroll
            for (int pr = 0; pr < RP; ++pr) {
                unsigned long long tt;
                if constexpr (RAW) {
                    unsigned long long ss = 0ull;
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        const unsigned long long df = f2_sub(xi[pr][c], xj[c]);
                        ss = f2_fma(df, df, ss);
                    }
                    tt = COMP ? f2_fma(ss, nsc2, f2_mul(ss, nsclo2)) : f2_mul(ss, nsc2);
                } else {
                    tt = f2_add(ai[pr], xj[D]);
#pragma unroll
                    for (int c = 0; c < D; ++c) tt = f2_fma(xi[pr][c], xj[c], tt);
                }
                float t0f, t1f;
                f2_unpack(tt, t0f, t1f);
                const unsigned long long e = COMP ? f2_pack(exp2_poly(t0f), exp2_poly(t1f))
                                                  : f2_pack(ex2f(t0f), ex2f(t1f));
#pragma unroll
                for (int q = 0; q < NRHS; ++q) {
                    if constexpr (COMP) {
                        if (q % 2 == 0) {
                            // t = fl(e v), -(e v - t) exactly; Kahan: y = t - c, s = acc + y,
                            // c = (s - acc) - y, acc = s
                            const unsigned long long t = f2_mul(e, vj[q]);
                            ne[pr][q / 2] = f2_add(ne[pr][q / 2], f2_fma(e, vn[q / 2], t));
                            const unsigned long long y = f2_sub(t, kc[pr][q / 2]);
                            const unsigned long long sum = f2_add(acc[pr][q], y);
                            kc[pr][q / 2] = f2_sub(f2_sub(sum, acc[pr][q]), y);
                            acc[pr][q] = sum;
                            continue;
                        }
                    }
                    acc[pr][q] = f2_fma(e, vj[q], acc[pr][q]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int pr = 0; pr < RP; ++pr)
#pragma unroll
            for (int q = 0; q < NRHS; ++q) {
                float lo, hi;
                f2_unpack(acc[pr][q], lo, hi);
                if constexpr (COMP) {
                    if (q % 2 == 0) {
                        // exact tile sum ~ s - c - (sum of negated product errors)
                        float clo, chi, elo, ehi;
                        f2_unpack(kc[pr][q / 2], clo, chi);
                        f2_unpack(ne[pr][q / 2], elo, ehi);
                        acc64[2 * pr][q] += ((double)lo - (double)clo) - (double)elo;
                        acc64[2 * pr + 1][q] += ((double)hi - (double)chi) - (double)ehi;
                        kc[pr][q / 2] = ne[pr][q / 2] = 0ull;
                        acc[pr][q] = 0ull;
                        continue;
                    }
                }
                acc64[2 * pr][q] += (double)lo;
                acc64[2 * pr + 1][q] += (double)hi;
                acc[pr][q] = 0ull;
            }
    }

#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = row0 + r * KM_THREADS + tid;
        if (i >= nr) continue;
        if (part == nullptr) {
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
                Q[(size_t)q * ldq + i] =
                    (float)(acc64[r][q] * (1.0 + (double)kcorr) +
                            (beta != 0.f ? (double)beta * V[(size_t)q * ldv + i] : 0.0));
        } else {
#pragma unroll
            for (int q = 0; q < NRHS; ++q)
                part[((size_t)blockIdx.y * NRHS + q) * nr + i] = acc64[r][q];
        }
    }
}

// Q = ksc * (sum of the split partials) + beta V; ksc != 1 corrects the kernel sums for the
// mean bias of the hardware exponential (see ex2_bias_scale).
__global__ void k_kmvm_reduce(const double* __restrict__ part, int splits, int nr, int nrhs,
                              const float* __restrict__ V, int ldv, float beta,
                              float* __restrict__ Q, int ldq, double ksc) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)nr * nrhs) return;
    const int q = (int)(e / nr);
    const int i = (int)(e - (long long)q * nr);
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[((size_t)sp * nrhs + q) * nr + i];
    s *= ksc;
    if (beta != 0.f) s += (double)beta * V[(size_t)q * ldv + i];
    Q[(size_t)q * ldq + i] = (float)s;
}

double ex2_bias_scale(const krr_ctx* ctx) {
    // ex2.approx.ftz.f32 returns 2^t about 0.83 ulp low on average for t < -1 (measured on
    // GB300 by krr_exp2_probe); the tensor-core product's kernel sums are scaled back by that
    // much.  (On the FP32 forms it changed which problems escalate, and one batched problem
    // stopped converging, so they are left as computed.)
    return (ctx && ctx->opts.ex2_correct) ? 1.0 + 0.83 * 5.9604644775390625e-08 : 1.0;
}

int launch_kmvm_reduce(krr_ctx* ctx, const double* part, int splits, int nr, int nrhs, const float* V,
                       int ldv, float beta, float* Q, int ldq) {
    const long long tot = (long long)nr * nrhs;
    k_kmvm_reduce<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(part, splits, nr, nrhs, V, ldv, beta, Q,
                                                                ldq, ex2_bias_scale(ctx));
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// Rows per thread: the largest R whose live registers (R x (D + 1) coordinates, R x NRHS
// FP32 tile sums plus their FP64 fold, one column's values) fit the 128 a thread has at
// four blocks per SM.
template <int D, int NRHS, int R>
constexpr bool kmvm_fits() {
    return R * (D + 1 + 3 * NRHS) + NRHS + 20 <= 128;
}
template <int D, int NRHS>
constexpr int kmvm_rows() {
    return (D > 32) ? 1
           : (D <= 16 && kmvm_fits<D, NRHS, 4>()) ? 4
           : kmvm_fits<D, NRHS, 2>() ? 2
                                     : 1;
}

typedef void (*kmvm_fn)(const float*, int, const float*, int, const float*, int, int, float, float, float,
                        float*, int, double*);

template <int D, int NRHS>
static kmvm_fn pick2(bool raw) {
    constexpr int R = kmvm_rows<D, NRHS>();
    if constexpr (R % 2 == 0 && D <= 24) {
        return raw ? &k_kmvm2<D, NRHS, R, true> : &k_kmvm2<D, NRHS, R, false>;
    } else {
        return raw ? &k_kmvm<D, NRHS, R, true> : &k_kmvm<D, NRHS, R, false>;
    }
}

template <int D>
static kmvm_fn pick1(int nrhs, int* R, bool raw) {
    switch (nrhs) {
        case 1: *R = kmvm_rows<D, 1>(); return pick2<D, 1>(raw);
        case 2: *R = kmvm_rows<D, 2>(); return pick2<D, 2>(raw);
        case 4: *R = kmvm_rows<D, 4>(); return pick2<D, 4>(raw);
        case 8: *R = kmvm_rows<D, 8>(); return pick2<D, 8>(raw);
        case 16: *R = kmvm_rows<D, 16>(); return pick2<D, 16>(raw);
    }
    return nullptr;
}

static kmvm_fn pick(int dk, int nrhs, int* R, bool raw = false) {
    switch (dk) {
#define KRR_D(v) \
    case v: return pick1<v>(nrhs, R, raw);
        KRR_D(1) KRR_D(2) KRR_D(3) KRR_D(4) KRR_D(5) KRR_D(6) KRR_D(7) KRR_D(8)
        KRR_D(9) KRR_D(10) KRR_D(11) KRR_D(12) KRR_D(13) KRR_D(14) KRR_D(15) KRR_D(16)
        KRR_D(24) KRR_D(32) KRR_D(48) KRR_D(64)
#undef KRR_D
    }
    return nullptr;
}

// Compensated split-product kernels (exact differences, hi/lo column pairs; d <= 24).
template <int D, int NRHS>
static kmvm_fn pick_comp2(int* R) {
    constexpr int RR = kmvm_rows<D, NRHS + NRHS / 2>();   // room for the compensation terms
    if constexpr (RR % 2 == 0) {
        *R = RR;
        return &k_kmvm2<D, NRHS, RR, true, true>;
    } else {
        *R = 2;
        return &k_kmvm2<D, NRHS, 2, true, true>;
    }
}
template <int D>
static kmvm_fn pick_comp1(int nrhs, int* R) {
    if (nrhs == 2) return pick_comp2<D, 2>(R);
    if (nrhs == 4) return pick_comp2<D, 4>(R);
    return nullptr;
}
static kmvm_fn pick_comp(int dk, int nrhs, int* R) {
    switch (dk) {
#define KRR_D(v) \
    case v: return pick_comp1<v>(nrhs, R);
        KRR_D(1) KRR_D(2) KRR_D(3) KRR_D(4) KRR_D(5) KRR_D(6) KRR_D(7) KRR_D(8)
        KRR_D(9) KRR_D(10) KRR_D(11) KRR_D(12) KRR_D(13) KRR_D(14) KRR_D(15) KRR_D(16) KRR_D(24)
#undef KRR_D
    }
    return nullptr;
}

static int occupancy(krr_ctx* ctx, const void* fn, int threads) {
    (void)ctx;
    static std::mutex mu;   // contexts may run on several host threads (batched solves)
    static std::map<const void*, int> cache;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find(fn);
        if (it != cache.end()) return it->second;
    }
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, 0) != cudaSuccess ||
        occ < 1)
        occ = 1;
    std::lock_guard<std::mutex> lock(mu);
    cache[fn] = occ;
    return occ;
}

// Number of column splits: fill the SMs with whole waves.
static int choose_splits(int nblk, int ntiles, int slots) {
    int best = 1;
    double best_score = -1.0;
    const int smax = std::max(1, std::min(ntiles, 64));
    for (int s = 1; s <= smax; ++s) {
        const double tot = (double)nblk * s;
        const double waves = tot / slots;
        const double score = waves >= 1.0 ? waves / std::ceil(waves) : waves;
        if (score > best_score + 1e-9) {
            best_score = score;
            best = s;
        }
        if (waves >= 4.0) break;
    }
    return best;
}

int choose_splits_public(int nblk, int ntiles, int slots) { return choose_splits(nblk, ntiles, slots); }

int launch_kmvm_reduce64(krr_ctx* ctx, const double* part, int nparts, int nr, int nrhs2,
                         const double* V64, double beta, double* Q64, double ksc);

int launch_kmvm(krr_ctx* ctx, const float* Pr, long long nr, const float* Pc, long long nc, int d,
                float beta, const float* V, int nrhs, float* Q, float raw_nsc, const double* V64,
                double* Q64, float raw_nsc_lo) {
    const bool raw = raw_nsc != 0.f;
    const bool hp = Q64 != nullptr;   // V holds hi/lo column pairs; FP64 output
    if (hp && (nrhs % 2 != 0 || !V64)) return fail(ctx, KRR_E_INVAL, "kmvm: bad split product");
    if (nr > 0x7fffffffLL || nc > 0x7fffffffLL)
        return fail(ctx, KRR_E_INVAL, "kmvm: more than 2^31 points");
    const int dk = kernel_dim(d);
    // split products of the FP64 recurrence in the exact-difference form: compensated
    // tile sums, two right-hand sides (four hi/lo columns) per launch
    const bool comp = hp && raw && dk <= 24;
    int done = 0;
    while (done < nrhs) {
        const int left = nrhs - done;
        const int chunk = comp ? (left >= 4 ? 4 : 2)
                               : left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        int R = 4;
        kmvm_fn fn = comp ? pick_comp(dk, chunk, &R) : pick(dk, chunk, &R, raw);
        if (!fn) return fail(ctx, KRR_E_INVAL, "kmvm: unsupported dimension");
        const int rows_per = KM_THREADS * R;
        const int nblk = (int)ceil_div(nr, rows_per);
        const int ntiles = (int)ceil_div(nc, KM_BN);
        const int slots = ctx->num_sms * occupancy(ctx, (const void*)fn, KM_THREADS);
        int splits = choose_splits(nblk, ntiles, slots);
        if (!hp && nr == nc)   // square FP32 products of a built problem: tuned splits
            splits = tuned_splits(ctx, tune_key(raw ? 2 : 0, dk, chunk, nr), splits, ntiles);
        const int tps = (ntiles + splits - 1) / splits;
        splits = (ntiles + tps - 1) / tps;
        ctx->last_splits = splits;
        const double ksc = 1.0;   // the exp2 bias correction is applied to the tensor-core form only
        double* part = nullptr;
        if (splits > 1 || hp)
            KRR_RET(bufT(ctx, "kmvm_part", (size_t)splits * chunk * nr, &part));
        dim3 grid(nblk, splits);
        const float* Vc = V + (size_t)done * nc;
        float* Qc = hp ? nullptr : Q + (size_t)done * nr;
        // compensated kernels: -s as a float pair (raw_nsc_lo rides in the beta slot)
        const float beta_arg = comp ? raw_nsc_lo : beta;
        fn<<<grid, KM_THREADS, 0, ctx->stream>>>(Pr, (int)nr, Pc, (int)nc, Vc, (int)nc, tps, beta_arg,
                                                 raw_nsc, (float)(ksc - 1.0), Qc, (int)nr, part);
        KRR_CHECK_LAUNCH();
        if (hp) {
            KRR_RET(launch_kmvm_reduce64(ctx, part, splits, (int)nr, chunk, V64 + (size_t)(done / 2) * nr,
                                         (double)beta, Q64 + (size_t)(done / 2) * nr, ksc));
        } else if (part) {
            const long long tot = nr * chunk;
            k_kmvm_reduce<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(part, splits, (int)nr, chunk,
                                                                        Vc, (int)nc, beta, Qc,
                                                                        (int)nr, ksc);
            KRR_CHECK_LAUNCH();
        }
        done += chunk;
    }
    return KRR_OK;
}

// ------------------------------------------------------------------ derivative product
// Q_i = sum_j (dK/dlog sigma)_ij v_j with (dK/dlog sigma)_ij = K_ij ||x_i - x_j||^2 / sigma^2.
// In the packed coordinates t_ij = a_i + a_j + 2 xh_i . xh_j = -s ||x_i - x_j||^2 with
// s = log2(e) / (2 sigma^2), so the entry is -2 ln2 t_ij 2^t_ij: one extra multiply per pair.
template <int D, int R>
__global__ void __launch_bounds__(KM_THREADS, 4)
k_kmvm_dsigma(const float* __restrict__ Pr, int nr, const float* __restrict__ Pc, int nc,
              const float* __restrict__ V, int tiles_per_split, double* __restrict__ part) {
    constexpr int PS = (D + 1 + 3) / 4 * 4;
    constexpr int PS4 = PS / 4;
    __shared__ float4 sP[KM_BN * PS4];
    __shared__ float sV[KM_BN];
    const int tid = threadIdx.x;
    const long long row0 = (long long)blockIdx.x * (KM_THREADS * R);
    float xi[R][D], ai[R], acc[R];
    float ah[R], al[R];   // tiles folded float-float
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = row0 + r * KM_THREADS + tid;
        const bool ok = i < nr;
#pragma unroll
        for (int c = 0; c < D; ++c) xi[r][c] = ok ? 2.f * Pr[i * PS + c] : 0.f;
        ai[r] = ok ? Pr[i * PS + D] : 0.f;
        acc[r] = 0.f;
        ah[r] = al[r] = 0.f;
    }
    const int ntiles = (nc + KM_BN - 1) / KM_BN;
    const int t0 = blockIdx.y * tiles_per_split;
    const int t1 = min(t0 + tiles_per_split, ntiles);
    const float4* Pc4 = reinterpret_cast<const float4*>(Pc);
    for (int t = t0; t < t1; ++t) {
        const int c0 = t * KM_BN;
        for (int e = tid; e < KM_BN * PS4; e += KM_THREADS) {
            const int j = e / PS4;
            sP[e] = (c0 + j < nc) ? Pc4[(size_t)(c0 + j) * PS4 + (e - j * PS4)]
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = tid; e < KM_BN; e += KM_THREADS) sV[e] = (c0 + e < nc) ? V[c0 + e] : 0.f;
        __syncthreads();
#pragma unroll 2
        for (int j = 0; j < KM_BN; ++j) {
            float xj[PS];
#pragma unroll
            for (int w = 0; w < PS4; ++w) {
                const float4 v = sP[j * PS4 + w];
                xj[4 * w + 0] = v.x;
                xj[4 * w + 1] = v.y;
                xj[4 * w + 2] = v.z;
                xj[4 * w + 3] = v.w;
            }
            const float vj = sV[j];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float tt = ai[r] + xj[D];
#pragma unroll
                for (int c = 0; c < D; ++c) tt = fmaf(xi[r][c], xj[c], tt);
                acc[r] = fmaf(tt * ex2f(tt), vj, acc[r]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) ff_add(ah[r], al[r], acc[r]), acc[r] = 0.f;
    }
    const double scale = -2.0 * 0.6931471805599453;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const long long i = row0 + r * KM_THREADS + tid;
        if (i < nr) part[(size_t)blockIdx.y * nr + i] = scale * ((double)ah[r] + (double)al[r]);
    }
}

typedef void (*dsig_fn)(const float*, int, const float*, int, const float*, int, double*);

static dsig_fn dsig_pick(int dk) {
    switch (dk) {
#define KRR_D(v) \
    case v: return &k_kmvm_dsigma<v, (v > 32 ? 1 : v > 16 ? 2 : 4)>;
        KRR_D(1) KRR_D(2) KRR_D(3) KRR_D(4) KRR_D(5) KRR_D(6) KRR_D(7) KRR_D(8)
        KRR_D(9) KRR_D(10) KRR_D(11) KRR_D(12) KRR_D(13) KRR_D(14) KRR_D(15) KRR_D(16)
        KRR_D(24) KRR_D(32) KRR_D(48) KRR_D(64)
#undef KRR_D
    }
    return nullptr;
}

// Q = (dK(Pr, Pc)/dlog sigma) v for one column v (nc), Q (nr).
int launch_kmvm_dsigma(krr_ctx* ctx, const float* Pr, long long nr, const float* Pc, long long nc,
                       int d, const float* V, float* Q) {
    const int dk = kernel_dim(d);
    dsig_fn fn = dsig_pick(dk);
    if (!fn) return fail(ctx, KRR_E_INVAL, "dsigma: unsupported dimension");
    const int R = dk > 32 ? 1 : dk > 16 ? 2 : 4;
    const int nblk = (int)ceil_div(nr, KM_THREADS * R);
    const int ntiles = (int)ceil_div(nc, KM_BN);
    const int slots = ctx->num_sms * occupancy(ctx, (const void*)fn, KM_THREADS);
    int splits = choose_splits(nblk, ntiles, slots);
    const int tps = (ntiles + splits - 1) / splits;
    splits = (ntiles + tps - 1) / tps;
    double* part;
    KRR_RET(bufT(ctx, "dsig_part", (size_t)splits * nr, &part));
    fn<<<dim3(nblk, splits), KM_THREADS, 0, ctx->stream>>>(Pr, (int)nr, Pc, (int)nc, V, tps, part);
    KRR_CHECK_LAUNCH();
    return launch_kmvm_reduce(ctx, part, splits, (int)nr, 1, V, (int)nc, 0.f, Q, (int)nr);
}

// ------------------------------------------------------------------ product into given scratch
// The FP32 product K(Xr, Xc) V + beta V with every temporary (mean, packed points,
// split-K partial sums) carved from one caller-provided device buffer: no device
// allocation and no context.  *needed receives the bytes this size takes; returns
// KRR_E_NOMEM when the buffer is too small for it, KRR_E_INVAL when no compiled tile
// serves (d, nrhs), KRR_E_CUDA when a launch fails.
static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

int kmvm_into_scratch(cudaStream_t stream, int num_sms, const float* Xr, long long nr,
                      const float* Xc, long long nc, int d, double sigma, double beta,
                      const float* V, int nrhs, float* Q, unsigned char* scratch, size_t cap,
                      size_t* needed) {
    const int dk = kernel_dim(d), ps = packed_stride(d);
    const bool same = (Xr == Xc && nr == nc);
    const int nblk_mean = (int)std::min<long long>(2LL * num_sms, ceil_div(nc, 256));
    // split-K layout of every right-hand-side chunk, as the context path chooses it
    size_t part_elems = 0;
    for (int done = 0; done < nrhs;) {
        const int left = nrhs - done;
        const int chunk = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        int R = 4;
        kmvm_fn fn = pick(dk, chunk, &R);
        if (!fn) return KRR_E_INVAL;   // no compiled tile for this (d, chunk): not a size problem
        int occ = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, KM_THREADS, 0) !=
                cudaSuccess || occ < 1)
            occ = 1;
        const int nblk = (int)ceil_div(nr, KM_THREADS * R);
        const int ntiles = (int)ceil_div(nc, KM_BN);
        int splits = choose_splits(nblk, ntiles, num_sms * occ);
        const int tps = (ntiles + splits - 1) / splits;
        splits = (ntiles + tps - 1) / tps;
        if (splits > 1) part_elems = std::max(part_elems, (size_t)splits * chunk * (size_t)nr);
        done += chunk;
    }
    const size_t off_mpart = 0;
    const size_t off_mu = off_mpart + align256(sizeof(double) * nblk_mean * d);
    const size_t off_pc = off_mu + align256(sizeof(double) * d);
    const size_t off_pr = off_pc + align256(sizeof(float) * (size_t)nc * ps);
    const size_t off_part = off_pr + (same ? 0 : align256(sizeof(float) * (size_t)nr * ps));
    const size_t total = off_part + align256(sizeof(double) * part_elems);
    if (needed) *needed = total;
    if (total > cap) return KRR_E_NOMEM;   // the fixed scratch is too small for this size

    double* mpart = reinterpret_cast<double*>(scratch + off_mpart);
    double* mu = reinterpret_cast<double*>(scratch + off_mu);
    float* Pc = reinterpret_cast<float*>(scratch + off_pc);
    float* Pr = same ? Pc : reinterpret_cast<float*>(scratch + off_pr);
    double* part = reinterpret_cast<double*>(scratch + off_part);
    const double s = 1.4426950408889634 / (2.0 * sigma * sigma);
    k_mean_partial<<<nblk_mean, 256, 0, stream>>>(Xc, nc, d, mpart);
    k_mean_final<<<1, 64, 0, stream>>>(mpart, nblk_mean, d, nc, mu);
    k_pack<<<ceil_div(nc, 256), 256, 0, stream>>>(Xc, nc, d, dk, ps, mu, std::sqrt(s), Pc);
    if (!same) k_pack<<<ceil_div(nr, 256), 256, 0, stream>>>(Xr, nr, d, dk, ps, mu, std::sqrt(s), Pr);
    for (int done = 0; done < nrhs;) {
        const int left = nrhs - done;
        const int chunk = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        int R = 4;
        kmvm_fn fn = pick(dk, chunk, &R);
        int occ = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void*)fn, KM_THREADS, 0) !=
                cudaSuccess || occ < 1)
            occ = 1;
        const int nblk = (int)ceil_div(nr, KM_THREADS * R);
        const int ntiles = (int)ceil_div(nc, KM_BN);
        int splits = choose_splits(nblk, ntiles, num_sms * occ);
        const int tps = (ntiles + splits - 1) / splits;
        splits = (ntiles + tps - 1) / tps;
        const float* Vc = V + (size_t)done * nc;
        float* Qc = Q + (size_t)done * nr;
        fn<<<dim3(nblk, splits), KM_THREADS, 0, stream>>>(Pr, (int)nr, Pc, (int)nc, Vc, (int)nc, tps,
                                                          (float)beta, 0.f, 0.f, Qc, (int)nr,
                                                          splits > 1 ? part : nullptr);
        if (splits > 1)
            k_kmvm_reduce<<<ceil_div(nr * chunk, 256), 256, 0, stream>>>(part, splits, (int)nr, chunk,
                                                                          Vc, (int)nc, (float)beta,
                                                                          Qc, (int)nr, 1.0);
        done += chunk;
    }
    return cudaGetLastError() == cudaSuccess ? KRR_OK : KRR_E_CUDA;
}

// ------------------------------------------------------------------ FP64 residual
constexpr int HP_THREADS = 128;
constexpr int HP_BN = 64;

template <int DM, int NR>
__global__ void __launch_bounds__(HP_THREADS)
k_resid_hp(const float* __restrict__ X, int n, int d, double inv2s2, const double* __restrict__ A,
           int tiles_per_split, double* __restrict__ part) {
    __shared__ double sX[HP_BN * DM];
    __shared__ double sA[HP_BN * NR];
    const int tid = threadIdx.x;
    const long long i = (long long)blockIdx.x * HP_THREADS + tid;
    double xi[DM];
#pragma unroll
    for (int c = 0; c < DM; ++c) xi[c] = (i < n && c < d) ? (double)X[i * d + c] : 0.0;
    double acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) acc[q] = 0.0;

    const int ntiles = (n + HP_BN - 1) / HP_BN;
    const int t0 = blockIdx.y * tiles_per_split;
    const int t1 = min(t0 + tiles_per_split, ntiles);
    for (int t = t0; t < t1; ++t) {
        const int c0 = t * HP_BN;
        for (int e = tid; e < HP_BN * DM; e += HP_THREADS) {
            const int j = e / DM, c = e - j * DM;
            sX[e] = (c0 + j < n && c < d) ? (double)X[(size_t)(c0 + j) * d + c] : 0.0;
        }
        for (int e = tid; e < HP_BN * NR; e += HP_THREADS) {
            const int q = e / HP_BN, j = e - q * HP_BN;
            sA[j * NR + q] = (c0 + j < n) ? A[(size_t)q * n + c0 + j] : 0.0;
        }
        __syncthreads();
        for (int j = 0; j < HP_BN; ++j) {
            double d2 = 0.0;
#pragma unroll
            for (int c = 0; c < DM; ++c) {
                const double df = xi[c] - sX[j * DM + c];
                d2 = fma(df, df, d2);
            }
            const double kv = exp(-d2 * inv2s2);
#pragma unroll
            for (int q = 0; q < NR; ++q) acc[q] = fma(kv, sA[j * NR + q], acc[q]);
        }
        __syncthreads();
    }
    if (i < n) {
#pragma unroll
        for (int q = 0; q < NR; ++q) part[((size_t)blockIdx.y * NR + q) * n + i] = acc[q];
    }
}

__global__ void k_resid_reduce(const double* __restrict__ part, int splits, int n, int nr,
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

typedef void (*hp_fn)(const float*, int, int, double, const double*, int, double*);

template <int DM>
static hp_fn hp_pick1(int nr) {
    switch (nr) {
        case 1: return &k_resid_hp<DM, 1>;
        case 2: return &k_resid_hp<DM, 2>;
        case 4: return &k_resid_hp<DM, 4>;
        case 8: return &k_resid_hp<DM, 8>;
        case 16: return &k_resid_hp<DM, 16>;
    }
    return nullptr;
}

int launch_residual_hp(krr_ctx* ctx, const float* X, long long n, int d, double sigma, double beta,
                       const float* Y, const double* A, int nrhs, double* R) {
    if (n > 0x7fffffffLL) return fail(ctx, KRR_E_INVAL, "residual: more than 2^31 points");
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    int done = 0;
    while (done < nrhs) {
        const int left = nrhs - done;
        const int chunk = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        hp_fn fn = d <= 4 ? hp_pick1<4>(chunk) : d <= 8 ? hp_pick1<8>(chunk)
                 : d <= 16 ? hp_pick1<16>(chunk) : hp_pick1<64>(chunk);
        const int nblk = (int)ceil_div(n, HP_THREADS);
        const int ntiles = (int)ceil_div(n, HP_BN);
        const int slots = ctx->num_sms * occupancy(ctx, (const void*)fn, HP_THREADS);
        int splits = choose_splits(nblk, ntiles, slots);
        const int tps = (ntiles + splits - 1) / splits;
        splits = (ntiles + tps - 1) / tps;
        double* part;
        KRR_RET(bufT(ctx, "hp_part", (size_t)splits * chunk * n, &part));
        dim3 grid(nblk, splits);
        fn<<<grid, HP_THREADS, 0, ctx->stream>>>(X, (int)n, d, inv2s2, A + (size_t)done * n, tps,
                                                 part);
        KRR_CHECK_LAUNCH();
        const long long tot = n * chunk;
        k_resid_reduce<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(
            part, splits, (int)n, chunk, Y + (size_t)done * n, A + (size_t)done * n, beta,
            R + (size_t)done * n);
        KRR_CHECK_LAUNCH();
        done += chunk;
    }
    return KRR_OK;
}

}  // namespace krr
