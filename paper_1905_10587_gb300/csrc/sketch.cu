// Algorithm 1 step 1-2 (the Gaussian test matrix and the sketch Y = K Omega^T),
// the contraction F = K(X, X_S) W used by Algorithm 3, and the Gram matrix
// G = beta I + F^T F of Eq. (10).
//
// The two contractions have the shape of a GEMM whose left operand is produced on
// the fly: each K-step generates a BK x BM tile of kernel values exp2(a_i + a_j +
// 2 xh_i . xh_j) into shared memory and multiplies it with a BK x BN tile of the
// right operand, with an 8 x 8 register tile per thread (FP32 SIMT).
#include "internal.cuh"

#include <algorithm>
#include <cuda_bf16.h>

namespace krr {

// ------------------------------------------------------------------ Philox / Omega
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64
// multiplications with the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// OmT[j * ld + a] = omega_{a, j}; entries with l <= a < ld are zero.
__global__ void k_omega(unsigned long long seed, int l, long long n, int ld,
                        float* __restrict__ OmT) {
    const int half = ld / 2;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * half) return;
    const long long j = e / half;
    const int c = (int)(e - j * half);
    float z0 = 0.f, z1 = 0.f;
    if (2 * c < l) {
        const uint4 r = philox4x32_10(
            make_uint4((unsigned)(j & 0xffffffffu), (unsigned)(j >> 32), (unsigned)c, 0u),
            make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)));
        const float u1 = (float)((r.x >> 8) + 1u) * 0x1p-24f;
        const float u2 = (float)(r.y >> 8) * 0x1p-24f;
        const float rad = sqrtf(-2.f * logf(u1));
        float sn, cs;
        sincospif(2.f * u2, &sn, &cs);
        z0 = rad * cs;
        z1 = (2 * c + 1 < l) ? rad * sn : 0.f;
    }
    float* o = OmT + j * ld + 2 * c;
    if (ld % 2 == 0) {
        *reinterpret_cast<float2*>(o) = make_float2(z0, z1);
    }
}

__global__ void k_omega_exact(unsigned long long seed, int l, long long n, float* __restrict__ OmT) {
    // exact-stride variant for odd l (ABI output)
    const int half = (l + 1) / 2;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * half) return;
    const long long j = e / half;
    const int c = (int)(e - j * half);
    const uint4 r = philox4x32_10(
        make_uint4((unsigned)(j & 0xffffffffu), (unsigned)(j >> 32), (unsigned)c, 0u),
        make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)));
    const float u1 = (float)((r.x >> 8) + 1u) * 0x1p-24f;
    const float u2 = (float)(r.y >> 8) * 0x1p-24f;
    const float rad = sqrtf(-2.f * logf(u1));
    float sn, cs;
    sincospif(2.f * u2, &sn, &cs);
    OmT[j * l + 2 * c] = rad * cs;
    if (2 * c + 1 < l) OmT[j * l + 2 * c + 1] = rad * sn;
}

// The same Omega rounded to BF16 and laid out for the tensor-core sketch: tiles of
// 256 projections x 64 points in the core-matrix order (8 rows x 16 bytes per
// 128-byte block; row = projection a, K = point j), tile (ab, jc) at byte offset
// (ab * njc + jc) * 32 KB.  Entries with a >= l or j >= n are zero.
__global__ void k_omega_bf16_tiled(unsigned long long seed, int l, long long n, int nab, int njc,
                                   __nv_bfloat16* __restrict__ out) {
    const long long npad = (long long)njc * 64;
    const int half = nab * 128;                       // pairs of projections
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npad * half) return;
    const long long j = e / half;
    const int c = (int)(e - j * half);
    float z0 = 0.f, z1 = 0.f;
    if (j < n && 2 * c < l) {
        const uint4 r = philox4x32_10(
            make_uint4((unsigned)(j & 0xffffffffu), (unsigned)(j >> 32), (unsigned)c, 0u),
            make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)));
        const float u1 = (float)((r.x >> 8) + 1u) * 0x1p-24f;
        const float u2 = (float)(r.y >> 8) * 0x1p-24f;
        const float rad = sqrtf(-2.f * logf(u1));
        float sn, cs;
        sincospif(2.f * u2, &sn, &cs);
        z0 = rad * cs;
        z1 = (2 * c + 1 < l) ? rad * sn : 0.f;
    }
    const int jc = (int)(j >> 6), jl = (int)(j & 63);
    for (int u = 0; u < 2; ++u) {
        const int a = 2 * c + u;
        const int ab = a >> 8, al = a & 255;
        const size_t tile = ((size_t)ab * njc + jc) * (256 * 64);
        const size_t off = (size_t)(((al >> 3) * 8 + (jl >> 3)) * 64 + (al & 7) * 8 + (jl & 7));
        out[tile + off] = __float2bfloat16_rn(u ? z1 : z0);
    }
}

int launch_omega_bf16_tiled(krr_ctx* ctx, unsigned long long seed, int l, long long n, int nab,
                            int njc, void* out) {
    const long long tot = (long long)njc * 64 * nab * 128;
    k_omega_bf16_tiled<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(seed, l, n, nab, njc,
                                                                    static_cast<__nv_bfloat16*>(out));
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

int launch_omega(krr_ctx* ctx, unsigned long long seed, int l, long long n, int ld, float* OmT) {
    if (ld % 2 == 0) {
        const long long tot = n * (ld / 2);
        k_omega<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(seed, l, n, ld, OmT);
    } else {
        if (ld != l) return fail(ctx, KRR_E_INVAL, "omega: odd padded stride");
        const long long tot = n * ((l + 1) / 2);
        k_omega_exact<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(seed, l, n, OmT);
    }
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// ------------------------------------------------------------------ Algorithm 2 sketch
// The draws of Algorithm 2, steps 3-4: for projection i and entry m, Philox4x32-10 with
// counter (i, m, 0x53505253, 0) and key (seed lo, seed hi); the row index is the high
// word of r0 * n and the sign is - when the top bit of r1 is set.  Indices are drawn
// independently (a repeat counts twice).  R, S: l x r.
__global__ void k_sparse_draw(unsigned long long seed, int l, int r, long long n, int* __restrict__ R,
                              float* __restrict__ S) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)l * r) return;
    const unsigned i = (unsigned)(e / r), m = (unsigned)(e - (long long)i * r);
    const uint4 w = philox4x32_10(make_uint4(i, m, 0x53505253u, 0u),
                                  make_uint2((unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)));
    R[e] = (int)(((unsigned long long)w.x * (unsigned long long)n) >> 32);
    S[e] = (w.y >> 31) ? -1.f : 1.f;
}

int launch_sparse_draw(krr_ctx* ctx, unsigned long long seed, int l, int r, long long n, int* R, float* S) {
    const long long tot = (long long)l * r;
    k_sparse_draw<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(seed, l, r, n, R, S);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// Algorithm 2, steps 5-6: Y[j * ldy + i] = sum_m K(x_j, x_{R[i, m]}) S[i, m] from the packed
// points P (expansion form, as the Gaussian sketch).  A CTA takes 128 rows and `lc`
// projections: the lc x r gathered points sit in shared memory, each thread sums its
// row's lc outputs, and the 128 x lc block leaves through shared memory row by row.
constexpr int SP_THREADS = 128;
__global__ void __launch_bounds__(SP_THREADS)
k_sparse_sketch(const float* __restrict__ P, long long n, int dk, int ps, const int* __restrict__ R,
                const float* __restrict__ S, int l, int r, int lc, float* __restrict__ Y, int ldy) {
    extern __shared__ float ssp[];
    float* sG = ssp;                           // lc * r * ps gathered points
    float* sS = sG + (size_t)lc * r * ps;      // lc * r signs
    float* sO = sS + (size_t)lc * r;           // SP_THREADS x (lc + 1) outputs
    const int tid = threadIdx.x;
    const int i0 = blockIdx.y * lc;
    const int nl = min(lc, l - i0);
    for (int e = tid; e < nl * r; e += SP_THREADS) {
        const long long src = R[(size_t)i0 * r + e];
        for (int c = 0; c < ps; ++c) sG[(size_t)e * ps + c] = P[src * ps + c];
        sS[e] = S[(size_t)i0 * r + e];
    }
    __syncthreads();
    const long long j = (long long)blockIdx.x * SP_THREADS + tid;
    if (j < n) {
        const float* xj = P + j * ps;
        const float aj = xj[dk];
        for (int ii = 0; ii < nl; ++ii) {
            float acc = 0.f;
            for (int m = 0; m < r; ++m) {
                const float* g = sG + (size_t)(ii * r + m) * ps;
                float t = aj + g[dk];
                for (int c = 0; c < dk; ++c) t = fmaf(2.f * xj[c], g[c], t);
                acc = fmaf(ex2f(t), sS[ii * r + m], acc);
            }
            sO[tid * (lc + 1) + ii] = acc;
        }
    }
    __syncthreads();
    // row by row: lanes write consecutive projections of one row
    const int lane = tid & 31, w = tid >> 5;
    for (int rr = w; rr < SP_THREADS; rr += SP_THREADS / 32) {
        const long long row = (long long)blockIdx.x * SP_THREADS + rr;
        if (row >= n) continue;
        for (int ii = lane; ii < nl; ii += 32) Y[row * ldy + i0 + ii] = sO[rr * (lc + 1) + ii];
    }
}

int launch_sparse_sketch(krr_ctx* ctx, const float* P, long long n, int d, const int* R, const float* S,
                         int l, int r, float* Y, int ldy) {
    const int dk = kernel_dim(d), ps = packed_stride(d);
    // projections per CTA: as many as 40 KB of shared memory hold (at most 32)
    const size_t per = (size_t)r * ps * 4 + (size_t)r * 4 + (size_t)SP_THREADS * 4;
    int lc = (int)std::max<size_t>(1, std::min<size_t>(32, (40u << 10) / per));
    lc = std::min(lc, l);
    const size_t smem = (size_t)lc * per + (size_t)SP_THREADS * 4;
    if (smem > (48u << 10)) return fail(ctx, KRR_E_INVAL, "sparse sketch: r too large for this d");
    dim3 grid((unsigned)ceil_div(n, SP_THREADS), (unsigned)ceil_div(l, lc));
    k_sparse_sketch<<<grid, SP_THREADS, smem, ctx->stream>>>(P, n, dk, ps, R, S, l, r, lc, Y, ldy);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// ------------------------------------------------------------------ generated-operand GEMM
constexpr int KG_THREADS = 256;
constexpr int KG_BM = 128, KG_BN = 128, KG_BK = 16;

// Out[i * ldo + a] = sum_j K(Pr_i, Pc_j) V[j * ldv + a]  for i < nr, a < ncol.
template <int D>
__global__ void __launch_bounds__(KG_THREADS)
k_kgemm(const float* __restrict__ Pr, int nr, const float* __restrict__ Pc, int nc,
        const float* __restrict__ V, int ldv, int ncol, float* __restrict__ Out, int ldo) {
    constexpr int PS = (D + 1 + 3) / 4 * 4;
    __shared__ float sXr[PS][KG_BM];                  // row points, coordinate-major
    __shared__ float sXc[KG_BK][PS];
    __shared__ __align__(16) float sPt[KG_BK][KG_BM];   // kernel tile, transposed
    __shared__ __align__(16) float sV[KG_BK][KG_BN];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const long long row0 = (long long)blockIdx.y * KG_BM;
    const int col0 = blockIdx.x * KG_BN;

    for (int e = tid; e < KG_BM * PS; e += KG_THREADS) {
        const int i = e / PS, c = e - i * PS;
        float v = (row0 + i < nr) ? Pr[(row0 + i) * PS + c] : 0.f;
        if (c < D) v *= 2.f;
        sXr[c][i] = v;
    }

    float acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

    const bool vec = (ldv % 4 == 0);
    for (int j0 = 0; j0 < nc; j0 += KG_BK) {
        for (int e = tid; e < KG_BK * PS; e += KG_THREADS) {
            const int kk = e / PS, c = e - kk * PS;
            sXc[kk][c] = (j0 + kk < nc) ? Pc[(size_t)(j0 + kk) * PS + c] : 0.f;
        }
        if (vec) {
            for (int e = tid; e < KG_BK * KG_BN / 4; e += KG_THREADS) {
                const int kk = e / (KG_BN / 4), c4 = (e - kk * (KG_BN / 4)) * 4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j0 + kk < nc) {
                    const float* src = V + (size_t)(j0 + kk) * ldv + col0 + c4;
                    if (col0 + c4 + 3 < ncol) {
                        v = *reinterpret_cast<const float4*>(src);
                    } else {
                        if (col0 + c4 + 0 < ncol) v.x = src[0];
                        if (col0 + c4 + 1 < ncol) v.y = src[1];
                        if (col0 + c4 + 2 < ncol) v.z = src[2];
                    }
                }
                *reinterpret_cast<float4*>(&sV[kk][c4]) = v;
            }
        } else {
            for (int e = tid; e < KG_BK * KG_BN; e += KG_THREADS) {
                const int kk = e / KG_BN, c = e - kk * KG_BN;
                sV[kk][c] = (j0 + kk < nc && col0 + c < ncol) ? V[(size_t)(j0 + kk) * ldv + col0 + c]
                                                               : 0.f;
            }
        }
        __syncthreads();
        for (int e = tid; e < KG_BK * KG_BM; e += KG_THREADS) {
            const int kk = e / KG_BM, i = e - kk * KG_BM;
            float t = sXr[D][i] + sXc[kk][D];
#pragma unroll
            for (int c = 0; c < D; ++c) t = fmaf(sXr[c][i], sXc[kk][c], t);
            sPt[kk][i] = (j0 + kk < nc) ? ex2f(t) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KG_BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sPt[kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sPt[kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sV[kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sV[kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const long long i = row0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
        if (i >= nr) continue;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int a = col0 + (c < 4 ? tx * 4 + c : 64 + tx * 4 + c - 4);
            if (a < ncol) Out[i * ldo + a] = acc[r][c];
        }
    }
}

typedef void (*kgemm_fn)(const float*, int, const float*, int, const float*, int, int, float*,
                         int);

static kgemm_fn kgemm_pick(int dk) {
    switch (dk) {
#define KRR_D(v) \
    case v: return &k_kgemm<v>;
        KRR_D(1) KRR_D(2) KRR_D(3) KRR_D(4) KRR_D(5) KRR_D(6) KRR_D(7) KRR_D(8)
        KRR_D(9) KRR_D(10) KRR_D(11) KRR_D(12) KRR_D(13) KRR_D(14) KRR_D(15) KRR_D(16)
        KRR_D(24) KRR_D(32) KRR_D(48) KRR_D(64)
#undef KRR_D
    }
    return nullptr;
}

int launch_kgemm(krr_ctx* ctx, const float* Pr, long long nr, const float* Pc, long long nc, int d,
                 const float* V, int ldv, int ncol, float* Out, int ldo) {
    if (nr > 0x7fffffffLL || nc > 0x7fffffffLL)
        return fail(ctx, KRR_E_INVAL, "kgemm: more than 2^31 points");
    kgemm_fn fn = kgemm_pick(kernel_dim(d));
    if (!fn) return fail(ctx, KRR_E_INVAL, "kgemm: unsupported dimension");
    dim3 grid(ceil_div(ncol, KG_BN), ceil_div(nr, KG_BM));
    if (grid.y > 65535u) return fail(ctx, KRR_E_INVAL, "kgemm: too many row blocks");
    fn<<<grid, KG_THREADS, 0, ctx->stream>>>(Pr, (int)nr, Pc, (int)nc, V, ldv, ncol, Out, ldo);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// ------------------------------------------------------------------ Gram  G = beta I + F^T F
constexpr int GR_THREADS = 256, GR_B = 64, GR_BK = 32, GR_FOLD = 256;

// One CTA: a 64x64 block (ba, bb), ba >= bb, of F^T F over rows [r0, r1).
// Products are summed in FP32 over GR_FOLD rows and folded into FP64.
__global__ void __launch_bounds__(GR_THREADS)
k_gram(const float* __restrict__ F, long long n, int k, int ldF, const int2* __restrict__ pairs,
       long long rows_per_split, double* __restrict__ part) {
    __shared__ __align__(16) float sA[GR_BK][GR_B];
    __shared__ __align__(16) float sB[GR_BK][GR_B];
    const int2 pr = pairs[blockIdx.x];
    const int a0 = pr.x * GR_B, b0 = pr.y * GR_B;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long r0 = (long long)blockIdx.y * rows_per_split;
    const long long r1 = min(n, r0 + rows_per_split);
    float acc[4][4];
    double acc64[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f, acc64[r][c] = 0.0;
    int since_fold = 0;
    for (long long i0 = r0; i0 < r1; i0 += GR_BK) {
        for (int e = tid; e < GR_BK * GR_B; e += GR_THREADS) {
            const int kk = e / GR_B, c = e - kk * GR_B;
            const long long i = i0 + kk;
            const bool ok = i < r1;
            sA[kk][c] = (ok && a0 + c < k) ? F[i * ldF + a0 + c] : 0.f;
            sB[kk][c] = (ok && b0 + c < k) ? F[i * ldF + b0 + c] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GR_BK; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(&sA[kk][ty * 4]);
            const float4 bv = *reinterpret_cast<const float4*>(&sB[kk][tx * 4]);
            const float a[4] = {av.x, av.y, av.z, av.w};
            const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
        since_fold += GR_BK;
        if (since_fold >= GR_FOLD) {
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc64[r][c] += (double)acc[r][c], acc[r][c] = 0.f;
            since_fold = 0;
        }
    }
    double* out = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * GR_B * GR_B;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            out[(ty * 4 + r) * GR_B + tx * 4 + c] = acc64[r][c] + (double)acc[r][c];
}

__global__ void k_gram_reduce(const double* __restrict__ part, int splits, int npairs,
                              const int2* __restrict__ pairs, int k, double beta,
                              double* __restrict__ G) {
    const int p = blockIdx.x;
    const int2 pr = pairs[p];
    for (int e = threadIdx.x; e < GR_B * GR_B; e += blockDim.x) {
        const int r = e / GR_B, c = e - r * GR_B;
        const int a = pr.x * GR_B + r, b = pr.y * GR_B + c;
        if (a >= k || b >= k) continue;
        double s = 0.0;
        for (int sp = 0; sp < splits; ++sp) s += part[((size_t)sp * npairs + p) * GR_B * GR_B + e];
        if (a == b) s += beta;
        G[(size_t)a * k + b] = s;
        G[(size_t)b * k + a] = s;
    }
}

int launch_gram(krr_ctx* ctx, const float* F, long long n, int k, int ldF, double beta, double* G) {
    const int nb = (k + GR_B - 1) / GR_B;
    const int npairs = nb * (nb + 1) / 2;
    int2* pairs;
    KRR_RET(bufT(ctx, "gram_pairs", (size_t)npairs, &pairs));
    {
        int2* hp = new int2[npairs];
        int p = 0;
        for (int a = 0; a < nb; ++a)
            for (int b = 0; b <= a; ++b) hp[p++] = make_int2(a, b);
        cudaError_t e = cudaMemcpyAsync(pairs, hp, sizeof(int2) * npairs, cudaMemcpyHostToDevice,
                                        ctx->stream);
        cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
        delete[] hp;
        if (e != cudaSuccess || e2 != cudaSuccess)
            return fail(ctx, KRR_E_CUDA, "gram: pair table upload failed");
    }
    const int target = 3 * ctx->num_sms * 2;
    int splits = (int)std::max<long long>(1, std::min<long long>(target / npairs + 1, ceil_div(n, 4 * GR_FOLD)));
    const long long rps = ((ceil_div(n, splits) + GR_BK - 1) / GR_BK) * GR_BK;
    splits = (int)ceil_div(n, rps);
    double* part;
    KRR_RET(bufT(ctx, "gram_part", (size_t)splits * npairs * GR_B * GR_B, &part));
    dim3 grid(npairs, splits);
    k_gram<<<grid, GR_THREADS, 0, ctx->stream>>>(F, n, k, ldF, pairs, rps, part);
    KRR_CHECK_LAUNCH();
    k_gram_reduce<<<npairs, 256, 0, ctx->stream>>>(part, splits, npairs, pairs, k, beta, G);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

}  // namespace krr
