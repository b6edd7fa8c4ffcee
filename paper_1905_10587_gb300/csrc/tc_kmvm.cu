// Tensor-core (tcgen05) kernel product for sm_103a.
//
// The exponent of every pair is an inner product: with xh = (x - mu) sqrt(s) and
// a = -||xh||^2, t_ij = 2 xh_i . xh_j + a_i + a_j = -s ||x_i - x_j||^2 (log2 units).
// Each FP32 value v is split into three BF16 pieces v = h + m + l (24 significant
// bits), and t_ij is one BF16 GEMM over an augmented K dimension:
//     row i    : [2h, 2h, 2m, 2h, 2m, 2l]_c ... , a1, a2, a3, 1, 1, 1
//     column j : [ H,  M,  H,  L,  M,  H]_c ... ,  1,  1,  1, A1, A2, A3
// (the products hH + hM + mH + hL + mM + lH keep every term above 2^-24 relative).
// A work item is 128 rows (one M = 128 MMA) against a range of 256-column tiles:
// features arrive by cp.async.bulk on an mbarrier, tcgen05.mma accumulates t into
// TMEM (two 256-column buffers, so the MMA of tile t+1 overlaps the epilogue of tile
// t), and the epilogue reads TMEM with tcgen05.ld and does one ex2 (MUFU) per pair and
// one FFMA per pair and right-hand side, or, with one right-hand side folded into the
// exponent, one add.  With many right-hand sides the contraction runs as a second
// tcgen05 MMA (k_kmvm_tcpv below).  Every wait is bounded; on timeout the kernel sets
// an error word, stops issuing work, frees its TMEM and returns.
#include "internal.cuh"

#include <algorithm>
#include <string>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace krr {

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One bounded probe of the phase: the thread may suspend (up to the 1 ms hint) until the
// phase completes instead of spinning, which keeps waiting warps off the issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000000;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false once `limit` cycles have passed (default 2^32 cycles, ~2 s).
constexpr long long kWaitLimitDefault = 1LL << 32;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          long long limit = kWaitLimitDefault) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulation.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
// 32 lanes x 32 consecutive 32-bit columns: thread = lane, r[c] = column c.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
// Waits for this thread's TMEM loads; r is tied in as read-write so that no use of the
// loaded registers can be scheduled above the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
                   "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                   "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]),
                   "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns from registers (thread = lane), then wait
// until the stores are done.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, "
        "%17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
        "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
        "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// 32 lanes x 16 consecutive 32-bit columns into registers.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]),
                   "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}
// D[tmem] (+)= A[tmem] * B[smem]^T, FP16 inputs, FP32 accumulation.  A (M = 128) sits in
// TMEM lane = row, two K-neighbours per 32-bit column (the even one in the low half).
__device__ __forceinline__ void mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T with the types of idesc (kind::f16: FP16 or BF16).
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    mma_bf16(d_tmem, adesc, bdesc, idesc, accumulate);
}
// Two floats as one f16x2 word, round to nearest: lo in bits 0-15, hi in bits 16-31.
__device__ __forceinline__ uint32_t pack_f16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x
// 16 bytes stored as contiguous 128-byte blocks; lbo = byte distance between core
// matrices adjacent along K, sbo = between 8-row groups; bits 46-47 = 1 (version),
// layout type 0 (no swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// The same descriptor for the 128-byte swizzled K-major layout (mode 2 at bits 61-63):
// rows of 128 bytes (64 BF16 along K), 8-row atoms of 1024 bytes at sbo = 1024, the
// 16-byte chunk c of row r stored at chunk c ^ (r & 7).  The leading offset is unused
// for this layout (field 1).  A K step of 16 elements inside the atom advances the
// start address by 32 bytes; atoms must be 1024-byte aligned.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// The same with A and B FP16 (type code 0).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (r, k) in the core-matrix tiled layout of a tile with Kp columns.
__host__ __device__ inline uint32_t tile_off(int r, int k, int Kp) {
    return (uint32_t)((((r >> 3) * (Kp >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Byte offset of element (r, k) in a feature tile of `rows` rows in the 128-byte swizzled
// layout: K in slabs of 64 (slab-major, each slab rows x 128 bytes), then the swizzle.
__host__ __device__ inline uint32_t tile_off_sw(int r, int k, int rows) {
    const uint32_t lin = (uint32_t)(k >> 6) * (uint32_t)rows * 128u + (uint32_t)r * 128u + (uint32_t)(k & 63) * 2u;
    return lin ^ (((lin >> 7) & 7u) << 4);
}

// ------------------------------------------------------------------ self-test
// M=128, N=32 MMAs on small integers (exact in BF16 and FP32); out[r*32 + c] receives D.
// variant 0: one K=16 step in the core-matrix layout, lbo = 128 (K neighbours), sbo = 256
// (row groups); variant 1 swaps them; variant 2: K = 64 in four steps in the 128-byte
// swizzled layout (the feature layout); variant 3 reads that swizzled data through an
// unswizzled descriptor; variant 4: FP16, K = 64 in four steps with A stored in TMEM
// (columns 32..63) and B in the swizzled layout (the multi-RHS product's P.V step).
// Every address stays inside the 20 KB of operands and the 64 TMEM columns.
__global__ void __launch_bounds__(128) k_tc_selftest(int variant, float* __restrict__ out,
                                                     int* __restrict__ err) {
    __shared__ __align__(1024) unsigned char sA[128 * 64 * 2];
    __shared__ __align__(1024) unsigned char sB[32 * 64 * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool sw = variant >= 2;
    const int K = sw ? 64 : 16;
    for (int e = tid; e < 128 * K && variant != 4; e += 128) {
        const int r = e / K, k = e % K;
        const float v = (float)((r % 7) - 3 + (k % 3));
        *reinterpret_cast<__nv_bfloat16*>(sA + (sw ? tile_off_sw(r, k, 128) : tile_off(r, k, 16))) =
            __float2bfloat16_rn(v);
    }
    for (int e = tid; e < 32 * K; e += 128) {
        const int c = e / K, k = e % K;
        const float v = (float)((c % 5) - 2 + (k % 4));
        if (variant == 4)
            *reinterpret_cast<__half*>(sB + tile_off_sw(c, k, 32)) = __float2half_rn(v);
        else
            *reinterpret_cast<__nv_bfloat16*>(sB + (sw ? tile_off_sw(c, k, 32) : tile_off(c, k, 16))) =
                __float2bfloat16_rn(v);
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    fence_proxy_async();
    __syncthreads();
    if (warp == 0) tmem_alloc(&tbase, 64);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tbase;
    if (variant == 4) {   // A (row = warp * 32 + lane) into TMEM columns 32..63
        const int r = warp * 32 + lane;
        uint32_t pk[32];
#pragma unroll
        for (int c = 0; c < 32; ++c)
            pk[c] = pack_f16x2((float)((r % 7) - 3 + ((2 * c) % 3)), (float)((r % 7) - 3 + ((2 * c + 1) % 3)));
        tmem_st32(tmem + ((uint32_t)(warp * 32) << 16) + 32u, pk);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    const uint32_t lbo = variant == 0 ? 128u : 256u, sbo = variant == 0 ? 256u : 128u;
    if (tid == 0) {
        if (variant == 4) {          // A from TMEM: 8 columns (16 FP16) per K step
            for (int kk = 0; kk < 4; ++kk)
                mma_f16_ts(tmem, tmem + 32u + 8u * kk, smem_desc_sw128(smem_u32(sB) + 32u * kk),
                           idesc_f16(128, 32), kk > 0 ? 1u : 0u);
        } else if (variant == 2) {   // four K steps of 16 inside the swizzle atom
            for (int kk = 0; kk < 4; ++kk)
                mma_bf16(tmem, smem_desc_sw128(smem_u32(sA) + 32u * kk),
                         smem_desc_sw128(smem_u32(sB) + 32u * kk), idesc_bf16(128, 32), kk > 0 ? 1u : 0u);
        } else if (variant == 3) {   // swizzled data read as unswizzled: must not match
            for (int kk = 0; kk < 4; ++kk)
                mma_bf16(tmem, smem_desc(smem_u32(sA) + 32u * kk, 16u, 1024u),
                         smem_desc(smem_u32(sB) + 32u * kk, 16u, 1024u), idesc_bf16(128, 32),
                         kk > 0 ? 1u : 0u);
        } else {
            mma_bf16(tmem, smem_desc(smem_u32(sA), lbo, sbo), smem_desc(smem_u32(sB), lbo, sbo),
                     idesc_bf16(128, 32), 0u);
        }
        mma_commit(&bar);
    }
    const bool ok = __syncthreads_and(mbar_wait(&bar, 0)) != 0;
    if (!ok && tid == 0) atomicExch(err, 1);
    tc_fence_after();
    if (ok) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), r);
        tmem_wait_ld(r);
        const int row = warp * 32 + lane;
        for (int c = 0; c < 32; ++c) out[row * 32 + c] = __uint_as_float(r[c]);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 64);
}

// ------------------------------------------------------------------ features
// bf16 pieces of a float: v = h + m + l
__device__ __forceinline__ void split3(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
    h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    l = __float2bfloat16_rn(r2);
}

// Features of point i (packed xh, a at P[i*ps + dk]) written into 128-row tiles in the
// 128-byte swizzled layout (K slabs of 64): role 0 = row operand, role 1 = column
// operand.  The row operand also has ones at K = 6 dk + 6 .. 6 dk + 8 (see the V-folded
// product).  Rows beyond n and the remaining K columns are zero.
__global__ void k_tc_features(const float* __restrict__ P, long long n, int dk, int ps, int Kp,
                              int role, long long nrows_pad, unsigned char* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows_pad) return;
    const long long tile = i >> 7;
    const int r = (int)(i & 127);
    unsigned char* base = out + tile * (128LL * Kp * 2);
    const __nv_bfloat16 one = __float2bfloat16_rn(1.f), zero = __float2bfloat16_rn(0.f);
    auto put = [&](int k, __nv_bfloat16 v) {
        *reinterpret_cast<__nv_bfloat16*>(base + tile_off_sw(r, k, 128)) = v;
    };
    if (i >= n) {
        for (int k = 0; k < Kp; ++k) put(k, zero);
        return;
    }
    int k = 0;
    for (int c = 0; c < dk; ++c) {
        const float x = P[i * ps + c];
        __nv_bfloat16 h, m, l;
        if (role == 0) {
            split3(2.f * x, h, m, l);
            put(k++, h); put(k++, h); put(k++, m); put(k++, h); put(k++, m); put(k++, l);
        } else {
            split3(x, h, m, l);
            put(k++, h); put(k++, m); put(k++, h); put(k++, l); put(k++, m); put(k++, h);
        }
    }
    __nv_bfloat16 a1, a2, a3;
    split3(P[i * ps + dk], a1, a2, a3);
    if (role == 0) {
        put(k++, a1); put(k++, a2); put(k++, a3); put(k++, one); put(k++, one); put(k++, one);
        // three more ones, against the column operand's log2|v_j| in the V-folded product
        // (zero in the plain column features, so they add nothing elsewhere)
        put(k++, one); put(k++, one); put(k++, one);
    } else {
        put(k++, one); put(k++, one); put(k++, one); put(k++, a1); put(k++, a2); put(k++, a3);
    }
    for (; k < Kp; ++k) put(k, zero);
}

// ------------------------------------------------------------------ V folded into the exponent
// With one right-hand side v the contraction folds into the exponent:
//     sum_j 2^t_ij v_j = sum_{v_j >= 0} 2^(t_ij + L_j) - sum_{v_j < 0} 2^(t_ij + L_j),
//     L_j = log2 |2^e v_j|   (-1000, so that 2^(t + L) = 0, for v_j = 0 and padding columns)
// with e putting max |2^e v| in [2^14, 2^15).  The column features carry L_j (BF16 x3 at
// K = 6 dk + 6 .. 6 dk + 8, against the row operand's ones) and the columns are partitioned
// stably, v >= 0 first: every 32-column chunk but the one at the boundary then adds to a
// single sum, and the epilogue does one ex2 and one FADD per pair with no V to load.
constexpr int VF_BLK = 1024;   // columns per block of the partition

// cnt[b] = number of v_j >= 0 in block b; *vmax = max |v_j| as float bits (non-negative
// floats order like their bits, so atomicMax on the bits is exact; *vmax starts at 0)
__global__ void __launch_bounds__(VF_BLK) k_vf_count(const float* __restrict__ V, int n, int* __restrict__ cnt,
                                                      unsigned* __restrict__ vmax) {
    __shared__ int wc[VF_BLK / 32];
    __shared__ unsigned wm[VF_BLK / 32];
    const int j = blockIdx.x * VF_BLK + threadIdx.x;
    const float v = j < n ? V[j] : 0.f;
    const unsigned m = __ballot_sync(0xffffffffu, j < n && !(v < 0.f));
    unsigned b = __float_as_uint(fabsf(v));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0) {
        wc[threadIdx.x >> 5] = __popc(m);
        wm[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        unsigned mb = 0;
        for (int w = 0; w < VF_BLK / 32; ++w) {
            t += wc[w];
            mb = max(mb, wm[w]);
        }
        cnt[blockIdx.x] = t;
        atomicMax(vmax, mb);
    }
}

// off[b] = exclusive prefix of cnt; *bnd = number of v_j >= 0; e = 15 - (binary exponent of
// max |v|) (0 when v is zero or not finite), vexp = e, vsc = 2^-(15 + e) (one thread;
// nblk <= 2^20 / 1024)
__global__ void k_vf_scan(const int* __restrict__ cnt, int nblk, int* __restrict__ off, int* __restrict__ bnd,
                          const unsigned* __restrict__ vmax, int* __restrict__ vexp, double* __restrict__ vsc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int t = 0;
    for (int b = 0; b < nblk; ++b) {
        off[b] = t;
        t += cnt[b];
    }
    *bnd = t;
    const float m = __uint_as_float(*vmax);
    int ex = 0;
    const bool ok = m > 0.f && m <= 3.4028234663852886e38f;
    if (ok) frexpf(m, &ex);
    const int e = ok ? 15 - ex : 0;
    *vexp = e;
    *vsc = ldexp(1.0, -(15 + e));
}

// Column j's feature row (Kp BF16 in the tiled, swizzled layout) moves to its place in the
// partition, with L_j written into K = k0 .. k0 + 2; rows n .. ncp - 1 stay in place with
// L = -1000.
__global__ void __launch_bounds__(VF_BLK)
k_vf_scatter(const float* __restrict__ V, int n, int ncp, const int* __restrict__ off, const int* __restrict__ bnd,
             const int* __restrict__ vexp, const unsigned char* __restrict__ FB, int Kp, int k0,
             unsigned char* __restrict__ FBv) {
    __shared__ int wpre[VF_BLK / 32];
    const int j = blockIdx.x * VF_BLK + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float vj = j < n ? V[j] : 0.f;
    const bool pos = j < n && !(vj < 0.f);
    const unsigned m = __ballot_sync(0xffffffffu, pos);
    if (lane == 0) wpre[w] = __popc(m);
    __syncthreads();
    if (j >= ncp) return;
    int before = 0;                               // v >= 0 columns before j in this block
    for (int i = 0; i < w; ++i) before += wpre[i];
    before += __popc(m & ((1u << lane) - 1u));
    int dst = j;
    if (j < n) {
        const int pb = off[blockIdx.x] + before;  // v >= 0 columns before j
        dst = pos ? pb : *bnd + (j - pb);
    }
    float L = -1000.f;
    if (j < n && vj != 0.f) L = log2f(fabsf(ldexpf(vj, vexp[0])));
    __nv_bfloat16 h, mm, l;
    split3(L, h, mm, l);
    if (L == -1000.f) { h = __float2bfloat16_rn(-1000.f); mm = __float2bfloat16_rn(0.f); l = mm; }
    const uint32_t tileA = 128u * Kp * 2u;
    const unsigned char* src = FB + (size_t)(j >> 7) * tileA + (size_t)(j & 127) * 128u;
    unsigned char* dd = FBv + (size_t)(dst >> 7) * tileA + (size_t)(dst & 127) * 128u;
    for (int kc = 0; kc < Kp / 8; ++kc) {         // 16-byte chunks of 8 K values
        const int sl = kc >> 3, c = kc & 7;
        // padding rows (j >= n) get zero features; they may lie past the base features
        uint4 x = j < n ? *reinterpret_cast<const uint4*>(src + sl * 16384 + ((c ^ (j & 7)) << 4))
                        : make_uint4(0u, 0u, 0u, 0u);
        if (kc * 8 + 7 >= k0 && kc * 8 <= k0 + 2) {
            __nv_bfloat16* e = reinterpret_cast<__nv_bfloat16*>(&x);
            for (int u = 0; u < 8; ++u) {
                const int k = kc * 8 + u;
                if (k == k0) e[u] = h;
                else if (k == k0 + 1) e[u] = mm;
                else if (k == k0 + 2) e[u] = l;
            }
        }
        *reinterpret_cast<uint4*>(dd + sl * 16384 + ((c ^ (dst & 7)) << 4)) = x;
    }
}

// ------------------------------------------------------------------ product kernel
// Warp-specialised persistent CTA (one per SM): warp 0 lane 0 streams feature tiles
// with cp.async.bulk, warp 1 lane 0 issues tcgen05.mma, warps 2..17 are the epilogue.
// A work item is 128 rows (one M = 128 MMA) against a range of 256-column tiles.  A
// tcgen05.mma of this kind costs at least ~99 cycles (N <= 64) and ~172 at N = 256
// (measured on GB300 with one thread issuing back to back), so the exponent MMAs run at
// the widest N: Kp / 16 MMAs per 32768 pairs, about 690 cycles at Kp = 64 (d <= 9)
// against 1024 cycles of ex2 at 32 per clock.  Measured per role with clock64 on the
// mixture (n = 10^5, v folded), an epilogue warp spends ~60% of its time on the
// exponentials, ~12% waiting for the MMA, and under 2% waiting for TMEM loads (each
// lands behind the previous chunk); a tile takes ~1500 cycles, ~66% of the MUFU rate,
// against ~88% for a free-running stream of 32-column loads, ex2 and adds.  The rest is
// the per-tile hand-off chain (MMA commit, TMEM release, a tile's first load): with a
// quarter of the MMAs, no exponentials or half the loads the tile is 2-11% shorter.
// Hand-offs are mbarrier full/empty pairs only (no block-wide barrier in the loop):
//   a_full / a_empty          the 128-row operand of the current work item
//   s_full[s] / s_empty[s]    column tile stage s (empty needs the MMA commit and the
//                             8 epilogue warps of the tile's parity, which read V from it)
//   t_full[b] / t_empty[b]    TMEM accumulator buffer b (2 x 256 columns), read by the
//                             8 epilogue warps of parity b
// EW epilogue warps: 16 (two per tile parity and TMEM lane quarter, 128 columns each); the
// code also takes 32 (64 columns each), which only fits a CTA without the two issuing warps
constexpr int tc_threads(int ew) { return 32 * (2 + ew); }
constexpr int TC_BN = 256;        // columns per tile
constexpr int TC_ROWS = 128;      // rows per work item
constexpr int TC_NSMAX = 4;       // most pipeline stages; the count is even, so that a
                                  // stage always holds tiles of one parity

struct TcShared {
    uint64_t a_full, a_empty, s_full[TC_NSMAX], s_empty[TC_NSMAX], t_full[2], t_empty[2], drain;
    uint32_t tbase;
    int abort;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// VF: V folded into the exponent (NRHS = 1; FB holds the partitioned, log2|v|-carrying
// column features, vf_bnd the number of v >= 0 columns and vf_sc = 2^-(15 + e), of which
// 2^15 vf_sc = 2^-e undoes the scale of v).
template <int NRHS, int EW, bool VF>
__global__ void __launch_bounds__(tc_threads(EW), 1)
k_kmvm_tc(const unsigned char* __restrict__ FA, const unsigned char* __restrict__ FB, int Kp,
          int nr, int nc, int ncp, const float* __restrict__ Vp, int items, int splits,
          int tiles_per_split, int ns, double* __restrict__ part, int* __restrict__ err,
          long long wlimit, int stall_copies, const int* __restrict__ vf_bnd, const double* __restrict__ vf_sc) {
    static_assert(!VF || NRHS == 1, "the V-folded form takes one right-hand side");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzle atoms need 1024-byte alignment; the launch adds 1 KB of slack for this
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t tileA = 128u * Kp * 2u;            // bytes of one 128-row feature tile
    const uint32_t tileB = 2u * tileA;                // a 256-column tile: slab-major, 256 rows
    unsigned char* sA = smem;                         // the item's 128 rows
    unsigned char* sB = smem + tileA;                 // ns column tiles
    float* sV = reinterpret_cast<float*>(sB + (size_t)ns * tileB);   // ns x NRHS x TC_BN
    TcShared* sh = reinterpret_cast<TcShared*>(sV + ns * NRHS * TC_BN);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&sh->a_full, 1);
        mbar_init(&sh->a_empty, 1);
        for (int s = 0; s < TC_NSMAX; ++s) {
            mbar_init(&sh->s_full[s], 1);
            // MMA + the epilogue warps of its parity, which read V from it (not when V is folded)
            mbar_init(&sh->s_empty[s], VF ? 1 : 1 + EW / 2);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->t_full[b], 1);
            mbar_init(&sh->t_empty[b], EW / 2);
        }
        mbar_init(&sh->drain, 1);
        sh->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == 0) tmem_alloc(&sh->tbase, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tbase;
    const int ntiles = (nc + TC_BN - 1) / TC_BN;
    const uint32_t vbytes = NRHS * TC_BN * 4u;
    const int nslab = Kp / 64;
    volatile int* abort = &sh->abort;
    auto give_up = [&]() {
        *abort = 1;
        atomicExch(err, 1);
    };

    if (warp == 0) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t g = 0, ic = 0;
            // stall_copies (failure-detection tests only): issue nothing, so that every
            // consumer's bounded wait runs out with no copy or MMA in flight
            for (int item = blockIdx.x; item < items && !*abort && !stall_copies; item += gridDim.x) {
                const int rb = item / splits, sp = item - rb * splits;
                const int t0 = sp * tiles_per_split;
                const int t1 = min(t0 + tiles_per_split, ntiles);
                if (!mbar_wait(&sh->a_empty, (ic & 1u) ^ 1u, wlimit)) { give_up(); break; }
                mbar_expect_tx(&sh->a_full, tileA);
                bulk_g2s(sA, FA + (size_t)rb * tileA, tileA, &sh->a_full);
                ++ic;
                bool ok = true;
                for (int t = t0; t < t1; ++t) {
                    const int s = (int)(g % (uint32_t)ns);
                    if (!mbar_wait(&sh->s_empty[s], ((g / ns) & 1u) ^ 1u, wlimit)) { ok = false; break; }
                    mbar_expect_tx(&sh->s_full[s], tileB + (VF ? 0u : vbytes));
                    // feature tiles 2t and 2t + 1 (128 rows each, slab-major) become one
                    // 256-row tile per 64-wide K slab: slab sl at sl x 32 KB, rows 128.. at +16 KB
                    unsigned char* dB = sB + (size_t)s * tileB;
                    for (int sl = 0; sl < nslab; ++sl)
                        for (int hf = 0; hf < 2; ++hf)
                            bulk_g2s(dB + sl * 32768u + hf * 16384u,
                                     FB + (size_t)(2 * t + hf) * tileA + (size_t)sl * 16384u, 16384u,
                                     &sh->s_full[s]);
                    float* dV = sV + s * NRHS * TC_BN;
                    for (int q = 0; q < NRHS && !VF; ++q)
                        bulk_g2s(dV + q * TC_BN, Vp + (size_t)q * ncp + (size_t)t * TC_BN, TC_BN * 4u,
                                 &sh->s_full[s]);
                    ++g;
                }
                if (!ok) { give_up(); break; }
            }
            // Drain: every copy issued lands before the CTA may exit.  Each barrier has
            // one arrival per phase (this thread's expect_tx), so the phase of the last
            // copy into it is the newest one and a parity wait on it is exact.
            for (uint32_t i = 0; i < (g < (uint32_t)ns ? g : (uint32_t)ns); ++i) {
                const uint32_t gg = g - 1 - i;
                mbar_wait(&sh->s_full[gg % ns], (gg / ns) & 1u, wlimit);
            }
            if (ic > 0) mbar_wait(&sh->a_full, (ic - 1) & 1u, wlimit);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(128, TC_BN);
            const uint32_t a_addr = smem_u32(sA);
            uint32_t g = 0, ic = 0;
            bool issued = false;
            for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x, ++ic) {
                const int sp = item % splits;
                const int t0 = sp * tiles_per_split;
                const int t1 = min(t0 + tiles_per_split, ntiles);
                if (!mbar_wait(&sh->a_full, ic & 1u, wlimit)) { give_up(); break; }
                bool ok = true;
                for (int t = t0; t < t1; ++t, ++g) {
                    const int s = (int)(g % (uint32_t)ns), b = g & 1;
                    if (!mbar_wait(&sh->s_full[s], (g / ns) & 1u, wlimit)) { ok = false; break; }
                    if (!mbar_wait(&sh->t_empty[b], ((g >> 1) & 1u) ^ 1u, wlimit)) { ok = false; break; }
                    issued = true;
                    tc_fence_after();
                    const uint32_t b_addr = smem_u32(sB + (size_t)s * tileB);
                    const uint32_t d = tmem + (uint32_t)(b * TC_BN);
                    for (int kk = 0; kk < Kp / 16; ++kk) {
                        // 32 bytes per K step inside a slab; slabs 16 KB apart for the 128
                        // rows of A, 32 KB apart for the 256 rows of B
                        const uint32_t kin = (uint32_t)(kk & 3) * 32u;
                        const uint64_t ad = smem_desc_sw128(a_addr + (uint32_t)(kk >> 2) * 16384u + kin);
                        const uint64_t bd = smem_desc_sw128(b_addr + (uint32_t)(kk >> 2) * 32768u + kin);
                        mma_bf16(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                    mma_commit(&sh->t_full[b]);
                    mma_commit(&sh->s_empty[s]);
                    if (t == t1 - 1) mma_commit(&sh->a_empty);
                }
                if (!ok) { give_up(); break; }
            }
            // Drain: a commit tracks every MMA this thread issued before it, so once the
            // drain barrier's first phase completes no MMA still writes TMEM.
            if (issued) {
                mma_commit(&sh->drain);
                mbar_wait(&sh->drain, 0, wlimit);
            }
        }
    } else {
        // ---------------------------------------------------------- epilogue
        // Warp e (0..15) reads TMEM lanes of its quarter (warp & 3), i.e. 32 rows of the
        // 128-row item, and 128 of the 256 columns (its column half), for the tiles of
        // its parity only: on each SM sub-partition two warps work on even tiles and two
        // on odd ones, so the TMEM load latency of one pair hides behind the exponentials
        // of the other.
        static_assert(EW == 16 || EW == 32, "16 or 32 epilogue warps");
        constexpr int NCP = EW / 8;                   // column parts per tile and parity
        constexpr int CW = TC_BN / NCP;               // columns per warp: 128 or 64
        const int e = warp - 2;                       // 0 .. EW - 1
        const int quarter = warp & 3;                 // TMEM lanes this warp may read
        const int gi = e >> 2;                        // four consecutive warps cover the quarters
        const int cpart = gi % NCP, par = gi / NCP;
        const int lrow = quarter * 32 + lane;
        uint32_t g = 0;
        for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x) {
            const int rb = item / splits, sp = item - rb * splits;
            const int t0 = sp * tiles_per_split;
            const int t1 = min(t0 + tiles_per_split, ntiles);
            constexpr int NA = NRHS >= 8 ? 1 : 4;    // independent FMA chains per right-hand side
            float acc[NRHS][NA];
            float accn[NA];                          // V folded: the sum over v < 0 columns
            float ah[NRHS], al[NRHS];               // tiles folded float-float (cancellation)
            float nh = 0.f, nl = 0.f;                // V folded: the v < 0 sum
#pragma unroll
            for (int q = 0; q < NRHS; ++q) {
                ah[q] = al[q] = 0.f;
#pragma unroll
                for (int a = 0; a < NA; ++a) acc[q][a] = 0.f;
            }
#pragma unroll
            for (int a = 0; a < NA; ++a) accn[a] = 0.f;
            const int bnd = VF ? *vf_bnd : 0;
            bool ok = true;
            for (int t = t0; t < t1; ++t, ++g) {
                if ((int)(g & 1u) != par) continue;
                const int s = (int)(g % (uint32_t)ns), b = par;
                ok = mbar_wait(&sh->t_full[b], (g >> 1) & 1u, wlimit) &&
                     (VF || mbar_wait(&sh->s_full[s], (g / ns) & 1u, wlimit));
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) { if (lane == 0) give_up(); break; }
                tc_fence_after();
                const float* v = sV + s * NRHS * TC_BN + cpart * CW;
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * TC_BN + cpart * CW);
                // one 32-column chunk of exponents r (columns 32 hh .. 32 hh + 31)
                auto chunk_vf = [&](const uint32_t (&r)[32], int hh) {
                    // which sum each column adds to: the chunk lies on one side of the
                    // partition boundary, except at most one chunk of the whole product
                    const int c0 = t * TC_BN + cpart * CW + 32 * hh;
                    if (c0 + 32 <= bnd) {
#pragma unroll
                        for (int u = 0; u < 32; ++u) acc[0][u % NA] += ex2f(__uint_as_float(r[u]));
                    } else if (c0 >= bnd) {
#pragma unroll
                        for (int u = 0; u < 32; ++u) accn[u % NA] += ex2f(__uint_as_float(r[u]));
                    } else {
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            const float ev = ex2f(__uint_as_float(r[u]));
                            if (c0 + u < bnd) acc[0][u % NA] += ev;
                            else accn[u % NA] += ev;
                        }
                    }
                };
                auto chunk = [&](const uint32_t (&r)[32], int hh) {
                    if constexpr (VF) {
                        chunk_vf(r, hh);
                        return;
                    }
#pragma unroll
                    for (int j4 = 0; j4 < 8; ++j4) {
                        float ev[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) ev[u] = ex2f(__uint_as_float(r[4 * j4 + u]));
#pragma unroll
                        for (int q = 0; q < NRHS; ++q) {
                            const float4 vv =
                                *reinterpret_cast<const float4*>(v + q * TC_BN + 32 * hh + 4 * j4);
                            acc[q][0 % NA] = fmaf(ev[0], vv.x, acc[q][0 % NA]);
                            acc[q][1 % NA] = fmaf(ev[1], vv.y, acc[q][1 % NA]);
                            acc[q][2 % NA] = fmaf(ev[2], vv.z, acc[q][2 % NA]);
                            acc[q][3 % NA] = fmaf(ev[3], vv.w, acc[q][3 % NA]);
                        }
                    }
                };
                auto release = [&]() {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sh->t_empty[b]);   // TMEM buffer free again
                };
                static_assert(TC_BN == 256, "32-column chunks");
                if constexpr (NRHS <= 2 && EW == 16) {
                    // two register sets: the load of chunk c + 1 is in flight while chunk c
                    // is exponentiated
                    uint32_t ra[32], rb[32];
                    tmem_ld32(tb, ra);
                    tmem_wait_ld(ra);
                    tmem_ld32(tb + 32, rb);
                    chunk(ra, 0);
                    tmem_wait_ld(rb);
                    tmem_ld32(tb + 64, ra);
                    chunk(rb, 1);
                    tmem_wait_ld(ra);
                    tmem_ld32(tb + 96, rb);
                    chunk(ra, 2);
                    tmem_wait_ld(rb);
                    release();
                    chunk(rb, 3);
                } else {
                    // 32 live registers for the exponents
#pragma unroll 1
                    for (int hh = 0; hh < CW / 32; ++hh) {
                        uint32_t r0[32];
                        tmem_ld32(tb + 32 * hh, r0);
                        tmem_wait_ld(r0);
                        if (hh == CW / 32 - 1) release();
                        chunk(r0, hh);
                    }
                }
                __syncwarp();
                if (!VF && lane == 0) mbar_arrive(&sh->s_empty[s]);   // V of this stage consumed
#pragma unroll
                for (int q = 0; q < NRHS; ++q) {
                    float tot = acc[q][0];
#pragma unroll
                    for (int a = 1; a < NA; ++a) tot += acc[q][a];
                    ff_add(ah[q], al[q], tot);
#pragma unroll
                    for (int a = 0; a < NA; ++a) acc[q][a] = 0.f;
                }
                if constexpr (VF) {
                    float tn = accn[0];
#pragma unroll
                    for (int a = 1; a < NA; ++a) tn += accn[a];
                    ff_add(nh, nl, tn);
#pragma unroll
                    for (int a = 0; a < NA; ++a) accn[a] = 0.f;
                }
            }
            if (!ok) break;
            const long long row = (long long)rb * TC_ROWS + lrow;
            if (row < nr) {
                // vf_sc = 2^-(15 + e) undoes both scales of the P.V form; here P is unscaled
                const double sc = VF ? *vf_sc * 32768.0 : 1.0;
#pragma unroll
                for (int q = 0; q < NRHS; ++q)
                    part[(((size_t)sp * (2 * NCP) + par * NCP + cpart) * NRHS + q) * nr + row] =
                        ((double)ah[q] + (double)al[q] - (VF ? (double)nh + (double)nl : 0.0)) * sc;
            }
        }
    }
    // the producer and the MMA issuer drained their own copies and MMAs above
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------ multi-RHS product
// With R right-hand sides the contraction sum_j P_ij V_jq (P_ij = 2^t_ij) is a GEMM of its
// own and runs as a second tcgen05 MMA, transposed so that its N is the widest possible:
//   EXP   S (128 rows x 128 columns) = FA(rows) . FB(columns)^T    (the BF16 x3 split above)
//   split P' = 2^15 2^S = Ph + Pl, both FP16 (22 significant bits), stored to shared memory
//         as one 256 x 128 K-major operand: rows 0..127 Ph, rows 128..255 Pl
//   PV    D (M = 128 x N = 256) += [Vh; Vl] . [Ph; Pl]^T over the tile's 128 columns (K)
// with V'_q = 2^e_q V_q (e_q puts max |V'_q| in [2^14, 2^15)) split V' = Vh + Vl in FP16.
// Row q of D (q < R) and row R + q hold Vh_q and Vl_q against Ph (column i) and Pl (column
// 128 + i); their four sums are the output for row i.  Every product of two FP16 values is
// exact in FP32 and the representation errors are about 2^-22 relative per entry; the
// scale 2^15 keeps P' in the normal FP16 range down to P = 2^-29.
// Why transposed: a tcgen05.mma costs at least ~99 cycles whatever its N (measured), so
// the contraction wants few, wide instructions: one of N = 256 per 16 columns x 128 rows
// x (hi + lo) here, against two of N <= 32 per 16 columns with P as the M = 128 operand.  The A operand is the
// V tile (2R rows, at least 16); M = 128 reads 128 rows from its address, and the rows
// past 2R (whatever shared memory follows) only reach D rows that are never read.
// D accumulates in FP32 over 16 column tiles; warp 0 then folds it into FP64 sums.
// Roles: warp 0 folds D, warp 1 lane 0 issues MMAs, warps 2..17 exponentiate (tile
// parity x 64-column half x TMEM lane quarter), warp 18 lane 0 copies.
constexpr int PV_BN = 128;        // columns per tile
constexpr int PV_ROWS = 128;      // rows per work item
constexpr int PV_THREADS = 32 * 19;
constexpr int PV_NS = 2;          // column-tile stages (features, then V)
constexpr int PV_FOLD = 16;       // column tiles per FP32 accumulation of D
constexpr uint32_t PV_PBYTES = 256u * PV_BN * 2u;   // one P operand: 256 rows x 128 FP16
constexpr uint32_t PV_DCOL = 256;                   // D at TMEM columns 256..511

struct PvShared {
    uint64_t a_full, a_empty, f_full[PV_NS], f_empty[PV_NS], v_full[PV_NS], v_empty[PV_NS], t_full[2],
        t_empty[2], p_full[2], p_empty[2], c_full, c_empty, drain;
    uint32_t tbase;
    int abort;
};

// The problems of one launch: a device table (grouped) or a single problem by value.
struct PvWork {
    const PvProb* table;
    int nprob;
    PvProb one;
};
// Where item `item` works; `pc` is the running problem index of the caller, which visits
// items in increasing order.
struct PvItem {
    const PvProb* pb;
    int rb, sp, t0, t1;
};
__device__ __forceinline__ PvItem pv_item(const PvWork& w, int item, int& pc) {
    PvItem it;
    if (w.table) {
        while (pc + 1 < w.nprob && item >= w.table[pc + 1].item0) ++pc;
        it.pb = &w.table[pc];
    } else {
        it.pb = &w.one;
    }
    const PvProb& pb = *it.pb;
    // split-major: CTAs running at the same time share one column split, whose features
    // and V tiles then stay in L2 while every row block streams them
    const int li = item - pb.item0, nrb = pb.items / pb.splits;
    it.sp = li / nrb;
    it.rb = li - it.sp * nrb;
    it.t0 = it.sp * pb.tps;
    it.t1 = min(it.t0 + pb.tps, (pb.nc + PV_BN - 1) / PV_BN);
    return it;
}
// the item's D folds end at its local tiles FOLD - 1, 2 FOLD - 1, ... and at its last tile
__device__ __forceinline__ bool pv_fold_end(int t, const PvItem& it) {
    return t == it.t1 - 1 || ((t - it.t0) % PV_FOLD) == PV_FOLD - 1;
}

// 2^15 2^t for two neighbouring columns, as FP16 pairs hi (Ph) and lo (Pl = P' - Ph rounded)
__device__ __forceinline__ void pv_split2(uint32_t t0, uint32_t t1, uint32_t& hi, uint32_t& lo) {
    const float p0 = ex2f(__uint_as_float(t0)) * 32768.f;
    const float p1 = ex2f(__uint_as_float(t1)) * 32768.f;
    hi = pack_f16x2(p0, p1);
    float r0, r1;
    // r = P' - Ph exactly (Ph is within 2^-11 of P'): one mixed FP16 x FP16 + FP32 FMA each
    asm("{\n .reg .b16 h0, h1, m1;\n mov.b32 {h0, h1}, %2;\n mov.b16 m1, 0xBC00;\n"
        " fma.rn.f32.f16 %0, h0, m1, %3;\n fma.rn.f32.f16 %1, h1, m1, %4;\n}"
        : "=f"(r0), "=f"(r1)
        : "r"(hi), "f"(p0), "f"(p1));
    lo = pack_f16x2(r0, r1);
}

// Feature tiles have K = Kp = 64 (d <= 9) for every problem of the launch.
template <int NRHS>
__global__ void __launch_bounds__(PV_THREADS, 1)
k_kmvm_tcpv(const __grid_constant__ PvWork w, int items, int* __restrict__ err, long long wlimit,
            int stall_copies) {
    static_assert(NRHS == 1 || NRHS == 2 || NRHS == 4 || NRHS == 8 || NRHS == 16, "right-hand sides");
    constexpr uint32_t VROWS = 2 * NRHS < 16 ? 16 : 2 * NRHS;   // Vh rows, Vl rows, zero rows
    constexpr uint32_t VSLAB = VROWS * 128u;          // bytes of 64 K of the V tile
    constexpr uint32_t VBYTES = 2 * VSLAB;            // one 128-column V tile
    constexpr int Kp = 64;
    constexpr uint32_t tileA = 128u * Kp * 2u;        // a 128-row feature tile
    constexpr uint32_t stage = tileA + VBYTES;        // column features, then V
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* sA = smem;                                   // the item's 128 rows
    unsigned char* sB = sA + tileA;                             // PV_NS stages
    unsigned char* sP = sB + PV_NS * stage;                     // 2 P operands
    double* sAcc = reinterpret_cast<double*>(sP + 2 * PV_PBYTES);      // [NRHS][128] FP64
    float* sFold = reinterpret_cast<float*>(sAcc + NRHS * PV_ROWS);    // [NRHS][128] one fold
    PvShared* sh = reinterpret_cast<PvShared*>(sFold + NRHS * PV_ROWS);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&sh->a_full, 1);
        mbar_init(&sh->a_empty, 1);
        for (int s = 0; s < PV_NS; ++s) {
            mbar_init(&sh->f_full[s], 1);
            mbar_init(&sh->f_empty[s], 1);
            mbar_init(&sh->v_full[s], 1);
            mbar_init(&sh->v_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->t_full[b], 1);
            mbar_init(&sh->t_empty[b], 8);     // the 8 exponent warps of the tile's parity
            mbar_init(&sh->p_full[b], 8);
            mbar_init(&sh->p_empty[b], 1);
        }
        mbar_init(&sh->c_full, 1);
        mbar_init(&sh->c_empty, 1);
        mbar_init(&sh->drain, 1);
        sh->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == 0) tmem_alloc(&sh->tbase, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tbase;
    volatile int* abort = &sh->abort;
    auto give_up = [&]() {
        *abort = 1;
        atomicExch(err, 1);
    };

    if (warp == 18) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t T = 0, ic = 0;
            int pc = 0;
            for (int item = blockIdx.x; item < items && !*abort && !stall_copies; item += gridDim.x) {
                const PvItem it = pv_item(w, item, pc);
                if (!mbar_wait(&sh->a_empty, (ic & 1u) ^ 1u, wlimit)) { give_up(); break; }
                mbar_expect_tx(&sh->a_full, tileA);
                bulk_g2s(sA, it.pb->FA + (size_t)it.rb * tileA, tileA, &sh->a_full);
                ++ic;
                bool ok = true;
                // features are released by the exponent MMA and V by the P.V MMA, which
                // runs a tile later: the next features start loading that much earlier
                for (int t = it.t0; t < it.t1; ++t, ++T) {
                    const int s = (int)(T % PV_NS);
                    const uint32_t ph = ((T / PV_NS) & 1u) ^ 1u;
                    if (!mbar_wait(&sh->f_empty[s], ph, wlimit)) { ok = false; break; }
                    mbar_expect_tx(&sh->f_full[s], tileA);
                    bulk_g2s(sB + s * stage, it.pb->FB + (size_t)t * tileA, tileA, &sh->f_full[s]);
                    if (!mbar_wait(&sh->v_empty[s], ph, wlimit)) {
                        mbar_wait(&sh->f_full[s], (T / PV_NS) & 1u, wlimit);   // the copy just issued
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&sh->v_full[s], VBYTES);
                    bulk_g2s(sB + s * stage + tileA, it.pb->Vt + (size_t)t * VBYTES, VBYTES, &sh->v_full[s]);
                }
                if (!ok) { give_up(); break; }
            }
            // drain: one arrival per barrier phase, so a parity wait on the newest is exact
            // (a tile whose V copy was never issued has its features' copy waited on)
            for (uint32_t i = 0; i < (T < (uint32_t)PV_NS ? T : (uint32_t)PV_NS); ++i) {
                const uint32_t gg = T - 1 - i;
                mbar_wait(&sh->f_full[gg % PV_NS], (gg / PV_NS) & 1u, wlimit);
                mbar_wait(&sh->v_full[gg % PV_NS], (gg / PV_NS) & 1u, wlimit);
            }
            if (ic > 0) mbar_wait(&sh->a_full, (ic - 1) & 1u, wlimit);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t id_exp = idesc_bf16(128, PV_BN), id_pv = idesc_f16(128, 256);
            bool issued = false, ok = true;
            // EXP of tile T + 1 is issued before PV of tile T, so that the exponentials of the
            // next tile run while the tensor core contracts the current one
            int pc_e = 0, item_e = blockIdx.x, t_e = 0;
            uint32_t T_e = 0, ic_e = 0;
            PvItem it_e{};
            bool have_e = item_e < items;
            if (have_e) {
                it_e = pv_item(w, item_e, pc_e);
                t_e = it_e.t0;
            }
            auto exp_next = [&]() -> bool {      // EXP of the next tile in sequence, then advance
                const int s = (int)(T_e % PV_NS), b = (int)(T_e & 1u);
                if (t_e == it_e.t0 && !mbar_wait(&sh->a_full, ic_e & 1u, wlimit)) return false;
                if (!mbar_wait(&sh->f_full[s], (T_e / PV_NS) & 1u, wlimit)) return false;
                if (!mbar_wait(&sh->t_empty[b], ((T_e >> 1) & 1u) ^ 1u, wlimit)) return false;
                tc_fence_after();
                const uint32_t a_addr = smem_u32(sA), b_addr = smem_u32(sB + s * stage);
                for (int kk = 0; kk < Kp / 16; ++kk)
                    mma_bf16(tmem + (uint32_t)(b * PV_BN), smem_desc_sw128(a_addr + (uint32_t)kk * 32u),
                             smem_desc_sw128(b_addr + (uint32_t)kk * 32u), id_exp, kk > 0 ? 1u : 0u);
                mma_commit(&sh->t_full[b]);
                mma_commit(&sh->f_empty[s]);         // the features of this stage are used up
                issued = true;
                ++T_e;
                if (++t_e == it_e.t1) {
                    mma_commit(&sh->a_empty);    // the last use of the item's rows
                    ++ic_e;
                    item_e += gridDim.x;
                    have_e = item_e < items;
                    if (have_e) {
                        it_e = pv_item(w, item_e, pc_e);
                        t_e = it_e.t0;
                    }
                }
                return true;
            };
            if (have_e) ok = exp_next();
            uint32_t T = 0, fc = 0;
            int pc = 0;
            for (int item = blockIdx.x; item < items && ok && !*abort; item += gridDim.x) {
                const PvItem it = pv_item(w, item, pc);
                bool fold_start = true;
                for (int t = it.t0; t < it.t1; ++t, ++T) {
                    if (have_e && !(ok = exp_next())) break;
                    const int s = (int)(T % PV_NS), pb = (int)(T & 1u);
                    if (!(ok = mbar_wait(&sh->p_full[pb], (T >> 1) & 1u, wlimit))) break;
                    if (!(ok = mbar_wait(&sh->v_full[s], (T / PV_NS) & 1u, wlimit))) break;
                    if (fold_start && !(ok = mbar_wait(&sh->c_empty, (fc & 1u) ^ 1u, wlimit))) break;
                    tc_fence_after();
                    const uint32_t v_addr = smem_u32(sB + s * stage + tileA);
                    const uint32_t p_addr = smem_u32(sP + pb * PV_PBYTES);
                    for (int kk = 0; kk < PV_BN / 16; ++kk) {
                        const uint32_t ko = (uint32_t)(kk >> 2), ki = (uint32_t)(kk & 3) * 32u;
                        mma_f16(tmem + PV_DCOL, smem_desc_sw128(v_addr + ko * VSLAB + ki),
                                smem_desc_sw128(p_addr + ko * 32768u + ki), id_pv,
                                (fold_start && kk == 0) ? 0u : 1u);
                    }
                    fold_start = false;
                    mma_commit(&sh->p_empty[pb]);
                    mma_commit(&sh->v_empty[s]);
                    if (pv_fold_end(t, it)) {
                        mma_commit(&sh->c_full);
                        ++fc;
                        fold_start = true;
                    }
                }
            }
            if (!ok) give_up();
            if (issued) {   // every MMA issued has finished once the drain phase completes
                mma_commit(&sh->drain);
                mbar_wait(&sh->drain, 0, wlimit);
            }
        }
    } else if (warp >= 2) {
        // ---------------------------------------------------------- exponentials
        // warp e (0..15): TMEM lanes of its quarter (rows quarter*32 .. +31), the 64-column
        // half chalf of every tile of parity par; P goes to the tile's P operand, row i
        // (Ph) and row 128 + i (Pl), K-major with the 128-byte swizzle (slab = chalf)
        const int e = warp - 2, quarter = warp & 3, chalf = (e >> 2) & 1, par = e >> 3;
        const int i = quarter * 32 + lane;
        uint32_t T = 0;
        int pc = 0;
        for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x) {
            const PvItem it = pv_item(w, item, pc);
            bool ok = true;
            for (int t = it.t0; t < it.t1; ++t, ++T) {
                if ((int)(T & 1u) != par) continue;
                const int b = par;
                ok = mbar_wait(&sh->t_full[b], (T >> 1) & 1u, wlimit) &&
                     mbar_wait(&sh->p_empty[b], ((T >> 1) & 1u) ^ 1u, wlimit);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) { if (lane == 0) give_up(); break; }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * PV_BN + chalf * 64);
                unsigned char* ps = sP + b * PV_PBYTES + chalf * 32768u;   // slab chalf
#pragma unroll 1
                for (int c32 = 0; c32 < 2; ++c32) {
                    uint32_t r[32], hi[16], lo[16];
                    tmem_ld32(tb + 32u * c32, r);
                    tmem_wait_ld(r);
                    if (c32 == 1) {                 // S of this tile fully read
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sh->t_empty[b]);
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) pv_split2(r[2 * j], r[2 * j + 1], hi[j], lo[j]);
                    // columns 32 c32 .. +31 of the slab: 16-byte chunks 4 c32 .. 4 c32 + 3
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const uint32_t kc = (uint32_t)(4 * c32 + m);
                        const uint32_t oh = (uint32_t)i * 128u + ((kc ^ (uint32_t)(i & 7)) << 4);
                        const uint32_t ol = (uint32_t)(128 + i) * 128u + ((kc ^ (uint32_t)(i & 7)) << 4);
                        *reinterpret_cast<uint4*>(ps + oh) = make_uint4(hi[4 * m], hi[4 * m + 1], hi[4 * m + 2], hi[4 * m + 3]);
                        *reinterpret_cast<uint4*>(ps + ol) = make_uint4(lo[4 * m], lo[4 * m + 1], lo[4 * m + 2], lo[4 * m + 3]);
                    }
                }
                fence_proxy_async();                // the stores, visible to the MMA's reads
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->p_full[b]);
            }
            if (!ok) break;
        }
    } else {
        // ---------------------------------------------------------- fold (warp 0)
        // D lanes 0..31 are V rows: lane q < NRHS is Vh_q, lane NRHS + q is Vl_q; columns
        // 0..127 meet Ph (row i), 128..255 meet Pl (row i).  One fold: every lane sums its
        // Ph and Pl columns, lane q adds lane NRHS + q, and the FP32 fold goes to sFold;
        // after c_empty the fold is added into the FP64 sums.
        uint32_t fc = 0;
        int pc = 0;
        for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x) {
            const PvItem it = pv_item(w, item, pc);
            for (int e = lane; e < NRHS * PV_ROWS; e += 32) sAcc[e] = 0.0;
            bool ok = true;
            for (int t = it.t0; t < it.t1; ++t) {
                if (!pv_fold_end(t, it)) continue;
                ok = __all_sync(0xffffffffu, mbar_wait(&sh->c_full, fc & 1u, wlimit));
                if (!ok) { if (lane == 0) give_up(); break; }
                ++fc;
                tc_fence_after();
#pragma unroll 1
                for (int c = 0; c < PV_ROWS / 32; ++c) {
                    uint32_t dh[32], dl[32];
                    tmem_ld32(tmem + PV_DCOL + 32u * c, dh);
                    tmem_ld32(tmem + PV_DCOL + 128u + 32u * c, dl);
                    tmem_wait_ld(dh);
                    tmem_wait_ld(dl);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float v = __uint_as_float(dh[j]) + __uint_as_float(dl[j]);
                        v += __shfl_down_sync(0xffffffffu, v, NRHS);
                        if (lane < NRHS) sFold[lane * PV_ROWS + 32 * c + j] = v;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->c_empty);
                for (int e = lane; e < NRHS * PV_ROWS; e += 32) sAcc[e] += (double)sFold[e];
                __syncwarp();
            }
            if (!ok) break;
            const int nr = it.pb->nr;
            double* part = it.pb->part;
            const double* vsc = it.pb->vsc;
            for (int q = 0; q < NRHS; ++q) {
                const double sc = vsc[q];
                for (int r = lane; r < PV_ROWS; r += 32) {
                    const long long row = (long long)it.rb * PV_ROWS + r;
                    if (row < nr) part[((size_t)it.sp * NRHS + q) * nr + row] = sAcc[q * PV_ROWS + r] * sc;
                }
            }
            __syncwarp();
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// Per right-hand side q of V (ldv-strided columns, n entries): e_q = 15 - (binary exponent
// of max |V_q|) so that 2^e_q max |V_q| lies in [2^14, 2^15) (0 when the column is zero or
// not finite); vexp[q] = e_q and vsc[q] = 2^-(15 + e_q), the factor that undoes both scales.
__global__ void k_pv_vscale(const float* __restrict__ V, int ldv, int n, int* __restrict__ vexp,
                            double* __restrict__ vsc) {
    __shared__ float red[32];
    const int q = blockIdx.x;
    float m = 0.f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) m = fmaxf(m, fabsf(V[(size_t)q * ldv + j]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        m = warp_max(m);
        if (threadIdx.x == 0) {
            int ex = 0;
            const bool ok = m > 0.f && m <= 3.4028234663852886e38f;
            if (ok) frexpf(m, &ex);
            const int e = ok ? 15 - ex : 0;
            vexp[q] = e;
            vsc[q] = ldexp(1.0, -(15 + e));
        }
    }
}

// V' = 2^e_q V split as Vh + Vl (FP16, round to nearest) into 128-column tiles of
// rows = max(16, 2R) rows (Vh of every q, then Vl, then zeros) in the 128-byte swizzled
// K-major layout, zero beyond n.  One thread per (row, column).
__global__ void k_pv_vsplit(const float* __restrict__ V, int ldv, int n, int ncp, int nrhs, int rows,
                            const int* __restrict__ vexp, unsigned char* __restrict__ Vt) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rows * ncp) return;
    const int r = (int)(e / ncp), j = (int)(e - (long long)r * ncp);
    const int q = r < nrhs ? r : r - nrhs;
    float out = 0.f;
    if (r < 2 * nrhs && j < n) {
        const float v = ldexpf(V[(size_t)q * ldv + j], vexp[q]);
        const float hv = __half2float(__float2half_rn(v));
        out = r < nrhs ? hv : v - hv;
    }
    unsigned char* tile = Vt + (size_t)(j >> 7) * ((size_t)rows * 256u);
    *reinterpret_cast<__half*>(tile + tile_off_sw(r, j & 127, rows)) = __float2half_rn(out);
}

// ------------------------------------------------------------------ tensor-core sketch
// Y = K Omega^T for Algorithm 1, as two chained tcgen05 MMAs per 64-point chunk j:
//   MMA1  S(128 x 64)  = FA(rows) . FB(chunk)^T      (exponents, TMEM, 2 buffers)
//   epilogue: P = bf16(2^S) into shared memory in core-matrix order (2 buffers)
//   MMA2  C(128 x 256) += P . Omega(256 projections x chunk)^T   (TMEM, 256 columns)
// A work item is (128-row tile, block of 256 projections); the C tile is written to Y
// at the end of the item.  Roles: warp 0 bulk copies, warp 1 MMAs, warps 2..9 epilogue.
// BF16 P and Omega only perturb the sketch (about 4e-3 relative), which only steers
// the anchor choice.
constexpr int SK_EPI = 8;
constexpr int SK_THREADS = 32 * (2 + SK_EPI);
constexpr int SK_NS = 3;
constexpr int SK_JC = 64;            // points per chunk
constexpr int SK_NB = 256;           // projections per block
constexpr uint32_t SK_OMT = SK_NB * SK_JC * 2;   // bytes of one Omega tile

struct SkShared {
    uint64_t a_full, a_empty, s_full[SK_NS], s_empty[SK_NS], x_full[2], x_empty[2], p_full[2],
        p_empty[2], c_full, c_empty;
    uint32_t tbase;
    int abort;
};

__global__ void __launch_bounds__(SK_THREADS, 1)
k_sketch_tc(const unsigned char* __restrict__ FA, const unsigned char* __restrict__ FB,
            const unsigned char* __restrict__ Om, int Kp, int n, int nab, int njc, int njc_alloc,
            int items, float* __restrict__ Y, int ldy, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // swizzle atoms need 1024-byte alignment; the launch adds 1 KB of slack for this
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const uint32_t tileA = 128u * Kp * 2u;
    const uint32_t tileB1 = (uint32_t)SK_JC * Kp * 2u;   // Kp / 64 slabs of 64 rows x 128 bytes
    unsigned char* sA = smem;
    unsigned char* sB1 = sA + tileA;                        // SK_NS x tileB1
    unsigned char* sB2 = sB1 + SK_NS * tileB1;              // SK_NS x SK_OMT
    unsigned char* sP = sB2 + SK_NS * SK_OMT;               // 2 x (128 x 64 bf16)
    SkShared* sh = reinterpret_cast<SkShared*>(sP + 2 * 128 * SK_JC * 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&sh->a_full, 1);
        mbar_init(&sh->a_empty, 1);
        for (int s = 0; s < SK_NS; ++s) {
            mbar_init(&sh->s_full[s], 1);
            mbar_init(&sh->s_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sh->x_full[b], 1);
            mbar_init(&sh->x_empty[b], SK_EPI);
            mbar_init(&sh->p_full[b], SK_EPI);
            mbar_init(&sh->p_empty[b], 1);
        }
        mbar_init(&sh->c_full, 1);
        mbar_init(&sh->c_empty, SK_EPI);
        sh->abort = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (warp == 0) tmem_alloc(&sh->tbase, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tbase;            // S buffers at columns 0 and 64, C at 256
    volatile int* abort = &sh->abort;
    auto give_up = [&]() {
        *abort = 1;
        atomicExch(err, 1);
    };

    if (warp == 0) {
        if (lane == 0) {   // ------------------------------------------------ producer
            uint32_t g = 0, ic = 0;
            for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x, ++ic) {
                const int rt = item / nab, ab = item - rt * nab;
                if (!mbar_wait(&sh->a_empty, (ic & 1u) ^ 1u)) { give_up(); break; }
                mbar_expect_tx(&sh->a_full, tileA);
                bulk_g2s(sA, FA + (size_t)rt * tileA, tileA, &sh->a_full);
                for (int jc = 0; jc < njc; ++jc, ++g) {
                    const int s = g % SK_NS;
                    if (!mbar_wait(&sh->s_empty[s], ((g / SK_NS) & 1u) ^ 1u)) { give_up(); break; }
                    mbar_expect_tx(&sh->s_full[s], tileB1 + SK_OMT);
                    // the 64-row chunk jc is half of 128-row tile jc / 2: one 8 KB piece per slab
                    for (int sl = 0; sl < Kp / 64; ++sl)
                        bulk_g2s(sB1 + s * tileB1 + sl * 8192u,
                                 FB + (size_t)(jc >> 1) * tileA + (size_t)sl * 16384u + (size_t)(jc & 1) * 8192u,
                                 8192u, &sh->s_full[s]);
                    bulk_g2s(sB2 + s * SK_OMT, Om + ((size_t)ab * njc_alloc + jc) * SK_OMT, SK_OMT,
                             &sh->s_full[s]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // ------------------------------------------------ MMA issuer
            const uint32_t id1 = idesc_bf16(128, SK_JC), id2 = idesc_bf16(128, SK_NB);
            const uint32_t sbo2 = SK_JC * 16u;
            uint32_t g = 0, ic = 0;
            auto mma1 = [&](uint32_t gg) -> bool {      // exponents of chunk gg into S[gg & 1]
                const int s = gg % SK_NS, b = gg & 1;
                if (!mbar_wait(&sh->s_full[s], (gg / SK_NS) & 1u)) return false;
                if (!mbar_wait(&sh->x_empty[b], ((gg >> 1) & 1u) ^ 1u)) return false;
                tc_fence_after();
                const uint32_t a_addr = smem_u32(sA), b_addr = smem_u32(sB1 + s * tileB1);
                for (int kk = 0; kk < Kp / 16; ++kk)   // swizzled slabs: A 16 KB, B 8 KB apart
                    mma_bf16(tmem + (uint32_t)(b * SK_JC),
                             smem_desc_sw128(a_addr + (uint32_t)(kk >> 2) * 16384u + (uint32_t)(kk & 3) * 32u),
                             smem_desc_sw128(b_addr + (uint32_t)(kk >> 2) * 8192u + (uint32_t)(kk & 3) * 32u),
                             id1, kk > 0 ? 1u : 0u);
                mma_commit(&sh->x_full[b]);
                return true;
            };
            for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x, ++ic) {
                if (!mbar_wait(&sh->a_full, ic & 1u)) { give_up(); break; }
                const uint32_t g0 = g;
                bool ok = mma1(g0);
                for (int jc = 0; jc < njc && ok; ++jc) {
                    const uint32_t gg = g0 + jc;
                    if (jc + 1 < njc) ok = mma1(gg + 1);
                    else mma_commit(&sh->a_empty);          // last exponent MMA of the item
                    if (!ok) break;
                    const int s = gg % SK_NS, b = gg & 1;
                    if (!mbar_wait(&sh->p_full[b], (gg >> 1) & 1u)) { ok = false; break; }
                    if (jc == 0 && !mbar_wait(&sh->c_empty, (ic & 1u) ^ 1u)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t p_addr = smem_u32(sP + b * 128 * SK_JC * 2);
                    const uint32_t o_addr = smem_u32(sB2 + s * SK_OMT);
                    for (int kk = 0; kk < SK_JC / 16; ++kk)
                        mma_bf16(tmem + 256u, smem_desc(p_addr + kk * 256u, 128u, sbo2),
                                 smem_desc(o_addr + kk * 256u, 128u, sbo2), id2,
                                 (jc > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&sh->p_empty[b]);
                    mma_commit(&sh->s_empty[s]);
                    if (jc == njc - 1) mma_commit(&sh->c_full);
                }
                g = g0 + njc;
                if (!ok) { give_up(); break; }
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int e = warp - 2;
        const int quarter = warp & 3, cg = e >> 2;   // cg: which 32 of the 64 S columns
        const int r = quarter * 32 + lane;             // row inside the 128-row tile
        uint32_t g = 0, ic = 0;
        for (int item = blockIdx.x; item < items && !*abort; item += gridDim.x, ++ic) {
            const int rt = item / nab, ab = item - rt * nab;
            bool ok = true;
            for (int jc = 0; jc < njc; ++jc, ++g) {
                const int b = g & 1;
                ok = mbar_wait(&sh->x_full[b], (g >> 1) & 1u) && mbar_wait(&sh->p_empty[b], ((g >> 1) & 1u) ^ 1u);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) { if (lane == 0) give_up(); break; }
                tc_fence_after();
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * SK_JC + cg * 32), v);
                tmem_wait_ld(v);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->x_empty[b]);
                unsigned char* pb = sP + b * 128 * SK_JC * 2;
#pragma unroll
                for (int u = 0; u < 4; ++u) {   // 8 consecutive K = one core-matrix row
                    uint32_t w[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const float e0 = ex2f(__uint_as_float(v[8 * u + 2 * h]));
                        const float e1 = ex2f(__uint_as_float(v[8 * u + 2 * h + 1]));
                        const __nv_bfloat162 pr = __floats2bfloat162_rn(e0, e1);
                        w[h] = *reinterpret_cast<const uint32_t*>(&pr);
                    }
                    *reinterpret_cast<uint4*>(pb + tile_off(r, cg * 32 + 8 * u, SK_JC)) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh->p_full[b]);
            }
            if (!ok) break;
            // the item's C tile: this warp's 32 rows, 128 of the 256 projections
            ok = __all_sync(0xffffffffu, mbar_wait(&sh->c_full, ic & 1u));
            if (!ok) { if (lane == 0) give_up(); break; }
            tc_fence_after();
            const long long row = (long long)rt * 128 + r;
            for (int u = 0; u < 4; ++u) {
                uint32_t cv[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(256 + cg * 128 + 32 * u), cv);
                tmem_wait_ld(cv);
                const int a0 = ab * SK_NB + cg * 128 + 32 * u;
                if (row < n) {
                    float4* dst = reinterpret_cast<float4*>(Y + (size_t)row * ldy + a0);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (a0 + 4 * q < ldy)
                            dst[q] = make_float4(__uint_as_float(cv[4 * q]), __uint_as_float(cv[4 * q + 1]),
                                                 __uint_as_float(cv[4 * q + 2]), __uint_as_float(cv[4 * q + 3]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->c_empty);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (*abort) {
        mbar_wait(&sh->c_full, 0);
        mbar_wait(&sh->p_empty[0], 0);
    }
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ------------------------------------------------------------------ host side
int tc_feature_kp(int d) { return ((6 * kernel_dim(d) + 6) + 63) / 64 * 64; }

// Y (n x ldy, FP32) = K Omega^T on tensor cores; Om from launch_omega_bf16_tiled with
// njc_alloc = (padded n) / 64 chunks per projection block.
int launch_sketch_tc(krr_ctx* ctx, const unsigned char* FA, const unsigned char* FB, long long n, int d,
                     const void* Om, int l, int njc_alloc, float* Y, int ldy) {
    const int Kp = tc_feature_kp(d);
    const uint32_t tileA = 128u * Kp * 2u, tileB1 = (uint32_t)SK_JC * Kp * 2u;
    const size_t smem = tileA + (size_t)SK_NS * (tileB1 + SK_OMT) + 2 * 128 * SK_JC * 2 + 256 + 1024;
    KRR_RET(allow_max_dynamic_smem(ctx, (const void*)k_sketch_tc));
    int* err;
    KRR_RET(bufT(ctx, "tc_err", 1, &err));
    KRR_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    const int nab = (l + SK_NB - 1) / SK_NB;
    const int njc = (int)((n + SK_JC - 1) / SK_JC);
    const int nrt = (int)((n + 127) / 128);
    const int items = nrt * nab;
    const int grid = std::min(items, ctx->num_sms);
    k_sketch_tc<<<grid, SK_THREADS, smem, ctx->stream>>>(FA, FB, static_cast<const unsigned char*>(Om), Kp,
                                                         (int)n, nab, njc, njc_alloc, items, Y, ldy, err);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

int launch_tc_features(krr_ctx* ctx, const float* P, long long n, int d, int role,
                       unsigned char* out) {
    const int dk = kernel_dim(d), Kp = tc_feature_kp(d);
    const long long npad = (n + 255) / 256 * 256;
    k_tc_features<<<ceil_div(npad, 256), 256, 0, ctx->stream>>>(P, n, dk, packed_stride(d), Kp, role,
                                                                npad, out);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

size_t tc_feature_bytes(long long n, int d) {
    return (size_t)((n + 255) / 256 * 256) * tc_feature_kp(d) * 2;
}

typedef void (*tc_fn)(const unsigned char*, const unsigned char*, int, int, int, int, const float*,
                      int, int, int, int, double*, int*, long long, int, const int*, const double*);


// ---- grouped form: the same kernels over the problems of a batch, one launch each
// Per (problem, right-hand side) block: the column's scale exponent, as k_pv_vscale.
__global__ void k_pv_vscale_g(const PvPrep* __restrict__ tab, int nrhs) {
    __shared__ float red[32];
    const PvPrep& pp = tab[blockIdx.x / nrhs];
    const int q = blockIdx.x % nrhs;
    float m = 0.f;
    for (int j = threadIdx.x; j < pp.n; j += blockDim.x) m = fmaxf(m, fabsf(pp.V[(size_t)q * pp.ldv + j]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        m = warp_max(m);
        if (threadIdx.x == 0) {
            int ex = 0;
            const bool ok = m > 0.f && m <= 3.4028234663852886e38f;
            if (ok) frexpf(m, &ex);
            const int e = ok ? 15 - ex : 0;
            pp.vexp[q] = e;
            pp.vsc[q] = ldexp(1.0, -(15 + e));
        }
    }
}

// The split of every problem's V into its tiles, as k_pv_vsplit; blocks blk0 .. of problem p.
__global__ void k_pv_vsplit_g(const PvPrep* __restrict__ tab, int nprob, int nrhs, int rows) {
    int lo = 0, hi = nprob - 1;   // last problem whose first block is <= blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[mid].blk0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const PvPrep& pp = tab[lo];
    const long long e = (long long)((int)blockIdx.x - pp.blk0) * blockDim.x + threadIdx.x;
    if (e >= (long long)rows * pp.ncp) return;
    const int r = (int)(e / pp.ncp), j = (int)(e - (long long)r * pp.ncp);
    const int q = r < nrhs ? r : r - nrhs;
    float out = 0.f;
    if (r < 2 * nrhs && j < pp.n) {
        const float v = ldexpf(pp.V[(size_t)q * pp.ldv + j], pp.vexp[q]);
        const float hv = __half2float(__float2half_rn(v));
        out = r < nrhs ? hv : v - hv;
    }
    unsigned char* tile = pp.Vt + (size_t)(j >> 7) * ((size_t)rows * 256u);
    *reinterpret_cast<__half*>(tile + tile_off_sw(r, j & 127, rows)) = __float2half_rn(out);
}

int pv_tile_bytes(int nrhs) { return std::max(16, 2 * nrhs) * PV_BN * 2; }

int launch_pv_prep_grouped(krr_ctx* ctx, const PvPrep* tab_dev, int nprob, int nblk, int nrhs) {
    k_pv_vscale_g<<<nprob * nrhs, 512, 0, ctx->stream>>>(tab_dev, nrhs);
    KRR_CHECK_LAUNCH();
    k_pv_vsplit_g<<<nblk, 256, 0, ctx->stream>>>(tab_dev, nprob, nrhs, std::max(16, 2 * nrhs));
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// Shared memory of the P.V kernel for nrhs right-hand sides (K = 64 features).
static size_t pv_smem_bytes(int nrhs) {
    const size_t tileA = 128u * 64u * 2u;
    const size_t vbytes = (size_t)pv_tile_bytes(nrhs);
    return 1024 + tileA + PV_NS * (tileA + vbytes) + 2 * (size_t)PV_PBYTES + (size_t)nrhs * PV_ROWS * 12 +
           sizeof(PvShared);
}

// One launch of the product over the items of every problem in the device table (item0
// prefix, `items` in all); every problem has K = 64 features (d <= 9).
int launch_kmvm_tcpv_table(krr_ctx* ctx, const PvProb* table_dev, int nprob, int items, int nrhs,
                           int* err) {
    auto fn = nrhs == 16 ? &k_kmvm_tcpv<16> : nrhs == 8 ? &k_kmvm_tcpv<8> : nrhs == 4 ? &k_kmvm_tcpv<4>
            : nrhs == 2 ? &k_kmvm_tcpv<2> : &k_kmvm_tcpv<1>;
    KRR_RET(allow_max_dynamic_smem(ctx, (const void*)fn));
    const long long wlimit = ctx->opts.wait_limit_log2 > 0 ? (1LL << ctx->opts.wait_limit_log2)
                                                           : kWaitLimitDefault;
    PvWork w{};
    w.table = table_dev;
    w.nprob = nprob;
    const int grid = std::min(items, ctx->num_sms);
    fn<<<grid, PV_THREADS, pv_smem_bytes(nrhs), ctx->stream>>>(w, items, err, wlimit, ctx->opts.test_stall_copies);
    KRR_CHECK_LAUNCH();
    return KRR_OK;
}

// Q = K(rows, cols) V + beta V for 8 or 16 right-hand sides with P.V on the tensor cores.
static int launch_kmvm_tcpv(krr_ctx* ctx, const unsigned char* FA, long long nr, const unsigned char* FB,
                            long long nc, int Kp, float beta, const float* V, int nrhs, float* Q, int* err) {
    const int ncp = (int)((nc + PV_BN - 1) / PV_BN * PV_BN);
    const int vrows = std::max(16, 2 * nrhs);
    const size_t vbytes = (size_t)vrows * PV_BN * 2;        // one V tile: Vh, Vl (and zeros), FP16
    unsigned char* Vt;
    int* vexp;
    double* vsc;
    KRR_RET(bufT(ctx, "pv_vt", vbytes * (ncp / PV_BN), &Vt));
    KRR_RET(bufT(ctx, "pv_vexp", 16, &vexp));
    KRR_RET(bufT(ctx, "pv_vsc", 16, &vsc));
    k_pv_vscale<<<nrhs, 512, 0, ctx->stream>>>(V, (int)nc, (int)nc, vexp, vsc);
    KRR_CHECK_LAUNCH();
    const long long nsplit = (long long)vrows * ncp;
    k_pv_vsplit<<<ceil_div(nsplit, 256), 256, 0, ctx->stream>>>(V, (int)nc, (int)nc, ncp, nrhs, vrows, vexp, Vt);
    KRR_CHECK_LAUNCH();
    if (Kp != 64) return fail(ctx, KRR_E_INVAL, "P.V on tensor cores needs d <= 9");
    auto fn = nrhs == 16 ? &k_kmvm_tcpv<16> : nrhs == 8 ? &k_kmvm_tcpv<8> : nrhs == 4 ? &k_kmvm_tcpv<4>
            : nrhs == 2 ? &k_kmvm_tcpv<2> : &k_kmvm_tcpv<1>;
    KRR_RET(allow_max_dynamic_smem(ctx, (const void*)fn));
    const int nrb = (int)ceil_div(nr, PV_ROWS);
    const int ntiles = ncp / PV_BN;
    // items run split-major: one split's features and V tiles (all row blocks stream them
    // at about the same time) should fit in about a third of the 129 MB L2
    const long long col_bytes = (long long)ntiles * (128 * 64 * 2 + (long long)pv_tile_bytes(nrhs));
    const int sc_min = (int)std::min<long long>(std::max<long long>(1, ntiles), ceil_div(col_bytes, 40LL << 20));
    int splits = sc_min;
    long long best = -1;
    for (int sc = sc_min; sc <= std::max(sc_min, std::min(64, ntiles)); ++sc) {   // as in launch_kmvm_tc
        const long long per = (ntiles + sc - 1) / sc;
        const long long waves = ((long long)nrb * sc + ctx->num_sms - 1) / ctx->num_sms;
        const long long cost = waves * (per + 8);
        if (best < 0 || cost < best) {
            best = cost;
            splits = sc;
        }
    }
    splits = std::max(sc_min, tuned_splits(ctx, tune_key(1, Kp, nrhs, nr), splits, ntiles));
    const int tps = (ntiles + splits - 1) / splits;
    splits = (ntiles + tps - 1) / tps;
    ctx->last_splits = splits;
    const int items = nrb * splits;
    double* part;
    KRR_RET(bufT(ctx, "tc_part", (size_t)splits * nrhs * nr, &part));
    const int grid = std::min(items, ctx->num_sms);
    const long long wlimit = ctx->opts.wait_limit_log2 > 0 ? (1LL << ctx->opts.wait_limit_log2)
                                                           : kWaitLimitDefault;
    PvWork w{};
    w.table = nullptr;
    w.nprob = 1;
    w.one = PvProb{FA, FB, Vt, vsc, part, (int)nr, (int)nc, Kp, splits, tps, items, 0, 0};
    fn<<<grid, PV_THREADS, pv_smem_bytes(nrhs), ctx->stream>>>(w, items, err, wlimit, ctx->opts.test_stall_copies);
    KRR_CHECK_LAUNCH();
    return launch_kmvm_reduce(ctx, part, splits, (int)nr, nrhs, V, (int)nc, beta, Q, (int)nr);
}

// Q = K(rows, cols) V + beta V using features FA (rows) and FB (cols).
int launch_kmvm_reduce64(krr_ctx* ctx, const double* part, int nparts, int nr, int nrhs2,
                         const double* V64, double beta, double* Q64, double ksc);
double ex2_bias_scale(const krr_ctx* ctx);

int launch_kmvm_tc(krr_ctx* ctx, const unsigned char* FA, long long nr, const unsigned char* FB,
                   long long nc, int d, float beta, const float* V, int nrhs, float* Q,
                   const double* V64, double* Q64) {
    if (kernel_dim(d) > 16) return fail(ctx, KRR_E_INVAL, "tensor-core product needs d <= 16");
    const bool hp = Q64 != nullptr;   // V holds hi/lo column pairs; FP64 output
    if (hp && (nrhs % 2 != 0 || !V64)) return fail(ctx, KRR_E_INVAL, "tensor-core product: bad split");
    const int Kp = tc_feature_kp(d);
    const int ncp = (int)((nc + TC_BN - 1) / TC_BN * TC_BN);
    // the error word is cleared by the caller (once per call or solve), so that a timeout
    // in any product stays visible until the caller reads it
    int* err;
    KRR_RET(bufT(ctx, "tc_err", 1, &err));
    int done = 0;
    while (done < nrhs) {
        const int left = nrhs - done;
        const int chunk = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
        const std::string key = tune_key(1, Kp, chunk, nr);
        bool use_pv = !hp && Kp == 64 && (ctx->opts.tc_pv == 2 || (ctx->opts.tc_pv == 1 && chunk >= 8));
        TuneEntry te;
        if (!hp && Kp == 64) {
            if (ctx->force_pv >= 0) use_pv = ctx->force_pv == 1;
            else if (ctx->opts.tc_pv != 0 && tune_lookup(ctx, key, &te)) use_pv = te.pv == 1;
        }
        if (use_pv) {
            KRR_RET(launch_kmvm_tcpv(ctx, FA, nr, FB, nc, Kp, beta, V + (size_t)done * nc, chunk,
                                     Q + (size_t)done * nr, err));
            done += chunk;
            continue;
        }
        // 16 epilogue warps (32 would need 34 warps with the producer and the MMA issuer,
        // above the 32 warps a CTA may have)
        const int ew = 16;
        // one right-hand side: V folded into the exponent (opts.tc_vfold)
        const bool vf = chunk == 1 && !hp && ctx->opts.tc_vfold;
        tc_fn fn = vf ? &k_kmvm_tc<1, 16, true> : chunk == 1 ? &k_kmvm_tc<1, 16, false>
                 : chunk == 2 ? &k_kmvm_tc<2, 16, false> : chunk == 4 ? &k_kmvm_tc<4, 16, false>
                 : chunk == 8 ? &k_kmvm_tc<8, 16, false> : &k_kmvm_tc<16, 16, false>;
        const int ngroups = ew / 4;                   // partial sums per split: parity x column part
        // V padded to whole 256-column tiles, RHS-major (16-byte aligned bulk copies), or, with
        // V folded into the exponent, the partitioned column features that carry log2 |v|
        float* Vp = nullptr;
        const unsigned char* FBk = FB;
        int* vf_bnd = nullptr;
        double* vf_sc = nullptr;
        if (vf) {
            unsigned char* FBv;
            int *vexp, *cnt, *off;
            const int nblk = (int)ceil_div(nc, VF_BLK);
            KRR_RET(bufT(ctx, "vf_fb", (size_t)(ncp / 128) * 128 * Kp * 2, &FBv));
            KRR_RET(bufT(ctx, "vf_exp", 1, &vexp));
            KRR_RET(bufT(ctx, "vf_sc", 1, &vf_sc));
            KRR_RET(bufT(ctx, "vf_cnt", (size_t)nblk, &cnt));
            KRR_RET(bufT(ctx, "vf_off", (size_t)nblk, &off));
            KRR_RET(bufT(ctx, "vf_bnd", 1, &vf_bnd));
            unsigned* vmax;
            KRR_RET(bufT(ctx, "vf_max", 1, &vmax));
            const float* Vc = V + (size_t)done * nc;
            KRR_TRY_CUDA(cudaMemsetAsync(vmax, 0, sizeof(unsigned), ctx->stream));
            k_vf_count<<<nblk, VF_BLK, 0, ctx->stream>>>(Vc, (int)nc, cnt, vmax);
            KRR_CHECK_LAUNCH();
            k_vf_scan<<<1, 32, 0, ctx->stream>>>(cnt, nblk, off, vf_bnd, vmax, vexp, vf_sc);
            KRR_CHECK_LAUNCH();
            k_vf_scatter<<<(unsigned)ceil_div(ncp, VF_BLK), VF_BLK, 0, ctx->stream>>>(
                Vc, (int)nc, ncp, off, vf_bnd, vexp, FB, Kp, 6 * kernel_dim(d) + 6, FBv);
            KRR_CHECK_LAUNCH();
            FBk = FBv;
        } else {
            KRR_RET(bufT(ctx, "tc_vpad", (size_t)chunk * ncp, &Vp));
            KRR_TRY_CUDA(cudaMemsetAsync(Vp, 0, sizeof(float) * chunk * ncp, ctx->stream));
            KRR_TRY_CUDA(cudaMemcpy2DAsync(Vp, sizeof(float) * ncp, V + (size_t)done * nc, sizeof(float) * nc,
                                           sizeof(float) * nc, chunk, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        const uint32_t tileA = 128u * Kp * 2u;
        // stages: four where they fit (K = 64), else two
        int optin = 0;
        KRR_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        const size_t stage = 2 * (size_t)tileA + (size_t)chunk * TC_BN * 4;
        const size_t fixed = (size_t)tileA + sizeof(TcShared) + 1024;
        const int ns = fixed + 4 * stage <= (size_t)optin ? 4 : 2;
        if (fixed + ns * stage > (size_t)optin) return fail(ctx, KRR_E_INVAL, "tensor-core product: tiles too wide");
        const size_t smem_launch = std::max<size_t>(fixed + ns * stage, 120 * 1024);   // one CTA per SM (TMEM)
        KRR_RET(allow_max_dynamic_smem(ctx, (const void*)fn));
        const int nrb = (int)ceil_div(nr, TC_ROWS);
        const int ntiles = ncp / TC_BN;
        // column splits: the CTA with the most items sets the time, so minimise
        // ceil(items / SMs) x (tiles per item + the per-item cost, about 8 tiles)
        int splits = 1;
        long long best = -1;
        for (int sc = 1; sc <= std::min(64, ntiles); ++sc) {
            const long long per = (ntiles + sc - 1) / sc;
            const long long waves = ((long long)nrb * sc + ctx->num_sms - 1) / ctx->num_sms;
            const long long cost = waves * (per + 8);
            if (best < 0 || cost < best) {
                best = cost;
                splits = sc;
            }
        }
        splits = tuned_splits(ctx, key, splits, ntiles);
        const int tps = (ntiles + splits - 1) / splits;
        splits = (ntiles + tps - 1) / tps;
        ctx->last_splits = splits;
        const int items = nrb * splits;
        double* part;
        KRR_RET(bufT(ctx, "tc_part", (size_t)ngroups * splits * chunk * nr, &part));
        const int grid = std::min(items, ctx->num_sms);
        const long long wlimit = ctx->opts.wait_limit_log2 > 0 ? (1LL << ctx->opts.wait_limit_log2)
                                                               : kWaitLimitDefault;
        fn<<<grid, tc_threads(ew), smem_launch, ctx->stream>>>(FA, FBk, Kp, (int)nr, (int)nc, ncp, Vp, items,
                                                               splits, tps, ns, part, err, wlimit,
                                                               ctx->opts.test_stall_copies, vf_bnd, vf_sc);
        KRR_CHECK_LAUNCH();
        // column groups (tile parity x column part) per split: ngroups * splits partial sums
        if (hp)
            KRR_RET(launch_kmvm_reduce64(ctx, part, ngroups * splits, (int)nr, chunk, V64 + (size_t)(done / 2) * nr,
                                         (double)beta, Q64 + (size_t)(done / 2) * nr, ex2_bias_scale(ctx)));
        else
            KRR_RET(launch_kmvm_reduce(ctx, part, ngroups * splits, (int)nr, chunk, V + (size_t)done * nc, (int)nc,
                                       beta, Q + (size_t)done * nr, (int)nr));
        done += chunk;
    }
    return KRR_OK;
}

}  // namespace krr

using namespace krr;

// Known-answer test of the tcgen05 descriptor encodings (host entry, see krr.h).
extern "C" int krr_tc_selftest(int variant, int* mismatches, float* max_err, void* stream_v) {
    if (!mismatches || !max_err || variant < 0 || variant > 4) return KRR_E_INVAL;
    cudaStream_t stream = (cudaStream_t)stream_v;
    float* out = nullptr;
    int* err = nullptr;
    if (cudaMalloc(&out, 128 * 32 * sizeof(float)) != cudaSuccess) return KRR_E_NOMEM;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
        cudaFree(out);
        return KRR_E_NOMEM;
    }
    cudaMemsetAsync(err, 0, sizeof(int), stream);
    cudaMemsetAsync(out, 0, 128 * 32 * sizeof(float), stream);
    k_tc_selftest<<<1, 128, 0, stream>>>(variant, out, err);
    float h[128 * 32];
    int herr = 0;
    cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, stream);
    cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream);
    const cudaError_t e = cudaStreamSynchronize(stream);
    cudaFree(out);
    cudaFree(err);
    if (e != cudaSuccess) return KRR_E_CUDA;
    if (herr) return KRR_E_CUDA;
    int bad = 0;
    float mx = 0.f;
    for (int r = 0; r < 128; ++r)
        for (int c = 0; c < 32; ++c) {
            float ref = 0.f;
            for (int k = 0; k < (variant >= 2 ? 64 : 16); ++k)
                ref += (float)((r % 7) - 3 + (k % 3)) * (float)((c % 5) - 2 + (k % 4));
            const float d = std::fabs(h[r * 32 + c] - ref);
            mx = std::max(mx, d);
            if (d > 0.f) ++bad;
        }
    *mismatches = bad;
    *max_err = mx;
    return KRR_OK;
}
