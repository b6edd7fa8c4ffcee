// Grouped batched solves: the PCG recurrences (Algorithm 5 step 3 with the Algorithm 4
// preconditioner) of many independent problems advance in lockstep, and every step of an
// iteration is ONE launch over the work items of all active problems:
//   product      items (problem, 128-row block, column split) of the tensor-core product
//                with P.V on the tensor cores (tc_kmvm.cu, d <= 9), after one V-split launch
//   vectors      blocks (problem, column, 2048-row chunk) of the concatenated x, r, z, p, q
//   Woodbury     blocks (problem, 1024-row chunk) of F^T r, threads (problem, column, anchor)
//                of its reduction, blocks (problem, anchor) of the two triangular products,
//                blocks (problem, 64-row chunk) of (r - F v) / beta
//   scalars      warps (problem, column) sum the partials of their own blocks
// Every problem keeps its own CG scalars, column activity and convergence state.  The host
// reads every problem's recursive residuals once per iteration, runs the true-residual
// replacements (float-float, per problem) of the problems that call for one, and removes
// finished problems from the work tables.  A problem whose expansion-form recurrence breaks
// down, stalls or keeps showing gaps escalates in place to the exact-difference product (run
// on its own stream), as krr_solve does; one that fails in that form or reaches a limit is
// finished by its own krr_solve, so the grouped path ends every problem as the one-by-one
// path would.
#include "internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

namespace krr {

constexpr int GV_T = 256;        // threads of the vector kernels
constexpr int GV_ROWS = 2048;    // rows per vector block
constexpr int GF_ROWS = 1024;    // rows per F^T r block
constexpr int GF_STAGE = 256;    // rows of r staged in shared memory at a time
constexpr int GN_ROWS = 64;      // rows per (r - F v) / beta block: 8 warps x 8 rows
constexpr int GMAXQ = 8;         // right-hand sides per Woodbury pass
constexpr int GSPLIT_CAP = 16;   // most column splits of one problem's product

// rows [r0, r1) of column c of problem p; base = element offset of (p, c, row 0)
struct GVBlk {
    long long base;
    int p, c, r0, r1;
};
// one (problem, column): its vector blocks b0 .. b0 + nb - 1
struct GSeg {
    int p, c, b0, nb;
};
struct GProb {
    long long off;              // element offset of the problem's n x nrhs block
    const float* F;
    const double* T2;
    const double* T2t;
    double* upart;              // F^T r partials [chunk][GMAXQ][ldF]
    double* u;                  // [GMAXQ][k] FP64
    double* u1;
    double* v;
    double* part;               // product partials [split][chunk columns][n]
    int n, k, ldF, nft;         // nft: F^T r chunks
    int ft0, tri0, gn0, ngn;    // first block of each Woodbury table, apply blocks
    int red0, splits;           // first thread of the F^T r reduction; product splits
    int tc, pad;                // 1: product on tensor cores through the grouped launch
    float beta, inv_beta;
};

__device__ __forceinline__ double g_block_sum(double v) {
    __shared__ double red[GV_T / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// last index i of the ascending first[0 .. n-1] with first[i] <= x (first[0] <= x)
template <typename T, typename F>
__device__ __forceinline__ int g_find(const T* tab, int n, int x, F first) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first(tab[mid]) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------- vector kernels
// q = ksc * (sum of the product's split partials) + beta p for the columns c0 .. c0 + nch - 1
// (from_part), and the blocks' partial sums of p . q
__global__ void __launch_bounds__(GV_T)
k_g_reduce_pq(const GVBlk* __restrict__ vb, const GProb* __restrict__ gp, int c0, int nch, double ksc,
              bool from_part, const float* __restrict__ P, float* __restrict__ Q, double* __restrict__ vpart,
              int boff) {
    const GVBlk blk = vb[boff + blockIdx.x];
    const GProb& g = gp[blk.p];
    const int cc = blk.c - c0;
    double s = 0.0;
    for (int i = blk.r0 + threadIdx.x; i < blk.r1; i += GV_T) {
        const long long e = blk.base + i;
        float qv;
        if (from_part && g.tc) {
            double t = 0.0;
            for (int sp = 0; sp < g.splits; ++sp) t += g.part[((size_t)sp * nch + cc) * g.n + i];
            qv = (float)(t * ksc + (double)g.beta * (double)P[e]);
            Q[e] = qv;
        } else {
            qv = Q[e];
        }
        s += (double)P[e] * (double)qv;
    }
    s = g_block_sum(s);
    if (threadIdx.x == 0) vpart[boff + blockIdx.x] = s;
}

// x += a p, r -= a q (a of the block's problem and column), partial sums of r . r
__global__ void __launch_bounds__(GV_T)
k_g_update_xr(const GVBlk* __restrict__ vb, const double* __restrict__ a, int nrhs, float* __restrict__ x,
              float* __restrict__ r, const float* __restrict__ P, const float* __restrict__ Q,
              double* __restrict__ vpart) {
    const GVBlk blk = vb[blockIdx.x];
    const float av = (float)a[blk.p * nrhs + blk.c];
    double s = 0.0;
    for (int i = blk.r0 + threadIdx.x; i < blk.r1; i += GV_T) {
        const long long e = blk.base + i;
        const float rv = fmaf(-av, Q[e], r[e]);
        x[e] = fmaf(av, P[e], x[e]);
        r[e] = rv;
        s += (double)rv * (double)rv;
    }
    s = g_block_sum(s);
    if (threadIdx.x == 0) vpart[blockIdx.x] = s;
}

// p = z (restart of the problem) or z + b p
__global__ void __launch_bounds__(GV_T)
k_g_beta_p(const GVBlk* __restrict__ vb, const double* __restrict__ b, const int* __restrict__ restart,
           int nrhs, float* __restrict__ P, const float* __restrict__ Z) {
    const GVBlk blk = vb[blockIdx.x];
    const bool rs = restart[blk.p] != 0;
    const float bv = (float)b[blk.p * nrhs + blk.c];
    for (int i = blk.r0 + threadIdx.x; i < blk.r1; i += GV_T) {
        const long long e = blk.base + i;
        P[e] = rs ? Z[e] : fmaf(bv, P[e], Z[e]);
    }
}

// ---------------------------------------------------------------- scalar kernels
// one warp per (problem, column) segment
// mode 0: pq = sum, a = rz / pq on active columns (non-positive or non-finite: bad)
// mode 1: rr = sum
__global__ void k_g_scalars(const GSeg* __restrict__ seg, int nseg, int nrhs, int mode,
                            const double* __restrict__ vpart, double* __restrict__ rz, double* __restrict__ pq,
                            double* __restrict__ a, double* __restrict__ rr, int* __restrict__ act,
                            int* __restrict__ bad) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= nseg) return;
    const GSeg sg = seg[w];
    double s = 0.0;
    for (int i = lane; i < sg.nb; i += 32) s += vpart[sg.b0 + i];
    s = warp_sum(s);
    if (lane != 0) return;
    const int id = sg.p * nrhs + sg.c;
    if (mode == 0) {
        pq[id] = s;
        double av = 0.0;
        if (act[id]) {
            if (!(s > 0.0) || !isfinite(s) || !isfinite(rz[id])) {
                bad[sg.p] = 1;
                act[id] = 0;
            } else {
                av = rz[id] / s;
            }
        }
        a[id] = av;
    } else {
        rr[id] = s;
        if (!isfinite(s)) bad[sg.p] = 1;
    }
}

// rz_new = r . z over the problem's apply blocks; b = rz_new / rz (0 on a restart)
__global__ void k_g_beta(const GSeg* __restrict__ seg, int nseg, int nrhs, int c0, int nq,
                         const GProb* __restrict__ gp, const double* __restrict__ gnpart,
                         const int* __restrict__ restart, double* __restrict__ rz, double* __restrict__ b,
                         int* __restrict__ bad) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= nseg) return;
    const GSeg sg = seg[w];
    if (sg.c < c0 || sg.c >= c0 + nq) return;
    const GProb& g = gp[sg.p];
    double s = 0.0;
    for (int i = lane; i < g.ngn; i += 32) s += gnpart[(size_t)(g.gn0 + i) * GMAXQ + (sg.c - c0)];
    s = warp_sum(s);
    if (lane != 0) return;
    const int id = sg.p * nrhs + sg.c;
    double bv = 0.0;
    if (!restart[sg.p]) {
        if (rz[id] > 0.0 && isfinite(s)) bv = s / rz[id];
        else if (!isfinite(s)) bad[sg.p] = 1;
    }
    if (!isfinite(s)) bad[sg.p] = 1;
    b[id] = bv;
    rz[id] = s;
}

// ---------------------------------------------------------------- Woodbury apply
// Error-free transformations for the compensated F^T r sums (as in cg.cu)
__device__ __forceinline__ void g_ff_acc(float& h, float& l, float f, float r) {
    const float p = __fmul_rn(f, r);
    const float pe = fmaf(f, r, -p);
    const float s = __fadd_rn(h, p);
    const float z = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, z)), __fsub_rn(p, z));
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, pe));
}

// upart[j][q][a] = sum over rows of chunk j of F[i, a] R[c0 + q][i], compensated; one
// block per (problem, chunk), one thread per anchor column a (stride GV_T).
template <int NQ>
__global__ void __launch_bounds__(GV_T)
k_g_ft(const GProb* __restrict__ gp, int nprob, int c0, const float* __restrict__ R) {
    __shared__ float sr[NQ][GF_STAGE];
    const int pi = g_find(gp, nprob, (int)blockIdx.x, [](const GProb& g) { return g.ft0; });
    const GProb& g = gp[pi];
    const int j = (int)blockIdx.x - g.ft0;
    const int r0 = j * GF_ROWS, r1 = min(g.n, r0 + GF_ROWS);
    for (int a0 = 0; a0 < g.k; a0 += GV_T) {
        const int a = a0 + threadIdx.x;
        float h[NQ], l[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) h[q] = l[q] = 0.f;
        for (int b0 = r0; b0 < r1; b0 += GF_STAGE) {
            const int nb = min(GF_STAGE, r1 - b0);
            __syncthreads();
            for (int e = threadIdx.x; e < NQ * GF_STAGE; e += GV_T) {
                const int q = e / GF_STAGE, i = e - q * GF_STAGE;
                sr[q][i] = i < nb ? R[g.off + (long long)(c0 + q) * g.n + b0 + i] : 0.f;
            }
            __syncthreads();
            if (a < g.k) {
                const float* fp = g.F + (size_t)b0 * g.ldF + a;
                for (int i = 0; i < nb; ++i) {
                    const float f = fp[(size_t)i * g.ldF];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) g_ff_acc(h[q], l[q], f, sr[q][i]);
                }
            }
        }
        if (a < g.k) {
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                g.upart[((size_t)j * GMAXQ + q) * g.ldF + a] = (double)h[q] + (double)l[q];
        }
    }
}

// u[q][a] = sum over the problem's chunks of upart[j][q][a]; one thread per (problem, q, a)
__global__ void k_g_ft_reduce(const GProb* __restrict__ gp, int nprob, int nq, int total) {
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (t >= total) return;
    const int pi = g_find(gp, nprob, t, [](const GProb& g) { return g.red0; });
    const GProb& g = gp[pi];
    const int lt = t - g.red0, q = lt / g.k, a = lt - q * g.k;
    if (q >= nq) return;
    double s = 0.0;
    for (int j = 0; j < g.nft; ++j) s += g.upart[((size_t)j * GMAXQ + q) * g.ldF + a];
    g.u[(size_t)q * g.k + a] = s;
}

// y[q][a] = sum_b T[a][b] x[q][b], b <= a (lower, T2) or b >= a (upper, T2t); one block of
// 128 threads per (problem, row a)
__global__ void __launch_bounds__(128)
k_g_tri(const GProb* __restrict__ gp, int nprob, int nq, bool lower) {
    __shared__ double red[4];
    const int pi = g_find(gp, nprob, (int)blockIdx.x, [](const GProb& g) { return g.tri0; });
    const GProb& g = gp[pi];
    const int a = (int)blockIdx.x - g.tri0, k = g.k;
    const double* T = lower ? g.T2 : g.T2t;
    const double* x = lower ? g.u : g.u1;
    double* y = lower ? g.u1 : g.v;
    const int b0 = lower ? 0 : a, b1 = lower ? a + 1 : k;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = 0; q < nq; ++q) {
        double s = 0.0;
        for (int b = b0 + threadIdx.x; b < b1; b += 128) s = fma(T[(size_t)a * k + b], x[(size_t)q * k + b], s);
        s = warp_sum(s);
        __syncthreads();
        if (lane == 0) red[w] = s;
        __syncthreads();
        if (threadIdx.x == 0) y[(size_t)q * k + a] = red[0] + red[1] + red[2] + red[3];
    }
}

// Z = (R - F v) / beta for rows of one chunk of one problem (one warp per row), with the
// block's partial sums of R . Z per column into gnpart[blk][q]
template <int NQ>
__global__ void __launch_bounds__(GV_T)
k_g_gn(const GProb* __restrict__ gp, int nprob, int c0, const float* __restrict__ R, float* __restrict__ Z,
       double* __restrict__ gnpart) {
    extern __shared__ float sv[];   // [NQ][k]
    __shared__ double red[GV_T / 32][NQ];
    const int pi = g_find(gp, nprob, (int)blockIdx.x, [](const GProb& g) { return g.gn0; });
    const GProb& g = gp[pi];
    const int k = g.k;
    for (int e = threadIdx.x; e < NQ * k; e += GV_T) sv[e] = (float)g.v[e];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r0 = ((int)blockIdx.x - g.gn0) * GN_ROWS;
    double rz[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) rz[q] = 0.0;
    for (int i = r0 + w; i < min(g.n, r0 + GN_ROWS); i += GV_T / 32) {
        const float* f = g.F + (size_t)i * g.ldF;
        float t[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) t[q] = 0.f;
        for (int a = lane; a < k; a += 32) {
            const float fa = f[a];
#pragma unroll
            for (int q = 0; q < NQ; ++q) t[q] = fmaf(fa, sv[q * k + a], t[q]);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float tq = warp_sum(t[q]);
            if (lane == 0) {
                const long long e = g.off + (long long)(c0 + q) * g.n + i;
                const float rv = R[e];
                const float zv = (rv - tq) * g.inv_beta;
                Z[e] = zv;
                rz[q] += (double)rv * (double)zv;
            }
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) red[w][q] = rz[q];
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        double s = 0.0;
        for (int i = 0; i < GV_T / 32; ++i) s += red[i][threadIdx.x];
        gnpart[(size_t)blockIdx.x * GMAXQ + threadIdx.x] = s;
    }
}

}  // namespace krr

using namespace krr;

namespace {

double now_ms_g() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Device arrays of the grouped phase; owned here, freed on every exit path.
struct GDev {
    std::vector<void*> ptrs;
    template <typename T>
    T* alloc(size_t count) {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~GDev() {
        for (void* p : ptrs) cudaFree(p);
    }
};
struct GPinned {
    std::vector<void*> ptrs;
    template <typename T>
    T* alloc(size_t count) {
        void* p = nullptr;
        if (cudaMallocHost(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T*>(p);
    }
    ~GPinned() {
        for (void* p : ptrs) cudaFreeHost(p);
    }
};

// per-problem host state of the grouped recurrence
struct GState {
    bool active = false, done = false, fallback = false, esc_pending = false;
    int it = 0, since = 0, sweeps = 0, restarts = 0, gapped = 0, window = 500, it_best = 0;
    double best = 1.0;
    std::vector<double> yn, rtrue, rec;
    std::vector<int> act;
};

}  // namespace

extern "C" int krr_batch_solve_grouped(const krr_problem* probs, int nprob, int nrhs, double tol,
                                       unsigned long long seed, const krr_opts* opts, int workers,
                                       krr_solve_info* infos, int* statuses) {
    if (!probs || nprob < 1 || nrhs < 1 || nrhs > KRR_MAX_RHS || !(tol > 0.0) || !(tol < 1.0))
        return KRR_E_INVAL;
    for (int i = 0; i < nprob; ++i) {
        const krr_problem& p = probs[i];
        if (!p.X || !p.Y || !p.alpha || p.n < 1 || p.n > (1LL << 30) || p.d < 1 || p.d > KRR_MAX_DIM ||
            p.k < 1 || p.k > p.n || !(p.sigma > 0.0) || !(p.beta > 0.0))
            return KRR_E_INVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KRR_E_CUDA;
    krr_opts o;
    if (opts) o = *opts;
    else krr_default_opts(&o);
    const int W = std::max(1, std::min(workers > 0 ? workers : 8, nprob));

    // ---- contexts and builds (W threads, largest n^2 first), each on its own stream
    std::vector<krr_ctx*> ctxs(nprob, nullptr);
    std::vector<cudaStream_t> streams(nprob, nullptr);
    std::vector<int> status(nprob, KRR_E_STATE);
    std::vector<krr_solve_info> info(nprob);
    for (int i = 0; i < nprob; ++i) std::memset(&info[i], 0, sizeof(krr_solve_info));
    auto cleanup = [&]() {
        for (int i = 0; i < nprob; ++i) {
            if (ctxs[i]) krr_destroy(ctxs[i]);
            if (streams[i]) cudaStreamDestroy(streams[i]);
        }
    };
    for (int i = 0; i < nprob; ++i) {
        if (cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            krr_create(&ctxs[i], &o, streams[i]) != KRR_OK) {
            cleanup();
            return KRR_E_CUDA;
        }
    }
    std::vector<int> order(nprob);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)probs[a].n * probs[a].n > (double)probs[b].n * probs[b].n;
    });
    auto run_pool = [&](auto&& job) {
        std::atomic<int> next(0);
        std::vector<std::thread> pool;
        for (int w = 0; w < W; ++w)
            pool.emplace_back([&]() {
                cudaSetDevice(dev);
                for (;;) {
                    const int slot = next.fetch_add(1);
                    if (slot >= nprob) break;
                    job(order[slot]);
                }
            });
        for (auto& t : pool) t.join();
    };
    run_pool([&](int i) {
        const krr_problem& p = probs[i];
        const int rc = krr_build_precond(ctxs[i], p.X, p.n, p.d, p.sigma, p.beta, p.k,
                                         seed + (unsigned long long)i);
        status[i] = rc == KRR_E_NOCONV ? KRR_OK : rc;
        cudaStreamSynchronize(streams[i]);
    });

    // ---- the grouped phase on one stream
    const double t0 = now_ms_g();
    cudaStream_t S = nullptr;
    if (cudaStreamCreateWithFlags(&S, cudaStreamNonBlocking) != cudaSuccess) {
        cleanup();
        return KRR_E_CUDA;
    }
    krr_ctx* ctx = ctxs[0];   // launches of the grouped kernels are accounted to it
    int rc_all = KRR_OK;
    // fork/join events of the work that runs on the problems' own streams
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join(nprob, nullptr);
    bool ev_ok = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < nprob && ev_ok; ++i)
        ev_ok = cudaEventCreateWithFlags(&ev_join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ev_ok) rc_all = KRR_E_CUDA;
    // problems handed back to their own solve start at once, on a thread of their own
    std::vector<std::thread> fb_threads;
    std::vector<char> fb_started(nprob, 0);
    std::vector<krr_solve_info> fb_info(nprob);
    std::vector<int> fb_status(nprob, KRR_E_STATE);
    auto start_fallback = [&](int i) {
        cudaEventRecord(ev_fork, S);                     // after every grouped step that touched it
        cudaStreamWaitEvent(streams[i], ev_fork, 0);
        ctxs[i]->stream = streams[i];
        fb_started[i] = 1;
        fb_threads.emplace_back([&, i]() {
            cudaSetDevice(dev);
            const krr_problem& p = probs[i];
            std::memset(&fb_info[i], 0, sizeof(krr_solve_info));
            fb_status[i] = krr_solve(ctxs[i], p.X, p.Y, nrhs, tol, p.alpha, &fb_info[i]);
            cudaStreamSynchronize(streams[i]);
        });
    };
    {
        GDev gd;
        GPinned gh;
        std::vector<long long> off(nprob + 1, 0);
        for (int i = 0; i < nprob; ++i) off[i + 1] = off[i] + probs[i].n * nrhs;
        const long long L = off[nprob];
        float* x = gd.alloc<float>(L);
        float* r = gd.alloc<float>(L);
        float* z = gd.alloc<float>(L);
        float* pv = gd.alloc<float>(L);
        float* qv = gd.alloc<float>(L);
        const size_t ns = (size_t)nprob * nrhs;
        double* d_rz = gd.alloc<double>(ns);
        double* d_pq = gd.alloc<double>(ns);
        double* d_a = gd.alloc<double>(ns);
        double* d_b = gd.alloc<double>(ns);
        double* d_rr = gd.alloc<double>(ns);
        double* d_norm = gd.alloc<double>(ns);
        int* d_act = gd.alloc<int>(ns);
        int* d_bad = gd.alloc<int>(nprob);
        int* d_restart = gd.alloc<int>(nprob);
        int* d_err = gd.alloc<int>(1);
        double* h_rr = gh.alloc<double>(ns);
        double* h_norm = gh.alloc<double>(ns);
        int* h_act = gh.alloc<int>(ns);
        int* h_bad = gh.alloc<int>(nprob);
        int* h_restart = gh.alloc<int>(nprob);
        int* h_err = gh.alloc<int>(1);
        // tables: sized for every problem active
        long long nvb_max = 0, nft_max = 0, ntri_max = 0, ngn_max = 0, nred_max = 0, items_max = 0, nvs_max = 0;
        const int chunk_max = nrhs >= 16 ? 16 : nrhs >= 8 ? 8 : nrhs >= 4 ? 4 : nrhs >= 2 ? 2 : 1;
        const int vtile = pv_tile_bytes(chunk_max);
        std::vector<int> tcp(nprob, 0);
        // product form per problem: the requested one (1 needs tensor-core features, else 0),
        // and 2 (exact differences) after an escalation
        std::vector<int> form(nprob, 0);
        for (int i = 0; i < nprob; ++i)
            form[i] = o.precision == 1 ? (ctxs[i]->FA ? 1 : 0) : o.precision;
        for (int i = 0; i < nprob; ++i) {
            const krr_ctx* c = ctxs[i];
            const long long n = probs[i].n;
            nvb_max += (long long)nrhs * ((n + GV_ROWS - 1) / GV_ROWS);
            nft_max += (n + GF_ROWS - 1) / GF_ROWS;
            ntri_max += c->k_eff;
            ngn_max += (n + GN_ROWS - 1) / GN_ROWS;
            nred_max += (long long)GMAXQ * c->k_eff;
            // the grouped tensor-core launch takes K = 64 features (d <= 9); wider problems
            // built for tensor cores use their own tensor-core product inside the loop
            tcp[i] = (o.precision == 1 && c->FA && tc_feature_kp(c->d) == 64) ? 1 : 0;
            if (tcp[i]) {
                const long long ntl = (n + 127) / 128;
                items_max += ((n + 127) / 128) * std::min<long long>(GSPLIT_CAP, ntl);
                nvs_max += ((long long)std::max(16, 2 * chunk_max) * ntl * 128 + 255) / 256;
            }
        }
        GVBlk* d_vb = gd.alloc<GVBlk>(nvb_max);
        GSeg* d_seg = gd.alloc<GSeg>(ns);
        GProb* d_gp = gd.alloc<GProb>(nprob);
        PvProb* d_pv = gd.alloc<PvProb>(nprob);
        PvPrep* d_pp = gd.alloc<PvPrep>((size_t)nprob * 5);   // one table per RHS chunk
        double* d_vpart = gd.alloc<double>(nvb_max);
        double* d_gnpart = gd.alloc<double>(ngn_max * GMAXQ);
        GVBlk* h_vb = gh.alloc<GVBlk>(nvb_max);
        GSeg* h_seg = gh.alloc<GSeg>(ns);
        GProb* h_gp = gh.alloc<GProb>(nprob);
        PvProb* h_pv = gh.alloc<PvProb>(nprob);
        PvPrep* h_pp = gh.alloc<PvPrep>((size_t)nprob * 5);
        // per-problem device work arrays of the Woodbury apply and the product
        std::vector<GProb> base(nprob);
        std::vector<unsigned char*> vt(nprob, nullptr);
        std::vector<int*> vexp(nprob, nullptr);
        std::vector<double*> vsc(nprob, nullptr);
        bool ok_alloc = x && r && z && pv && qv && d_rz && d_pq && d_a && d_b && d_rr && d_norm && d_act &&
                        d_bad && d_restart && d_err && h_rr && h_norm && h_act && h_bad && h_restart && h_err &&
                        d_vb && d_seg && d_gp && d_pv && d_pp && d_vpart && d_gnpart && h_vb && h_seg && h_gp &&
                        h_pv && h_pp;
        for (int i = 0; i < nprob && ok_alloc; ++i) {
            const krr_ctx* c = ctxs[i];
            GProb& g = base[i];
            std::memset(&g, 0, sizeof(g));
            g.off = off[i];
            g.n = (int)probs[i].n;
            g.k = c->k_eff;
            g.ldF = c->ldF;
            g.F = c->F;
            g.T2 = c->T2;
            g.T2t = c->T2t;
            g.nft = (g.n + GF_ROWS - 1) / GF_ROWS;
            g.beta = (float)c->beta;
            g.inv_beta = (float)(1.0 / c->beta);
            g.upart = gd.alloc<double>((size_t)g.nft * GMAXQ * g.ldF);
            g.u = gd.alloc<double>((size_t)GMAXQ * g.k);
            g.u1 = gd.alloc<double>((size_t)GMAXQ * g.k);
            g.v = gd.alloc<double>((size_t)GMAXQ * g.k);
            ok_alloc = ok_alloc && g.upart && g.u && g.u1 && g.v;
            if (tcp[i]) {
                const long long ntl = (g.n + 127) / 128;
                g.part = gd.alloc<double>((size_t)std::min<long long>(GSPLIT_CAP, ntl) * chunk_max * g.n);
                vt[i] = gd.alloc<unsigned char>((size_t)ntl * vtile);
                vexp[i] = gd.alloc<int>(16);
                vsc[i] = gd.alloc<double>(16);
                ok_alloc = ok_alloc && g.part && vt[i] && vexp[i] && vsc[i];
            }
        }
        if (!ok_alloc) {
            rc_all = KRR_E_NOMEM;
        }
        std::vector<GState> st(nprob);
        int n_vb = 0, n_seg = 0, n_act = 0, n_ft = 0, n_tri = 0, n_gn = 0, n_red = 0, items = 0, n_vs = 0;
        std::vector<int> colstart(nrhs + 1, 0);
        std::vector<int> alist;   // active problems (table order)
        bool any_tc = false;
        const double ksc = 1.0 + (o.ex2_correct ? 0.83 * 5.9604644775390625e-08 : 0.0);

        // work tables of the active problems
        auto rebuild = [&]() -> int {
            alist.clear();
            for (int i = 0; i < nprob; ++i)
                if (st[i].active) alist.push_back(i);
            n_act = (int)alist.size();
            // product splits: about four items per SM over all active problems
            long long work = 0;
            for (int i : alist)
                if (tcp[i]) work += ((probs[i].n + 127) / 128) * ((probs[i].n + 127) / 128);
            const long long target = std::max<long long>(4, (work + 4LL * ctx->num_sms - 1) / (4LL * ctx->num_sms));
            int ft = 0, tri = 0, gn = 0, red = 0, it = 0, vs = 0, np = 0;
            any_tc = false;
            for (int ai = 0; ai < n_act; ++ai) {
                const int i = alist[ai];
                GProb g = base[i];
                g.ft0 = ft;
                g.tri0 = tri;
                g.gn0 = gn;
                g.ngn = (g.n + GN_ROWS - 1) / GN_ROWS;
                g.red0 = red;
                ft += g.nft;
                tri += g.k;
                gn += g.ngn;
                red += GMAXQ * g.k;
                g.splits = 1;
                g.tc = tcp[i];
                if (tcp[i]) {
                    const int ntl = (g.n + 127) / 128, nrb = (g.n + 127) / 128;
                    int splits = (int)std::min<long long>(GSPLIT_CAP, std::max<long long>(1, (ntl + target - 1) / target));
                    splits = std::min(splits, ntl);
                    const int tps = (ntl + splits - 1) / splits;
                    splits = (ntl + tps - 1) / tps;
                    g.splits = splits;
                    PvProb& pp = h_pv[np];
                    pp = PvProb{ctxs[i]->FA, ctxs[i]->FB, vt[i], vsc[i], g.part, g.n, g.n,
                                tc_feature_kp(ctxs[i]->d), splits, tps, nrb * splits, it, 0};
                    PvPrep& pr = h_pp[np];
                    pr = PvPrep{nullptr, vt[i], vexp[i], vsc[i], g.n, g.n, ntl * 128, vs};
                    it += nrb * splits;
                    vs += (int)(((long long)std::max(16, 2 * chunk_max) * ntl * 128 + 255) / 256);
                    ++np;
                    any_tc = true;
                }
                h_gp[ai] = g;
                // GProb is indexed by table slot in the Woodbury kernels and by problem in
                // the vector kernels: keep a slot for every problem, tables use slots < n_act
            }
            n_ft = ft;
            n_tri = tri;
            n_gn = gn;
            n_red = red;
            items = it;
            n_vs = vs;
            // vector blocks, column-major over (column, problem, chunk); segments per (p, c)
            int nb = 0, nsg = 0;
            for (int c = 0; c < nrhs; ++c) {
                colstart[c] = nb;
                for (int ai = 0; ai < n_act; ++ai) {
                    const int i = alist[ai];
                    const int n = (int)probs[i].n;
                    h_seg[nsg++] = GSeg{ai, c, nb, (n + GV_ROWS - 1) / GV_ROWS};
                    for (int r0 = 0; r0 < n; r0 += GV_ROWS)
                        h_vb[nb++] = GVBlk{off[i] + (long long)c * n, ai, c, r0, std::min(n, r0 + GV_ROWS)};
                }
            }
            colstart[nrhs] = nb;
            n_vb = nb;
            n_seg = nsg;
            if (n_act == 0) return KRR_OK;
            KRR_TRY_CUDA(cudaMemcpyAsync(d_gp, h_gp, sizeof(GProb) * n_act, cudaMemcpyHostToDevice, S));
            KRR_TRY_CUDA(cudaMemcpyAsync(d_vb, h_vb, sizeof(GVBlk) * n_vb, cudaMemcpyHostToDevice, S));
            KRR_TRY_CUDA(cudaMemcpyAsync(d_seg, h_seg, sizeof(GSeg) * n_seg, cudaMemcpyHostToDevice, S));
            if (np) {
                KRR_TRY_CUDA(cudaMemcpyAsync(d_pv, h_pv, sizeof(PvProb) * np, cudaMemcpyHostToDevice, S));
            }
            return KRR_OK;
        };
        // Per-slot scalars: the device arrays are indexed by table slot (p = slot) so that a
        // rebuild must carry every active problem's scalars to its new slot.
        std::vector<int> slot_of(nprob, -1);
        auto remap_scalars = [&](const std::vector<int>& old_list) -> int {
            // gather (old slot) -> (new slot) for rz, b, act on the host: the arrays are tiny
            std::vector<double> rz_h(ns), b_h(ns);
            KRR_TRY_CUDA(cudaMemcpyAsync(rz_h.data(), d_rz, sizeof(double) * ns, cudaMemcpyDeviceToHost, S));
            KRR_TRY_CUDA(cudaMemcpyAsync(b_h.data(), d_b, sizeof(double) * ns, cudaMemcpyDeviceToHost, S));
            KRR_TRY_CUDA(cudaStreamSynchronize(S));
            std::vector<double> rz_n(ns, 0.0), b_n(ns, 0.0);
            for (int ai = 0; ai < (int)alist.size(); ++ai) {
                const int i = alist[ai];
                const int os = slot_of[i];
                if (os < 0) continue;
                for (int c = 0; c < nrhs; ++c) {
                    rz_n[(size_t)ai * nrhs + c] = rz_h[(size_t)os * nrhs + c];
                    b_n[(size_t)ai * nrhs + c] = b_h[(size_t)os * nrhs + c];
                }
            }
            (void)old_list;
            KRR_TRY_CUDA(cudaMemcpyAsync(d_rz, rz_n.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, S));
            KRR_TRY_CUDA(cudaMemcpyAsync(d_b, b_n.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, S));
            KRR_TRY_CUDA(cudaStreamSynchronize(S));
            return KRR_OK;
        };
        auto upload_act = [&]() -> int {
            for (int ai = 0; ai < n_act; ++ai)
                for (int c = 0; c < nrhs; ++c) h_act[(size_t)ai * nrhs + c] = st[alist[ai]].act[c];
            KRR_TRY_CUDA(cudaMemcpyAsync(d_act, h_act, sizeof(int) * n_act * nrhs, cudaMemcpyHostToDevice, S));
            return KRR_OK;
        };

        // ---- the product q = (K + beta I) p of every active problem, and p . q partials
        auto product = [&]() -> int {
            // problems outside the grouped launch: their own product on their own stream,
            // forked from S and joined before the first reduction, so that they overlap one
            // another and the grouped launch
            std::vector<int> forked;
            for (int ai = 0; ai < n_act; ++ai) {
                const int i = alist[ai];
                if (tcp[i]) continue;
                if (forked.empty()) KRR_TRY_CUDA(cudaEventRecord(ev_fork, S));
                krr_ctx* c = ctxs[i];
                KRR_TRY_CUDA(cudaStreamWaitEvent(streams[i], ev_fork, 0));
                c->stream = streams[i];
                const int prc = square_product(c, pv + off[i], nrhs, qv + off[i], form[i]);
                c->stream = S;
                if (prc != KRR_OK) return prc;
                KRR_TRY_CUDA(cudaEventRecord(ev_join[i], streams[i]));
                forked.push_back(i);
            }
            int c0 = 0, ci = 0;
            while (c0 < nrhs) {
                const int left = nrhs - c0;
                const int ch = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
                if (any_tc) {
                    // this chunk's V columns; a staging slot per chunk, since the copies are
                    // asynchronous and the host reuses a slot only after the iteration's sync
                    PvPrep* hs = h_pp + (size_t)ci * nprob;
                    int np = 0;
                    for (int ai = 0; ai < n_act; ++ai) {
                        const int i = alist[ai];
                        if (!tcp[i]) continue;
                        hs[np] = h_pp[np];
                        hs[np].V = pv + off[i] + (long long)c0 * probs[i].n;
                        ++np;
                    }
                    PvPrep* ds = d_pp + (size_t)ci * nprob;
                    KRR_TRY_CUDA(cudaMemcpyAsync(ds, hs, sizeof(PvPrep) * np, cudaMemcpyHostToDevice, S));
                    KRR_RET(launch_pv_prep_grouped(ctx, ds, np, n_vs, ch));
                    KRR_RET(launch_kmvm_tcpv_table(ctx, d_pv, np, items, ch, d_err));
                }
                // the reduction (tensor-core problems) or the p . q partials alone (others)
                for (int i : forked) KRR_TRY_CUDA(cudaStreamWaitEvent(S, ev_join[i], 0));
                forked.clear();
                const int b0 = colstart[c0], nb = colstart[c0 + ch] - b0;
                if (nb > 0) {
                    k_g_reduce_pq<<<nb, GV_T, 0, S>>>(d_vb, d_gp, c0, ch, ksc, any_tc, pv, qv, d_vpart, b0);
                    KRR_CHECK_LAUNCH();
                }
                c0 += ch;
                ++ci;
            }
            return KRR_OK;
        };
        // ---- z = M^-1 r of every active problem and the new directions
        auto apply_and_direction = [&]() -> int {
            KRR_TRY_CUDA(cudaMemcpyAsync(d_restart, h_restart, sizeof(int) * n_act, cudaMemcpyHostToDevice, S));
            int kmax = 1;
            for (int i : alist) kmax = std::max(kmax, ctxs[i]->k_eff);
            int q0 = 0;
            while (q0 < nrhs) {   // passes of 8, 4, 2 or 1 right-hand sides
                const int left = nrhs - q0;
                const int w = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
                auto ft = w == 8 ? &k_g_ft<8> : w == 4 ? &k_g_ft<4> : w == 2 ? &k_g_ft<2> : &k_g_ft<1>;
                auto gn = w == 8 ? &k_g_gn<8> : w == 4 ? &k_g_gn<4> : w == 2 ? &k_g_gn<2> : &k_g_gn<1>;
                ft<<<n_ft, GV_T, 0, S>>>(d_gp, n_act, q0, r);
                KRR_CHECK_LAUNCH();
                k_g_ft_reduce<<<(unsigned)ceil_div(n_red, 256), 256, 0, S>>>(d_gp, n_act, w, n_red);
                KRR_CHECK_LAUNCH();
                k_g_tri<<<n_tri, 128, 0, S>>>(d_gp, n_act, w, true);
                KRR_CHECK_LAUNCH();
                k_g_tri<<<n_tri, 128, 0, S>>>(d_gp, n_act, w, false);
                KRR_CHECK_LAUNCH();
                const size_t smem = sizeof(float) * (size_t)w * kmax;
                if (smem > 48 * 1024) KRR_RET(allow_max_dynamic_smem(ctx, (const void*)gn));
                gn<<<n_gn, GV_T, smem, S>>>(d_gp, n_act, q0, r, z, d_gnpart);
                KRR_CHECK_LAUNCH();
                k_g_beta<<<(unsigned)ceil_div((long long)n_seg * 32, 256), 256, 0, S>>>(
                    d_seg, n_seg, nrhs, q0, w, d_gp, d_gnpart, d_restart, d_rz, d_b, d_bad);
                KRR_CHECK_LAUNCH();
                q0 += w;
            }
            k_g_beta_p<<<n_vb, GV_T, 0, S>>>(d_vb, d_b, d_restart, nrhs, pv, z);
            KRR_CHECK_LAUNCH();
            return KRR_OK;
        };

        // true residuals of the problems in U, each on its own stream (forked from S, joined
        // back), so that several problems' float-float residuals run at the same time
        auto true_residuals = [&](const std::vector<int>& U) -> int {
            KRR_TRY_CUDA(cudaEventRecord(ev_fork, S));
            for (int i : U) {
                krr_ctx* c = ctxs[i];
                KRR_TRY_CUDA(cudaStreamWaitEvent(streams[i], ev_fork, 0));
                c->stream = streams[i];
                const long long tot = probs[i].n * nrhs;
                double* r64;
                KRR_RET(bufT(c, "g_r64", (size_t)tot, &r64));   // allocated before the loop
                KRR_RET(launch_accumulate(c, x + off[i], probs[i].alpha, tot));
                KRR_TRY_CUDA(cudaMemsetAsync(x + off[i], 0, sizeof(float) * tot, c->stream));
                if (o.residual == 1)
                    KRR_RET(launch_residual_hp(c, probs[i].X, probs[i].n, probs[i].d, c->sigma, c->beta,
                                               probs[i].Y, probs[i].alpha, nrhs, r64));
                else
                    KRR_RET(launch_residual_ff(c, probs[i].X, probs[i].n, probs[i].d, c->sigma, c->beta,
                                               probs[i].Y, probs[i].alpha, nrhs, r64));
                KRR_RET(launch_dot64(c, r64, r64, probs[i].n, nrhs, d_norm + (size_t)i * nrhs));
                KRR_RET(launch_convert(c, r64, r + off[i], tot));
                KRR_TRY_CUDA(cudaEventRecord(ev_join[i], streams[i]));
                c->stream = S;
            }
            for (int i : U) KRR_TRY_CUDA(cudaStreamWaitEvent(S, ev_join[i], 0));
            KRR_TRY_CUDA(cudaMemcpyAsync(h_norm, d_norm, sizeof(double) * ns, cudaMemcpyDeviceToHost, S));
            KRR_TRY_CUDA(cudaStreamSynchronize(S));
            return KRR_OK;
        };

        if (rc_all == KRR_OK) {
            rc_all = [&]() -> int {
                for (int i = 0; i < nprob; ++i) {
                    ctxs[i]->stream = S;
                    double* r64;
                    KRR_RET(bufT(ctxs[i], "g_r64", (size_t)probs[i].n * nrhs, &r64));
                    st[i].yn.assign(nrhs, 0.0);
                    st[i].rtrue.assign(nrhs, 0.0);
                    st[i].rec.assign(nrhs, 0.0);
                    st[i].act.assign(nrhs, 0);
                    if (status[i] != KRR_OK) continue;
                    const long long tot = probs[i].n * nrhs;
                    KRR_TRY_CUDA(cudaMemsetAsync(probs[i].alpha, 0, sizeof(double) * tot, S));
                    KRR_TRY_CUDA(cudaMemcpyAsync(r + off[i], probs[i].Y, sizeof(float) * tot,
                                                 cudaMemcpyDeviceToDevice, S));
                    KRR_RET(launch_dot(ctxs[i], probs[i].Y, probs[i].Y, probs[i].n, nrhs, d_norm + (size_t)i * nrhs));
                }
                KRR_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * L, S));
                KRR_TRY_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int) * nprob, S));
                KRR_TRY_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), S));
                KRR_TRY_CUDA(cudaMemsetAsync(d_rz, 0, sizeof(double) * ns, S));
                KRR_TRY_CUDA(cudaMemsetAsync(d_b, 0, sizeof(double) * ns, S));
                KRR_TRY_CUDA(cudaMemcpyAsync(h_norm, d_norm, sizeof(double) * ns, cudaMemcpyDeviceToHost, S));
                KRR_TRY_CUDA(cudaStreamSynchronize(S));
                for (int i = 0; i < nprob; ++i) {
                    if (status[i] != KRR_OK) continue;
                    bool any = false;
                    for (int c = 0; c < nrhs; ++c) {
                        const double yn = h_norm[(size_t)i * nrhs + c];
                        if (!std::isfinite(yn)) {
                            status[i] = KRR_E_NONFINITE;
                            break;
                        }
                        st[i].yn[c] = yn;
                        st[i].rtrue[c] = yn;
                        st[i].act[c] = yn > 0.0 ? 1 : 0;
                        info[i].rel_residual[c] = yn > 0.0 ? 1.0 : 0.0;
                        any = any || st[i].act[c];
                    }
                    if (status[i] != KRR_OK) continue;
                    if (!any) {
                        st[i].done = true;
                        status[i] = KRR_OK;
                        continue;
                    }
                    st[i].active = true;
                    st[i].window = o.no_precond ? o.max_iter : 500;
                }
                KRR_RET(rebuild());
                for (int ai = 0; ai < n_act; ++ai) slot_of[alist[ai]] = ai;
                KRR_RET(upload_act());
                for (int ai = 0; ai < n_act; ++ai) h_restart[ai] = 1;
                if (n_act > 0) KRR_RET(apply_and_direction());
                const double delta2 = o.inner_tol * o.inner_tol;
                while (n_act > 0) {
                    KRR_RET(product());
                    k_g_scalars<<<(unsigned)ceil_div((long long)n_seg * 32, 256), 256, 0, S>>>(
                        d_seg, n_seg, nrhs, 0, d_vpart, d_rz, d_pq, d_a, d_rr, d_act, d_bad);
                    KRR_CHECK_LAUNCH();
                    k_g_update_xr<<<n_vb, GV_T, 0, S>>>(d_vb, d_a, nrhs, x, r, pv, qv, d_vpart);
                    KRR_CHECK_LAUNCH();
                    k_g_scalars<<<(unsigned)ceil_div((long long)n_seg * 32, 256), 256, 0, S>>>(
                        d_seg, n_seg, nrhs, 1, d_vpart, d_rz, d_pq, d_a, d_rr, d_act, d_bad);
                    KRR_CHECK_LAUNCH();
                    KRR_TRY_CUDA(cudaMemcpyAsync(h_rr, d_rr, sizeof(double) * n_act * nrhs, cudaMemcpyDeviceToHost, S));
                    KRR_TRY_CUDA(cudaMemcpyAsync(h_bad, d_bad, sizeof(int) * n_act, cudaMemcpyDeviceToHost, S));
                    KRR_TRY_CUDA(cudaMemcpyAsync(h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, S));
                    KRR_TRY_CUDA(cudaStreamSynchronize(S));
                    if (*h_err) return fail(ctx, KRR_E_TIMEOUT, "tensor-core product: a bounded wait timed out");
                    std::vector<int> U;
                    bool changed = false;
                    for (int ai = 0; ai < n_act; ++ai) {
                        const int i = alist[ai];
                        GState& s = st[i];
                        h_restart[ai] = 0;
                        s.it++;
                        s.since++;
                        info[i].mvm_count++;
                        if (h_bad[ai]) {
                            if (o.escalate && form[i] != 2) {
                                // non-positive curvature in an expansion form: the correction
                                // since the last true residual is unverified and is dropped;
                                // the problem goes on from its verified alpha in form 2
                                s.esc_pending = true;
                                KRR_TRY_CUDA(cudaMemsetAsync(x + off[i], 0, sizeof(float) * probs[i].n * nrhs, S));
                                U.push_back(i);
                            } else {              // finished by its own solve
                                s.fallback = true;
                                s.active = false;
                                changed = true;
                            }
                            continue;
                        }
                        const bool last = s.it >= o.max_iter;
                        bool update = last || s.since >= s.window;
                        for (int c = 0; c < nrhs; ++c) {
                            if (!s.act[c]) continue;
                            const double rrv = h_rr[(size_t)ai * nrhs + c];
                            s.rec[c] = rrv;
                            if (rrv <= delta2 * s.rtrue[c] || rrv <= 0.25 * tol * tol * s.yn[c]) update = true;
                        }
                        if (update) U.push_back(i);
                    }
                    if (!U.empty()) {
                        KRR_RET(true_residuals(U));
                        for (int i : U) {
                            GState& s = st[i];
                            const int ai = slot_of[i];
                            krr_solve_info& inf = info[i];
                            if (inf.sweeps < 8) inf.sweep_iters[inf.sweeps] = s.since;
                            if (inf.sweeps == 0) s.window = std::max(100, 3 * s.since);
                            inf.sweeps++;
                            s.sweeps++;
                            s.since = 0;
                            std::vector<int> was(s.act);
                            double worst = 0.0;
                            bool any = false, finite = true;
                            for (int c = 0; c < nrhs; ++c) {
                                const double rn = h_norm[(size_t)i * nrhs + c];
                                const double rel = s.yn[c] > 0.0 ? std::sqrt(rn / s.yn[c]) : 0.0;
                                if (!std::isfinite(rel)) finite = false;
                                inf.rel_residual[c] = rel;
                                s.rtrue[c] = rn;
                                s.act[c] = rel > tol ? 1 : 0;
                                any = any || s.act[c];
                                worst = std::max(worst, rel);
                            }
                            if (inf.sweeps <= 8) inf.sweep_residual[inf.sweeps - 1] = worst;
                            if (!finite) {
                                s.fallback = true;
                                s.active = false;
                                changed = true;
                                continue;
                            }
                            if (!any) {
                                s.done = true;
                                s.active = false;
                                status[i] = KRR_OK;
                                changed = true;
                                continue;
                            }
                            if (s.esc_pending) {          // the breakdown's escalation
                                s.esc_pending = false;
                                form[i] = 2;
                                tcp[i] = 0;
                                s.gapped = 0;
                                s.best = worst;
                                s.it_best = s.it;
                                s.restarts++;
                                h_restart[ai] = 1;
                                changed = true;
                                continue;
                            }
                            if (s.it >= o.max_iter || s.sweeps >= o.refine_max) {
                                s.fallback = true;
                                s.active = false;
                                changed = true;
                                continue;
                            }
                            bool restart = false;
                            for (int c = 0; c < nrhs; ++c)
                                if (was[c] && s.act[c] && s.rtrue[c] > kGapRestart2 * s.rec[c]) restart = true;
                            s.gapped = restart ? s.gapped + 1 : 0;
                            if (worst < 0.5 * s.best) {
                                s.best = worst;
                                s.it_best = s.it;
                            }
                            const bool stalled = s.it - s.it_best > s.window;
                            if (o.escalate && form[i] != 2 && (s.gapped >= 2 || stalled)) {
                                // the product form, not the recurrence, limits this problem: it
                                // goes on from the replaced residual in the exact-difference form
                                // (its product then runs on its own stream)
                                form[i] = 2;
                                tcp[i] = 0;
                                s.gapped = 0;
                                s.best = worst;
                                s.it_best = s.it;
                                s.restarts++;
                                h_restart[ai] = 1;
                                changed = true;
                                continue;
                            }
                            if (stalled) {
                                restart = true;
                                s.it_best = s.it;
                                s.best = worst;
                            }
                            if (restart) {
                                s.restarts++;
                                h_restart[ai] = 1;
                            }
                        }
                    }
                    if (changed) {
                        // compact the tables to the problems still running (finished ones had
                        // their correction folded by the true residual; abandoned ones are
                        // solved again from zero by their own solve, started now)
                        for (int i = 0; i < nprob; ++i)
                            if (st[i].fallback && !fb_started[i]) start_fallback(i);
                        std::vector<int> old = alist;
                        std::vector<int> keep_restart;
                        for (int ai = 0; ai < n_act; ++ai)
                            if (st[alist[ai]].active) keep_restart.push_back(h_restart[ai]);
                        KRR_RET(rebuild());
                        KRR_RET(remap_scalars(old));
                        for (int i = 0; i < nprob; ++i) slot_of[i] = -1;
                        for (int ai = 0; ai < n_act; ++ai) {
                            slot_of[alist[ai]] = ai;
                            h_restart[ai] = keep_restart[ai];
                        }
                        KRR_TRY_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int) * nprob, S));
                    }
                    if (n_act == 0) break;
                    if (changed || !U.empty()) KRR_RET(upload_act());
                    KRR_RET(apply_and_direction());
                }
                return KRR_OK;
            }();
        }
        const double solve_ms = now_ms_g() - t0;
        for (int i = 0; i < nprob; ++i) {
            info[i].iters = st[i].it;
            info[i].restarts = st[i].restarts;
            info[i].k_eff = ctxs[i]->k_eff;
            info[i].build_ms = ctxs[i]->build_ms;
            info[i].solve_ms = solve_ms;
            info[i].product_form = form[i];
            if (st[i].done) status[i] = KRR_OK;
        }
        cudaStreamSynchronize(S);
    }
    for (auto& t : fb_threads) t.join();
    for (int i = 0; i < nprob; ++i) {
        if (!fb_started[i]) continue;
        const int it = info[i].iters, mv = info[i].mvm_count;
        info[i] = fb_info[i];
        info[i].iters += it;                 // the grouped iterations count too
        info[i].mvm_count += mv;
        info[i].status = fb_status[i];
        status[i] = fb_status[i];
    }
    for (int i = 0; i < nprob; ++i) ctxs[i]->stream = streams[i];
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (cudaEvent_t e : ev_join)
        if (e) cudaEventDestroy(e);
    cudaStreamDestroy(S);
    if (rc_all != KRR_OK && rc_all != KRR_E_TIMEOUT) {
        cleanup();
        return rc_all;
    }

    // ---- problems the grouped recurrence handed back: their own solve, in parallel
    std::atomic<int> next(0);
    std::vector<int> todo;
    for (int i = 0; i < nprob; ++i) {
        // finished in the grouped phase: status OK with every column below tol
        bool conv = status[i] == KRR_OK;
        if (conv)
            for (int c = 0; c < nrhs; ++c)
                if (!(info[i].rel_residual[c] <= tol)) conv = false;
        if (!conv && !fb_started[i] && (status[i] == KRR_OK || status[i] == KRR_E_STATE)) todo.push_back(i);
    }
    if (!todo.empty()) {
        std::vector<std::thread> pool;
        const int nw = std::min<int>(W, (int)todo.size());
        for (int w = 0; w < nw; ++w)
            pool.emplace_back([&]() {
                cudaSetDevice(dev);
                for (;;) {
                    const int slot = next.fetch_add(1);
                    if (slot >= (int)todo.size()) break;
                    const int i = todo[slot];
                    const krr_problem& p = probs[i];
                    krr_solve_info si;
                    std::memset(&si, 0, sizeof(si));
                    const int rc = krr_solve(ctxs[i], p.X, p.Y, nrhs, tol, p.alpha, &si);
                    si.iters += info[i].iters;          // the grouped iterations count too
                    si.mvm_count += info[i].mvm_count;
                    info[i] = si;
                    info[i].status = rc;
                    status[i] = rc;
                    cudaStreamSynchronize(streams[i]);
                }
            });
        for (auto& t : pool) t.join();
    }
    int worst = KRR_OK;
    for (int i = 0; i < nprob; ++i) {
        info[i].status = status[i];
        if (infos) infos[i] = info[i];
        if (statuses) statuses[i] = status[i];
        if (status[i] != KRR_OK && (worst == KRR_OK || worst == KRR_E_NOCONV)) worst = status[i];
    }
    cleanup();
    return rc_all == KRR_E_TIMEOUT ? KRR_E_TIMEOUT : worst;
}
