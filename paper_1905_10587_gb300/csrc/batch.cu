// Batched solves: many independent problems of uneven size, each built and solved as one
// krr_build_precond + krr_solve would be.
//
// A small problem (n of a few thousand) cannot fill 152 SMs: its kernel products are a
// few microseconds and its PCG iterations are bound by launch latency and the per-
// iteration host read.  The batch executor runs W worker threads; each owns a CUDA
// stream and a solver context and takes the next problem, largest n^2 first (longest
// processing time first), so up to W builds and PCG recurrences overlap on the GPU.
#include "internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

using namespace krr;

extern "C" int krr_batch_solve(const krr_problem* probs, int nprob, int nrhs, double tol,
                               unsigned long long seed, const krr_opts* opts, int workers,
                               krr_solve_info* infos, int* statuses) {
    if (!probs || nprob < 1 || nrhs < 1 || nrhs > KRR_MAX_RHS || !(tol > 0.0) || !(tol < 1.0))
        return KRR_E_INVAL;
    for (int i = 0; i < nprob; ++i) {
        const krr_problem& p = probs[i];
        if (!p.X || !p.Y || !p.alpha || p.n < 1 || p.d < 1 || p.d > KRR_MAX_DIM || p.k < 1 ||
            p.k > p.n || !(p.sigma > 0.0) || !(p.beta > 0.0))
            return KRR_E_INVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KRR_E_CUDA;
    const int W = std::max(1, std::min(workers > 0 ? workers : 8, nprob));
    std::vector<int> order(nprob);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (double)probs[a].n * probs[a].n > (double)probs[b].n * probs[b].n;
    });
    std::atomic<int> next(0);
    std::vector<int> status(nprob, KRR_E_STATE);
    std::vector<krr_solve_info> info(nprob);
    std::atomic<int> setup_error(KRR_OK);

    auto worker = [&]() {
        if (cudaSetDevice(dev) != cudaSuccess) {
            setup_error = KRR_E_CUDA;
            return;
        }
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            setup_error = KRR_E_CUDA;
            return;
        }
        krr_ctx* ctx = nullptr;
        if (krr_create(&ctx, opts, st) != KRR_OK) {
            cudaStreamDestroy(st);
            setup_error = KRR_E_CUDA;
            return;
        }
        for (;;) {
            const int slot = next.fetch_add(1);
            if (slot >= nprob) break;
            const int i = order[slot];
            const krr_problem& p = probs[i];
            std::memset(&info[i], 0, sizeof(krr_solve_info));
            int rc = krr_build_precond(ctx, p.X, p.n, p.d, p.sigma, p.beta, p.k, seed + (unsigned long long)i);
            if (rc == KRR_OK || rc == KRR_E_NOCONV)
                rc = krr_solve(ctx, p.X, p.Y, nrhs, tol, p.alpha, &info[i]);
            info[i].status = rc;
            status[i] = rc;
        }
        krr_destroy(ctx);
        cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    pool.reserve(W);
    for (int w = 0; w < W; ++w) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    if (setup_error != KRR_OK) return setup_error;
    int worst = KRR_OK;
    for (int i = 0; i < nprob; ++i) {
        if (infos) infos[i] = info[i];
        if (statuses) statuses[i] = status[i];
        if (status[i] != KRR_OK && (worst == KRR_OK || worst == KRR_E_NOCONV)) worst = status[i];
    }
    return worst;
}
