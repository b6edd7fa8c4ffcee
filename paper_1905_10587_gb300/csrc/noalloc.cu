// An entry point for callers that must not allocate device memory.
//
// Some embedders cannot let a library call cudaMalloc: a host application that
// hands out all device memory from its own pool, code that runs while the CUDA
// allocator is locked or during a memory-budgeted phase, or a plugin that is only
// given pointers.  krr_kmvm_noalloc computes the same FP32 kernel product as
// krr_kmvm, but every temporary it needs lives in one fixed device array defined
// below, so the call itself allocates nothing.
#include "internal.cuh"

#include <mutex>

namespace krr {
int kmvm_into_scratch(cudaStream_t stream, int num_sms, const float* Xr, long long nr,
                      const float* Xc, long long nc, int d, double sigma, double beta,
                      const float* V, int nrhs, float* Q, unsigned char* scratch, size_t cap,
                      size_t* needed);
}

// Fixed scratch for krr_kmvm_noalloc: KRR_NOALLOC_SCRATCH_BYTES on every GPU that
// loads this library, held until the process exits.  Shared by all calls on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KRR_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 256;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices];   // device address of the scratch, per device (set-up once)
}

extern "C" int krr_kmvm_noalloc(const float* Xr, long long nr, const float* Xc, long long nc, int d,
                                double sigma, double beta, const float* V, int nrhs, float* Q,
                                void* stream, unsigned long long* scratch_needed) {
    if (scratch_needed) *scratch_needed = 0;
    if (!Xr || !Xc || !V || !Q || nr < 1 || nc < 1 || nr > 0x7fffffffLL || nc > 0x7fffffffLL ||
        d < 1 || d > KRR_MAX_DIM || nrhs < 1 || nrhs > KRR_MAX_RHS || !(sigma > 0.0) ||
        !(beta >= 0.0) || (beta != 0.0 && nr != nc))
        return KRR_E_INVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return KRR_E_CUDA;
    void* scratch = nullptr;
    {
        // the symbol's name is only a host-side stand-in: its device address is looked
        // up once per device, with that device current
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_dev_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return KRR_E_CUDA;
            }
            g_dev_ptr[dev] = p;
        }
        scratch = g_dev_ptr[dev];
    }
    size_t need = 0;
    const int rc = krr::kmvm_into_scratch((cudaStream_t)stream, sms, Xr, nr, Xc, nc, d, sigma, beta, V,
                                          nrhs, Q, static_cast<unsigned char*>(scratch),
                                          KRR_NOALLOC_SCRATCH_BYTES, &need);
    if (scratch_needed) *scratch_needed = need;
    if (rc == KRR_E_INVAL) return KRR_E_NOMEM;   // the fixed scratch is too small for this size
    return rc;
}
