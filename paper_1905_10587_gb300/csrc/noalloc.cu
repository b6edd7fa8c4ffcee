// An entry point for callers that must not allocate device memory.
//
// Some embedders cannot let a library call cudaMalloc: a host application that
// hands out all device memory from its own pool, code that runs while the CUDA
// allocator is locked or during a memory-budgeted phase, or a plugin that is only
// given pointers.  krr_kmvm_noalloc computes the same FP32 kernel product as
// krr_kmvm, but every temporary it needs lives in one fixed device array defined
// below, so the call itself allocates nothing.
#include "internal.cuh"

#include <cuda.h>

#include <mutex>

namespace krr {
int kmvm_into_scratch(cudaStream_t stream, int num_sms, const float* Xr, long long nr,
                      const float* Xc, long long nc, int d, double sigma, double beta,
                      const float* V, int nrhs, float* Q, unsigned char* scratch, size_t cap,
                      size_t* needed);
}

// Fixed scratch for krr_kmvm_noalloc: KRR_NOALLOC_SCRATCH_BYTES on every GPU that
// loads this library's device code, held until the process exits.  Shared by all
// calls on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KRR_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 256;

// In host code the name g_noalloc_scratch is a host-side stand-in, not a device
// address; the device address belongs to the CUDA context the module was loaded
// into.  It is looked up with that context current and cached together with the
// context's unique id, so a context created later on the same device (after a
// cudaDeviceReset, or a different non-primary context) is looked up afresh instead
// of receiving a stale pointer.
struct ScratchAddr {
    unsigned long long ctx_id = 0;
    void* ptr = nullptr;
};
std::mutex g_mu;
ScratchAddr g_addr[kMaxDevices];

typedef CUresult (*ctx_get_current_fn)(CUcontext*);
typedef CUresult (*ctx_get_id_fn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if it cannot be read).  The
// driver calls are reached through the runtime's entry-point table, so the library
// keeps no link-time dependency on the driver library.
unsigned long long current_context_id() {
    static ctx_get_current_fn get_cur = nullptr;
    static ctx_get_id_fn get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<ctx_get_current_fn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<ctx_get_id_fn>(f);
        cudaGetLastError();
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}
}  // namespace

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
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return KRR_E_CUDA;
    }
    // The first call on a device looks the array up, which makes the runtime set up its
    // context and load this module there, committing the array: make that call before
    // memory runs short and before any stream capture.
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        ScratchAddr& a = g_addr[dev];
        const unsigned long long cid = current_context_id();
        if (!a.ptr || cid == 0 || a.ctx_id != cid) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                a = ScratchAddr{};
                // under lazy module loading the array is committed by this lookup
                return e == cudaErrorMemoryAllocation ? KRR_E_NOMEM : KRR_E_CUDA;
            }
            a.ptr = p;
            a.ctx_id = current_context_id();   // 0 (unreadable): looked up again next call
        }
        scratch = a.ptr;
    }
    size_t need = 0;
    const int rc = krr::kmvm_into_scratch((cudaStream_t)stream, sms, Xr, nr, Xc, nc, d, sigma, beta, V,
                                          nrhs, Q, static_cast<unsigned char*>(scratch),
                                          KRR_NOALLOC_SCRATCH_BYTES, &need);
    if (scratch_needed) *scratch_needed = need;
    return rc;
}
