// Allocation-free variant of the 2D read-out transform (modes -> grid).
//
// For callers that cannot allocate device memory at all -- code running where
// cudaMalloc is forbidden or unavailable, e.g. inside a host that owns every
// allocation itself, a plugin with a fixed memory budget, or a process that
// must not grow its device footprint after start-up -- and therefore cannot
// hand the solver a workspace either.  The intermediate array of the two-pass
// transform (and the twiddle tables) live in one file-scope device array of
// fixed size instead of caller memory; the caller passes only the input modes
// and the output grid.
//
// Facts a caller must know:
//  * the array (TDSE_NOALLOC_SCRATCH_BYTES + tables) is part of the library
//    image: every GPU that loads the library holds it until the process exits;
//  * all calls share it, and it keeps the last call's contents: two calls
//    whose kernels overlap on the GPU (different streams, or different host
//    threads) race on it and give wrong results; serialise them;
//  * the first call on a device looks up the array's device address (with
//    that device current); make that first call before any stream capture.
//    The address is cached per device together with the id of the CUDA
//    context it belongs to; after a device reset (a new context) the next
//    call looks it up again, and that call too should precede any capture.
#include <cuda.h>

#include <mutex>

#include "kargs.h"
#include "tdse.h"

namespace tdse {

constexpr size_t NOALLOC_T1_BYTES = (size_t)TDSE_NOALLOC_MAX_POINTS * 16;
constexpr size_t NOALLOC_TW_OFF = NOALLOC_T1_BYTES;                 // 2 axes x 1024 x (16 + 8 + 8) bytes
constexpr size_t NOALLOC_DUMMY_OFF = NOALLOC_TW_OFF + 2 * 1024 * 32;     // one double read by the row pass
constexpr size_t NOALLOC_BYTES = NOALLOC_DUMMY_OFF + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the address of the array and the id of the CUDA context it was
// looked up in.  A device reset (cudaDeviceReset, or a primary-context reset)
// gives the device a new context in which the module, and so the array, may
// sit at another address; the id then differs and the address is looked up
// again instead of reusing a stale pointer.
void* g_addr[kMaxDevices] = {nullptr};
unsigned long long g_ctx_id[kMaxDevices] = {0};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Id of the current context (driver entry points found through the runtime,
// so the library needs no link against the driver library).
cudaError_t current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (!ctx) {         // no context yet: a runtime call creates the primary one
        *id = 0;
        return cudaSuccess;
    }
    if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    unsigned long long id = 0;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev] || id == 0 || g_ctx_id[dev] != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // creates the context if there was none
        if (e != cudaSuccess) return e;
        if (id == 0 && (e = current_context_id(&id)) != cudaSuccess) return e;
        g_addr[dev] = p;
        g_ctx_id[dev] = id;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}
}  // namespace

}  // namespace tdse

using namespace tdse;

extern "C" tdse_status tdse_modes_to_grid_2d_noalloc(const double* uhat, double* u, int n0, int n1, int batch,
                                                     void* stream) {
    if (!uhat || !u || batch < 1) return TDSE_EINVAL;
    if (!periodic2d_supported(n0, n1)) return TDSE_EINVAL;
    if ((long long)batch * n0 * n1 > (long long)TDSE_NOALLOC_MAX_POINTS) return TDSE_ENOMEM;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return TDSE_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* b = static_cast<char*>(base);
    double2* tw64_0 = reinterpret_cast<double2*>(b + NOALLOC_TW_OFF);
    double2* tw64_1 = tw64_0 + 1024;
    float2* tw32_0 = reinterpret_cast<float2*>(tw64_1 + 1024);
    float2* tw32_1 = tw32_0 + 1024;
    float2* tw32lo_0 = tw32_1 + 1024;
    float2* tw32lo_1 = tw32lo_0 + 1024;
    // The twiddles of this call's sizes are rewritten every call (stream-ordered
    // before the transform); the intermediate array needs no clearing because
    // every element is written before it is read.
    if (launch_twiddles(tw64_0, tw32_0, tw32lo_0, n0, s) != cudaSuccess) return TDSE_ECUDA;
    if (launch_twiddles(tw64_1, tw32_1, tw32lo_1, n1, s) != cudaSuccess) return TDSE_ECUDA;
    KArgs a{};
    a.mode = MODE_READ;
    a.B = batch;
    a.n0 = n0;
    a.n1 = n1;
    a.uhat = const_cast<double2*>(reinterpret_cast<const double2*>(uhat));   // only read in MODE_READ
    a.aux = reinterpret_cast<double2*>(b);                                   // intermediate [batch][n0][n1]
    a.aux2 = reinterpret_cast<double2*>(u);                                  // output grid
    a.tw64_0 = tw64_0;
    a.tw64_1 = tw64_1;
    a.tw32_0 = tw32_0;
    a.tw32_1 = tw32_1;
    a.tw32lo_0 = tw32lo_0;
    a.tw32lo_1 = tw32lo_1;
    a.tfac = reinterpret_cast<const double*>(b + NOALLOC_DUMMY_OFF);       // potential factor: unused on read-out
    a.ntf = 0;
    a.tf = 0;
    if (launch_periodic2d(a, COMBO_F64, s) != cudaSuccess) return TDSE_ECUDA;
    return TDSE_OK;
}
