// One-CTA-per-instance 1D step kernel and its launch (templates shared by
// the FP64 and FP32 translation units).
#pragma once
#include <type_traits>

#include "step1d.cuh"

namespace tdse {

// Resident warps per SM the FP32 kernels of n <= 2048 are sized for (64
// registers; the FP64 kernels and larger n keep the compiler's choice).  Step
// times at 3M points, 16 -> 32 warps: n = 256 0.113 -> 0.101 ms, 512 0.117 ->
// 0.105, 1024 0.131 -> 0.116, 2048 0.142 -> 0.124 (a few hundred bytes of
// spills cost less than the latency the extra warps hide).
#ifndef P1D_MINW32
#define P1D_MINW32 32
#endif
// 512-thread FP32 kernels (n = 4096, 8192): two resident CTAs per SM (64
// registers, ~200-280 bytes spilled): 0.163 -> 0.138 ms (4096) and 0.180 ->
// 0.157 ms (8192) per step at 3M points.  n = 16384 holds 128 KB of shared
// memory, one CTA per SM either way.
#ifndef P1D_MINB512
#define P1D_MINB512 2
#endif
template <class C, int N, int T>
constexpr int p1d_min_blocks() {
    if (!std::is_same<C, float2>::value || N > 8192 || T > 512) return 1;
    if (T > 256) return P1D_MINB512;
    const int b = P1D_MINW32 * 32 / T;
    return b < 1 ? 1 : (b > 32 ? 32 : b);
}

// Threads per instance of the alternative launch shape the batch tuner may
// pick (KArgs::shape1d = 1): n = 8192 with 1024 threads (8 points each, one
// radix-8 butterfly per thread and pass, against 16 points for the default
// 512), the other n >= 512 with half the default threads (twice the points
// per thread); 0: none built for this n.
constexpr int alt_threads_1d(int N) {
    return N == 8192 ? 1024 : (N >= 512 && threads_1d(N) / 2 >= 32 ? threads_1d(N) / 2 : 0);
}

template <class C, class RT, int N, int T = threads_1d(N)>
__global__ void __launch_bounds__(T, p1d_min_blocks<C, N, T>()) k_periodic1d(const KArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step1d<C, RT, N, T>(a, blockIdx.x, threadIdx.x, CtaSync{}, reinterpret_cast<C*>(smem_raw));
}

// One-time kernel attributes (shared memory above 48 KB); done before the
// first launch and, for stream capture, by periodic1d_prepare beforehand.
template <class C, class RT, int N, int T = threads_1d(N)>
static cudaError_t prepare_n() {
    static bool configured = false;
    if (configured) return cudaSuccess;
    const size_t smem = (size_t)N * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_periodic1d<C, RT, N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_periodic1d<C, RT, N, T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) configured = true;
    return e;
}

template <class C, class RT, int N, int T = threads_1d(N)>
static cudaError_t launch_n(const KArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)N * sizeof(C);
    cudaError_t e = prepare_n<C, RT, N, T>();
    if (e != cudaSuccess) return e;
    k_periodic1d<C, RT, N, T><<<a.B, T, smem, s>>>(a);
    return cudaGetLastError();
}

// The default launch shape, or the alternative one where built and selected.
template <class C, class RT, int N>
static cudaError_t launch_shape(const KArgs& a, cudaStream_t s) {
    if constexpr (alt_threads_1d(N) > 0)
        if (a.shape1d) return launch_n<C, RT, N, alt_threads_1d(N)>(a, s);
    return launch_n<C, RT, N>(a, s);
}
template <class C, class RT, int N>
static cudaError_t prepare_shapes() {
    cudaError_t e = prepare_n<C, RT, N>();
    if constexpr (alt_threads_1d(N) > 0)
        if (e == cudaSuccess) e = prepare_n<C, RT, N, alt_threads_1d(N)>();
    return e;
}

}  // namespace tdse
