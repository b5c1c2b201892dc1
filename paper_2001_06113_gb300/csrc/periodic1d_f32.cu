// 1D periodic step kernels with FP32 transforms (mixed-precision steps),
// n = 8..16384, and for n >= 512 the alternative launch shape (half the
// threads per instance) the batch tuner may select; see periodic1d.cu.
#include "p1d_launch.cuh"

namespace tdse {

cudaError_t launch_periodic1d_f32(const KArgs& a, cudaStream_t s) {
    switch (a.n0) {
        case 8: return launch_n<float2, float2, 8>(a, s);
        case 16: return launch_n<float2, float2, 16>(a, s);
        case 32: return launch_n<float2, float2, 32>(a, s);
        case 64: return launch_n<float2, float2, 64>(a, s);
        case 128: return launch_n<float2, float2, 128>(a, s);
        case 256: return launch_n<float2, float2, 256>(a, s);
        case 512: return launch_shape<float2, float2, 512>(a, s);
        case 1024: return launch_shape<float2, float2, 1024>(a, s);
        case 2048: return launch_shape<float2, float2, 2048>(a, s);
        case 4096: return launch_shape<float2, float2, 4096>(a, s);
        case 8192: return launch_shape<float2, float2, 8192>(a, s);
        case 16384: return launch_shape<float2, float2, 16384>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

int periodic1d_f32_threads(int n, int shape) {
    if (n < 8 || n > 16384 || (n & (n - 1))) return 0;
    return shape ? alt_threads_1d(n) : threads_1d(n);
}

cudaError_t prepare_periodic1d_f32(int n) {
    switch (n) {
        case 8: return prepare_n<float2, float2, 8>();
        case 16: return prepare_n<float2, float2, 16>();
        case 32: return prepare_n<float2, float2, 32>();
        case 64: return prepare_n<float2, float2, 64>();
        case 128: return prepare_n<float2, float2, 128>();
        case 256: return prepare_n<float2, float2, 256>();
        case 512: return prepare_shapes<float2, float2, 512>();
        case 1024: return prepare_shapes<float2, float2, 1024>();
        case 2048: return prepare_shapes<float2, float2, 2048>();
        case 4096: return prepare_shapes<float2, float2, 4096>();
        case 8192: return prepare_shapes<float2, float2, 8192>();
        case 16384: return prepare_shapes<float2, float2, 16384>();
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tdse
