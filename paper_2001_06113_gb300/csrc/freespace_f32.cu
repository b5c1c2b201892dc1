// Free-space kernels, FP32-transform variant (TDSE_MIXED): see freespace.cuh.
#include "freespace.cuh"

namespace tdse {

cudaError_t launch_fs_f32(const FsArgs& a, int which, int flag, cudaStream_t s) {
    return fs::dispatch<float2>(a, fs::axis_of(a, which), which, flag, s);
}

}  // namespace tdse
