// Free-space kernels: FP64 instantiation, phase tables and launchers
// (freespace.cuh has the kernels; freespace_f32.cu the FP32-transform ones).
#include "freespace.cuh"

namespace tdse {
namespace {

// P[iv][m] = exp(-i zeta_m^2 s + i zeta_m (phi(t1) - phi(t0))), s = t1 - t0
// (eq. uhatxirecur with zeta for k), one instance.
__global__ void k_fs_phase(double2* P, const double2* zeta, int N, const int2* iv, int n_int, const double* phi,
                           double dt8) {
    for (int it = blockIdx.y; it < n_int; it += gridDim.y) {
        const int2 q = iv[it];
        const double s = (double)(q.y - q.x) * dt8;
        const double dphi = phi[q.y] - phi[q.x];
        for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
            const double2 z = zeta[m];
            const double re = 2.0 * z.x * z.y * s - z.y * dphi;
            const double im = -(z.x * z.x - z.y * z.y) * s + z.x * dphi;
            double sn, cs;
            sincos(im, &sn, &cs);
            const double e = exp(re);
            P[(size_t)it * N + m] = make_double2(e * cs, e * sn);
        }
    }
}

__global__ void k_fs_to_f32(float2* dst, const double2* src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

cudaError_t run(const FsArgs& a, int which, int flag, int f32, cudaStream_t s) {
    if (f32) return launch_fs_f32(a, which, flag, s);
    return fs::dispatch<double2>(a, fs::axis_of(a, which), which, flag, s);
}

}  // namespace

bool fs_supported(int M, int R) {
    const bool m_ok = M == 32 || M == 64 || M == 128 || M == 256 || M == 512;
    const bool r_ok = R == 4 || R == 8 || R == 16;
    return m_ok && r_ok && M * R <= 4096;
}

cudaError_t launch_fs_1d(const FsArgs& a, int mode, int f32, cudaStream_t s) { return run(a, 0, mode, f32, s); }
cudaError_t launch_fs_row(const FsArgs& a, int flags, int f32, cudaStream_t s) { return run(a, 1, flags, f32, s); }
cudaError_t launch_fs_phys(const FsArgs& a, int from_usrc, int f32, cudaStream_t s) {
    return run(a, 2, from_usrc, f32, s);
}

cudaError_t launch_fs_phase(double2* P, const double2* zeta, int N, const int2* intervals, int n_int,
                            const double* phi, double dt, cudaStream_t s) {
    if (n_int <= 0) return cudaSuccess;
    const unsigned gy = n_int < 65535 ? (unsigned)n_int : 65535u;
    k_fs_phase<<<dim3((N + 255) / 256, gy), 256, 0, s>>>(P, zeta, N, intervals, n_int, phi, dt / 8.0);
    return cudaGetLastError();
}

cudaError_t launch_fs_to_f32(float2* dst, const double2* src, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_fs_to_f32<<<(unsigned)g, 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

}  // namespace tdse
