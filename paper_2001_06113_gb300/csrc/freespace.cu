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

// ---- FP64 residual check of the FP32-transform step
__global__ void k_fs_res_prep(double2* W, const double2* uhat, const float2* ring, size_t rstride, size_t NM,
                              size_t total, double hm0) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / NM, m = i - b * NM;
        const float2 r = ring[b * rstride + m];
        const double2 u = uhat[i];
        W[i] = make_double2(u.x - hm0 * (double)r.y, u.y + hm0 * (double)r.x);   // u^ + i hm0 R
    }
}

__global__ void k_fs_res_norms(const double2* R64, const float2* ring, size_t rstride, const double2* uhat, size_t NM,
                               double* sums) {
    const size_t b = blockIdx.y;
    double s0 = 0.0, s1 = 0.0;
    for (size_t m = blockIdx.x * (size_t)blockDim.x + threadIdx.x; m < NM; m += (size_t)gridDim.x * blockDim.x) {
        const double2 r64 = R64[b * NM + m];
        const float2 r = ring[b * rstride + m];
        const double dx = r64.x - (double)r.x, dy = r64.y - (double)r.y;
        const double2 u = uhat[b * NM + m];
        s0 += dx * dx + dy * dy;
        s1 += u.x * u.x + u.y * u.y;
    }
    __shared__ double red[2][8];
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][warp] = s0;
        red[1][warp] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            c += red[1][w];
        }
        atomicAdd(&sums[2 * b], a);
        atomicAdd(&sums[2 * b + 1], c);
    }
}

__global__ void k_fs_res_decide(const double* sums, int B, double hm0, double tol, double* rho, int* flags,
                                int* ncorr) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double r = hm0 * sqrt(sums[2 * b] / sums[2 * b + 1]);
    const int bad = !(r <= tol);
    rho[b] = r;
    flags[b] = bad;
    ncorr[b] += bad;
}

__global__ void k_fs_res_apply(const int* flags, size_t NM, size_t NX, size_t total_m, size_t total_x, double2* uhat,
                               const double2* Wc, float2* ring, size_t rstride, const double2* R64, double2* u,
                               const double2* u64) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total_m; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / NM, m = i - b * NM;
        if (!flags[b]) continue;
        uhat[i] = Wc[i];
        const double2 r = R64[i];
        ring[b * rstride + m] = make_float2((float)r.x, (float)r.y);
    }
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total_x; i += (size_t)gridDim.x * blockDim.x) {
        if (flags[i / NX]) u[i] = u64[i];
    }
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
cudaError_t launch_fs_mid(const FsArgs& a, int dir, int f32, cudaStream_t s) { return run(a, 3, dir, f32, s); }

cudaError_t launch_fs_phase(double2* P, const double2* zeta, int N, const int2* intervals, int n_int,
                            const double* phi, double dt, cudaStream_t s) {
    if (n_int <= 0) return cudaSuccess;
    const unsigned gy = n_int < 65535 ? (unsigned)n_int : 65535u;
    k_fs_phase<<<dim3((N + 255) / 256, gy), 256, 0, s>>>(P, zeta, N, intervals, n_int, phi, dt / 8.0);
    return cudaGetLastError();
}

static unsigned grid_of(size_t n) {
    size_t g = (n + 255) / 256;
    return (unsigned)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

cudaError_t launch_fs_res_prep(double2* W, const double2* uhat, const float2* ring, size_t rstride, size_t NM, int B,
                               double hm0, cudaStream_t s) {
    const size_t total = NM * (size_t)B;
    k_fs_res_prep<<<grid_of(total), 256, 0, s>>>(W, uhat, ring, rstride, NM, total, hm0);
    return cudaGetLastError();
}

cudaError_t launch_fs_res_norms(const double2* R64, const float2* ring, size_t rstride, const double2* uhat, size_t NM,
                                int B, double* sums, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(sums, 0, (size_t)B * 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    unsigned gx = grid_of(NM);
    if (gx > 256) gx = 256;
    k_fs_res_norms<<<dim3(gx, (unsigned)B), 256, 0, s>>>(R64, ring, rstride, uhat, NM, sums);
    return cudaGetLastError();
}

cudaError_t launch_fs_res_decide(const double* sums, int B, double hm0, double tol, double* rho, int* flags, int* ncorr,
                                 cudaStream_t s) {
    k_fs_res_decide<<<(B + 127) / 128, 128, 0, s>>>(sums, B, hm0, tol, rho, flags, ncorr);
    return cudaGetLastError();
}

cudaError_t launch_fs_res_apply(const int* flags, int B, size_t NM, size_t NX, double2* uhat, const double2* Wc,
                                float2* ring, size_t rstride, const double2* R64, double2* u, const double2* u64,
                                cudaStream_t s) {
    const size_t tm = NM * (size_t)B, tx = NX * (size_t)B;
    k_fs_res_apply<<<grid_of(tm > tx ? tm : tx), 256, 0, s>>>(flags, NM, NX, tm, tx, uhat, Wc, ring, rstride, R64, u,
                                                                u64);
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
