// Device tables for the periodic scheme, built once per problem in FP64.
//
//  * twiddles  tw[m] = e^{-2 pi i m / n}                      (FFT passes)
//  * 1D kinetic factors  kin[c][m] = e^{-i k^2 h_c}, h_c = dt / 2^c, for the
//    step sizes of the Richardson chains (Sec. 2.2) and the Adams step;
//  * 1D advective factors per phase interval [t_a, t_b]:
//        e^{i k (phi(t_b) - phi(t_a))} = hi[m >> lb] * lo[m & (nl - 1)]
//    with k = m - n [m >= n/2] split as (m_hi nl - n [m_hi nl >= n/2]) + m_lo;
//  * 2D separable one-step phases per interval and axis d:
//        q_d[m] = e^{-i k_d^2 h + i k_d (phi_d(t_b) - phi_d(t_a))},
//    so that exp(-i |k|^2 h + i k.(phi(t_b) - phi(t_a))) = q_0[m0] q_1[m1]
//    (the one-step spectral Green's function of eq. uhatkrecur).
// Every table is computed in FP64 (argument reduction of the large angles
// k^2 h in double precision) and also stored rounded to FP32 for the
// mixed-precision history sum.
#include "kargs.h"

namespace tdse {

__device__ __forceinline__ double kmode(int m, int n) { return (double)(m < n / 2 ? m : m - n); }

__global__ void k_twiddles(double2* tw64, float2* tw32, int n) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(-2.0 * (double)m / (double)n, &s, &c);
    tw64[m] = make_double2(c, s);
    tw32[m] = make_float2((float)c, (float)s);
}

__global__ void k_kin1d(double2* kin64, float2* kin32, int n, int L, double dt) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (m >= n || c >= L) return;
    const double k = kmode(m, n);
    const double h = dt / (double)(1 << c);
    double s, co;
    sincos(-(k * k) * h, &s, &co);
    kin64[(size_t)c * n + m] = make_double2(co, s);
    kin32[(size_t)c * n + m] = make_float2((float)co, (float)s);
}

__global__ void k_adv1d(double2* adv64, float2* adv32, const int2* iv, int n_int, const double* phi,
                        int ntf, int n, int nh, int nl) {
    const int i = blockIdx.x;
    const int b = blockIdx.y;
    const int2 ab = iv[i];
    const double dphi = phi[(size_t)b * ntf + ab.y] - phi[(size_t)b * ntf + ab.x];
    const size_t base = ((size_t)b * n_int + i) * (size_t)(nh + nl);
    for (int t = threadIdx.x; t < nh + nl; t += blockDim.x) {
        double k;
        if (t < nh) {
            const int mh = t * nl;
            k = (double)(mh >= n / 2 ? mh - n : mh);
        } else {
            k = (double)(t - nh);
        }
        double s, c;
        sincos(k * dphi, &s, &c);
        adv64[base + t] = make_double2(c, s);
        adv32[base + t] = make_float2((float)c, (float)s);
    }
}

__global__ void k_q2d(double2* q64, float2* q32, const int2* iv, int n_int, const double* phi, int ntf,
                      int n0, int n1, double dt) {
    const int i = blockIdx.x;
    const int b = blockIdx.y;
    const int2 ab = iv[i];
    const double h = (double)(ab.y - ab.x) * (dt * 0.125);
    const double* ph0 = phi + (size_t)b * 2 * ntf;
    const double* ph1 = ph0 + ntf;
    const double d0 = ph0[ab.y] - ph0[ab.x];
    const double d1 = ph1[ab.y] - ph1[ab.x];
    const size_t base = ((size_t)b * n_int + i) * (size_t)(n0 + n1);
    for (int t = threadIdx.x; t < n0 + n1; t += blockDim.x) {
        const bool ax0 = t < n0;
        const int m = ax0 ? t : t - n0;
        const double k = kmode(m, ax0 ? n0 : n1);
        const double arg = -(k * k) * h + k * (ax0 ? d0 : d1);
        double s, c;
        sincos(arg, &s, &c);
        q64[base + t] = make_double2(c, s);
        q32[base + t] = make_float2((float)c, (float)s);
    }
}

__global__ void k_to_float(float* dst, const double* src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (float)src[i];
}

struct Coef4 { double c[4]; };

__global__ void k_combine(double2* uhat, const double2* chains, size_t stride, int L, Coef4 co, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int c = 0; c < L; ++c) {
            const double2 v = chains[c * stride + i];
            re = fma(co.c[c], v.x, re);
            im = fma(co.c[c], v.y, im);
        }
        uhat[i] = make_double2(re, im);
    }
}

__global__ void k_copy_slot(char* dst, const char* ring, int ring_slots, int slot, size_t bytes_per_inst) {
    const int b = blockIdx.y;
    const char* src = ring + ((size_t)b * ring_slots + slot) * bytes_per_inst;
    char* d = dst + (size_t)b * bytes_per_inst;
    const size_t n16 = bytes_per_inst / 16;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        reinterpret_cast<int4*>(d)[i] = reinterpret_cast<const int4*>(src)[i];
}

__global__ void k_count_nonfinite(const double* x, size_t n, int* count) {
    int local = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        local += isfinite(x[i]) ? 0 : 1;
    if (local) atomicAdd(count, local);
}

static int grid_for(size_t n, int threads) {
    size_t g = (n + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g ? g : 1);
}

cudaError_t launch_twiddles(double2* tw64, float2* tw32, int n, cudaStream_t s) {
    k_twiddles<<<(n + 255) / 256, 256, 0, s>>>(tw64, tw32, n);
    return cudaGetLastError();
}

cudaError_t launch_kin1d(double2* kin64, float2* kin32, int n, int L, double dt, cudaStream_t s) {
    k_kin1d<<<dim3((n + 255) / 256, L), 256, 0, s>>>(kin64, kin32, n, L, dt);
    return cudaGetLastError();
}

cudaError_t launch_adv1d(double2* adv64, float2* adv32, const int2* intervals, int n_int, const double* phi,
                         int ntf, int B, int n, int nh, int nl, cudaStream_t s) {
    k_adv1d<<<dim3(n_int, B), 128, 0, s>>>(adv64, adv32, intervals, n_int, phi, ntf, n, nh, nl);
    return cudaGetLastError();
}

cudaError_t launch_q2d(double2* q64, float2* q32, const int2* intervals, int n_int, const double* phi, int ntf,
                       int B, int n0, int n1, double dt, cudaStream_t s) {
    k_q2d<<<dim3(n_int, B), 256, 0, s>>>(q64, q32, intervals, n_int, phi, ntf, n0, n1, dt);
    return cudaGetLastError();
}

cudaError_t launch_to_float(float* dst, const double* src, size_t n, cudaStream_t s) {
    k_to_float<<<grid_for(n, 256), 256, 0, s>>>(dst, src, n);
    return cudaGetLastError();
}

cudaError_t launch_combine(double2* uhat, const double2* chains, size_t chain_stride, int L, const double* coef,
                           size_t n, cudaStream_t s) {
    Coef4 co{};
    for (int c = 0; c < L && c < 4; ++c) co.c[c] = coef[c];
    k_combine<<<grid_for(n, 256), 256, 0, s>>>(uhat, chains, chain_stride, L, co, n);
    return cudaGetLastError();
}

cudaError_t launch_copy_slot(void* dst, const void* ring, int ring_slots, int slot, int B, size_t NP,
                             size_t elem_bytes, cudaStream_t s) {
    const size_t bytes = NP * elem_bytes;   // multiple of 16 (NP >= 8, elem 8 or 16)
    size_t gx = (bytes / 16 + 255) / 256;
    if (gx > 64) gx = 64;
    k_copy_slot<<<dim3((unsigned)gx, B), 256, 0, s>>>(
        (char*)dst, (const char*)ring, ring_slots, slot, bytes);
    return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(const double* x, size_t n, int* count, cudaStream_t s) {
    k_count_nonfinite<<<grid_for(n, 256), 256, 0, s>>>(x, n, count);
    return cudaGetLastError();
}

}  // namespace tdse
