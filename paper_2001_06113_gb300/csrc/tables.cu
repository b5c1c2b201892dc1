// Device tables for the periodic scheme, computed in FP64 once per problem.
//
//  * twiddles  tw[m] = e^{-2 pi i m / n}                              (FFT passes)
//  * one-step (relative) phases of eq. uhatkrecur, lab-frame form:
//      1D: kin[c][m] = e^{-i k^2 h_c}, h_c = dt / 2^c, and per interval
//          [t_a, t_b] e^{i k (phi(t_b) - phi(t_a))} = adv[m >> lb] adv[nh + (m & (nl-1))],
//          k = m - n [m >= n/2] split as (m_hi nl - n [m_hi nl >= n/2]) + m_lo;
//      2D: q_d[m] = e^{-i k_d^2 h + i k_d (phi_d(t_b) - phi_d(t_a))} per interval/axis;
//    stored as FP64 (FP64 mode) or double-float (mixed start-up);
//  * absolute phases for the interaction picture, E_n = e^{-i |k|^2 t_n + i k.phi(t_n)}:
//      2D: separable per axis, e_d[n][m];  1D: kinetic part split over n as
//      e^{-i k^2 n dt} = khi[n / 32][m] klo[n % 32][m], advective part as above;
//    arguments reduced in FP64, values rounded once to FP32.  Each step's E_n
//    also carries a global phase e^{i theta_n} (theta_n = 2 pi frac(n g), g the
//    golden ratio): a global phase commutes with the linear step operator and
//    cancels between E_n (applied before the inverse transform) and conj(E_n)
//    (applied after the forward transform), so the arithmetic is unchanged,
//    but the FP32 rounding errors of the transforms no longer repeat from one
//    step to the next (the grid data changes slowly between steps, so without
//    it those errors add up coherently, linearly in the number of steps).
#include "step_common.cuh"

namespace tdse {

__device__ __forceinline__ double dither_angle(int n) {
    const double g = 0.61803398874989484820;
    const double f = (double)n * g;
    return 6.28318530717958647692 * (f - floor(f));
}

__device__ __forceinline__ float4 ff_from_cs(double c, double s) { return d_to_ffc(make_double2(c, s)); }

__global__ void k_twiddles(double2* tw64, float2* tw32, float2* tw32lo, int n) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(-2.0 * (double)m / (double)n, &s, &c);
    tw64[m] = make_double2(c, s);
    const float ch = (float)c, sh = (float)s;
    tw32[m] = make_float2(ch, sh);
    tw32lo[m] = make_float2((float)(c - (double)ch), (float)(s - (double)sh));
}

__global__ void k_kin1d(double2* kin64, float4* kinff, int n, int L, double dt) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (m >= n || c >= L) return;
    const double k = kmode(m, n);
    const double h = dt / (double)(1 << c);
    double s, co;
    sincos(-(k * k) * h, &s, &co);
    if (kin64) kin64[(size_t)c * n + m] = make_double2(co, s);
    if (kinff) kinff[(size_t)c * n + m] = ff_from_cs(co, s);
}

__device__ __forceinline__ double split_k(int t, int n, int nh, int nl) {
    if (t < nh) {
        const int mh = t * nl;
        return (double)(mh >= n / 2 ? mh - n : mh);
    }
    return (double)(t - nh);
}

__global__ void k_adv1d(double2* adv64, float4* advff, const int2* iv, int n_int, const double* phi, int ntf, int n,
                        int nh, int nl) {
    const int i = blockIdx.x;
    const int2 ab = iv[i];
    const double dphi = phi[ab.y] - phi[ab.x];
    const size_t base = (size_t)i * (size_t)(nh + nl);
    for (int t = threadIdx.x; t < nh + nl; t += blockDim.x) {
        double s, c;
        sincos(split_k(t, n, nh, nl) * dphi, &s, &c);
        if (adv64) adv64[base + t] = make_double2(c, s);
        if (advff) advff[base + t] = ff_from_cs(c, s);
    }
}

// Separable one-step phases of the 2D / 3D steps, one row of n0 + n1 (+ n2)
// factors per interval: exp(-i k^2 h + i k dphi_axis) for each axis's k.
__global__ void k_q2d(double2* q64, float4* qff, const int2* iv, int n_int, const double* phi, int ntf, int n0,
                      int n1, int n2, double dt) {
    const int i = blockIdx.x;
    const int2 ab = iv[i];
    const double h = (double)(ab.y - ab.x) * (dt * 0.125);
    const double* ph1 = phi + ntf;
    const double* ph2 = phi + 2 * (size_t)ntf;
    const double d0 = phi[ab.y] - phi[ab.x];
    const double d1 = ph1[ab.y] - ph1[ab.x];
    const double d2 = n2 > 0 ? ph2[ab.y] - ph2[ab.x] : 0.0;
    const size_t base = (size_t)i * (size_t)(n0 + n1 + n2);
    for (int t = threadIdx.x; t < n0 + n1 + n2; t += blockDim.x) {
        const int ax = t < n0 ? 0 : (t < n0 + n1 ? 1 : 2);
        const int m = ax == 0 ? t : (ax == 1 ? t - n0 : t - n0 - n1);
        const double k = kmode(m, ax == 0 ? n0 : (ax == 1 ? n1 : n2));
        double s, c;
        sincos(-(k * k) * h + k * (ax == 0 ? d0 : (ax == 1 ? d1 : d2)), &s, &c);
        if (q64) q64[base + t] = make_double2(c, s);
        if (qff) qff[base + t] = ff_from_cs(c, s);
    }
}

// Absolute phases E_n per axis (interaction picture), FP32, with the dither
// angle on the axis-0 factor.
__global__ void k_e2d(float2* e, const double* phi, int ntf, int n0, int n1, int n2, double dt) {
    const int n = blockIdx.x;
    const double t = (double)n * dt;
    const double p0 = phi[8 * (size_t)n], p1 = phi[ntf + 8 * (size_t)n];
    const double p2 = n2 > 0 ? phi[2 * (size_t)ntf + 8 * (size_t)n] : 0.0;
    const double th = dither_angle(n);
    const size_t base = (size_t)n * (size_t)(n0 + n1 + n2);
    for (int j = threadIdx.x; j < n0 + n1 + n2; j += blockDim.x) {
        const int ax = j < n0 ? 0 : (j < n0 + n1 ? 1 : 2);
        const int m = ax == 0 ? j : (ax == 1 ? j - n0 : j - n0 - n1);
        const double k = kmode(m, ax == 0 ? n0 : (ax == 1 ? n1 : n2));
        double s, c;
        sincos(-(k * k) * t + k * (ax == 0 ? p0 : (ax == 1 ? p1 : p2)) + (ax == 0 ? th : 0.0), &s, &c);
        e[base + j] = make_float2((float)c, (float)s);
    }
}

__global__ void k_k1d(float2* klo, float2* khi, int nhi, int n, double dt) {
    const int r = blockIdx.y;                      // rows 0..31: klo; 32..: khi
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    const double k = kmode(m, n);
    // k^2 * steps is an exact integer below 2^53 for every supported size
    const double steps = r < E1D_NLO ? (double)r : (double)(r - E1D_NLO) * E1D_NLO;
    double s, c;
    sincos(-(k * k * steps) * dt, &s, &c);
    if (r < E1D_NLO) klo[(size_t)r * n + m] = make_float2((float)c, (float)s);
    else if (r - E1D_NLO < nhi) khi[(size_t)(r - E1D_NLO) * n + m] = make_float2((float)c, (float)s);
}

__global__ void k_a1d(float2* a1d, const double* phi, int n, int nh, int nl) {
    const int step = blockIdx.x;
    const double p = phi[8 * (size_t)step];
    const double th = dither_angle(step);
    const size_t base = (size_t)step * (size_t)(nh + nl);
    for (int t = threadIdx.x; t < nh + nl; t += blockDim.x) {
        double s, c;
        sincos(split_k(t, n, nh, nl) * p + (t < nh ? th : 0.0), &s, &c);
        a1d[base + t] = make_float2((float)c, (float)s);
    }
}

__global__ void k_split_float(float2* hilo, const double* src, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float h = (float)src[i];
        hilo[i] = make_float2(h, (float)(src[i] - (double)h));
    }
}

struct Coef4 { double c[4]; };

template <class ST>
__global__ void k_combine(ST* state, const ST* chains, size_t stride, int L, Coef4 co, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int c = 0; c < L; ++c) {
            const double2 v = st_to_d(chains[c * stride + i]);
            re = fma(co.c[c], v.x, re);
            im = fma(co.c[c], v.y, im);
        }
        state[i] = d_to_st<ST>(make_double2(re, im));
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

__global__ void k_count_nonfinite(const double* x, size_t nwords, bool ff, int* count) {
    int local = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nwords; i += (size_t)gridDim.x * blockDim.x) {
        if (ff) {
            const float2 f = reinterpret_cast<const float2*>(x)[i];
            local += (isfinite(f.x) && isfinite(f.y)) ? 0 : 1;
        } else {
            local += isfinite(x[i]) ? 0 : 1;
        }
    }
    if (local) atomicAdd(count, local);
}

struct Steps8 { int s[8]; float z[8][2]; };

// state (double-float, lab frame at step n) -> v^ = conj(E_n) u^, and ring slot
// q (FP32, lab frame at step steps.s[q]) -> r~ = z_q conj(E) R; E in FP64.
__global__ void k_to_interaction(float4* state, float2* ring, int ring_slots, const double* phi, int ntf, int d,
                                 int n0, int n1, int n2, double dt, int n, Steps8 steps, int nslots) {
    const int b = blockIdx.y;
    const size_t NP = (size_t)n0 * n1 * n2;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < NP; idx += (size_t)gridDim.x * blockDim.x) {
        const int m0 = (int)(idx / ((size_t)n1 * n2));
        const int rem = (int)(idx - (size_t)m0 * n1 * n2);
        const int m1 = rem / n2, m2 = rem - (rem / n2) * n2;
        const double k0 = kmode(m0, n0), k1 = d >= 2 ? kmode(m1, n1) : 0.0, k2 = d == 3 ? kmode(m2, n2) : 0.0;
        const double* ph = phi + (size_t)b * d * ntf;
        auto E = [&](int step) {
            double arg = d == 3 ? -(k0 * k0 + k1 * k1 + k2 * k2) * ((double)step * dt) + k0 * ph[8 * (size_t)step]
                                : -(k0 * k0 + k1 * k1) * ((double)step * dt) + k0 * ph[8 * (size_t)step];
            if (d >= 2) arg += k1 * ph[ntf + 8 * (size_t)step];
            if (d == 3) arg += k2 * ph[2 * (size_t)ntf + 8 * (size_t)step];
            double s, c;
            sincos(arg, &s, &c);
            return make_double2(c, -s);     // conj(E)
        };
        float4* sv = state + (size_t)b * NP + idx;
        *sv = d_to_ffc(cmul(E(n), ffc_to_d(*sv)));
        for (int q = 0; q < nslots; ++q) {
            if (steps.s[q] < 0) continue;
            float2* r = ring + ((size_t)b * ring_slots + q) * NP + idx;
            const double2 zq = make_double2(steps.z[q][0], steps.z[q][1]);
            const double2 v = cmul(zq, cmul(E(steps.s[q]), make_double2(r->x, r->y)));
            *r = make_float2((float)v.x, (float)v.y);
        }
    }
}

// natural order (point j = n0 c + r) <-> [r][c]; one thread per element of the destination
template <class T>
__global__ void k_transpose_1d(T* dst, const T* src, int n0, int n1, int to_passes) {
    const size_t N = (size_t)n0 * n1;
    const size_t off = (size_t)blockIdx.y * N;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        if (to_passes) {          // dst [r][c] <- src[n0 c + r]
            const size_t r = p / n1, c = p % n1;
            dst[off + p] = src[off + n0 * c + r];
        } else {                  // dst[j] <- src[r][c], j = n0 c + r
            const size_t c = p / n0, r = p % n0;
            dst[off + p] = src[off + r * n1 + c];
        }
    }
}

static int grid_for(size_t n, int threads) {
    size_t g = (n + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g ? g : 1);
}

cudaError_t launch_transpose_1d(void* dst, const void* src, int n0, int n1, int B, int elem_bytes, int to_passes,
                                cudaStream_t s) {
    const size_t N = (size_t)n0 * n1;
    const dim3 grid((unsigned)grid_for(N, 256), (unsigned)B);
    if (elem_bytes == 8)
        k_transpose_1d<double><<<grid, 256, 0, s>>>(static_cast<double*>(dst), static_cast<const double*>(src), n0, n1,
                                                    to_passes);
    else if (elem_bytes == 16)
        k_transpose_1d<double2><<<grid, 256, 0, s>>>(static_cast<double2*>(dst), static_cast<const double2*>(src), n0,
                                                     n1, to_passes);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_twiddles(double2* tw64, float2* tw32, float2* tw32lo, int n, cudaStream_t s) {
    k_twiddles<<<(n + 255) / 256, 256, 0, s>>>(tw64, tw32, tw32lo, n);
    return cudaGetLastError();
}

cudaError_t launch_kin1d(double2* kin64, float4* kinff, int n, int L, double dt, cudaStream_t s) {
    k_kin1d<<<dim3((n + 255) / 256, L), 256, 0, s>>>(kin64, kinff, n, L, dt);
    return cudaGetLastError();
}

cudaError_t launch_adv1d(double2* adv64, float4* advff, const int2* intervals, int n_int, const double* phi, int ntf,
                         int n, int nh, int nl, cudaStream_t s) {
    if (n_int <= 0) return cudaSuccess;
    k_adv1d<<<n_int, 128, 0, s>>>(adv64, advff, intervals, n_int, phi, ntf, n, nh, nl);
    return cudaGetLastError();
}

cudaError_t launch_q2d(double2* q64, float4* qff, const int2* intervals, int n_int, const double* phi, int ntf,
                       int n0, int n1, int n2, double dt, cudaStream_t s) {
    if (n_int <= 0) return cudaSuccess;
    k_q2d<<<n_int, 256, 0, s>>>(q64, qff, intervals, n_int, phi, ntf, n0, n1, n2, dt);
    return cudaGetLastError();
}

cudaError_t launch_e2d(float2* e, const double* phi, int ntf, int nsteps, int n0, int n1, int n2, double dt,
                       cudaStream_t s) {
    k_e2d<<<nsteps + 1, 256, 0, s>>>(e, phi, ntf, n0, n1, n2, dt);
    return cudaGetLastError();
}

cudaError_t launch_k1d(float2* klo, float2* khi, int nhi, int n, double dt, cudaStream_t s) {
    k_k1d<<<dim3((n + 255) / 256, E1D_NLO + nhi), 256, 0, s>>>(klo, khi, nhi, n, dt);
    return cudaGetLastError();
}

cudaError_t launch_a1d(float2* a1d, const double* phi, int ntf, int nsteps, int n, int nh, int nl, cudaStream_t s) {
    (void)ntf;
    k_a1d<<<nsteps + 1, 128, 0, s>>>(a1d, phi, n, nh, nl);
    return cudaGetLastError();
}

// phi(t) = int_0^t A for the built-in pulse A(t) = A0 sin^2(pi t / Tp)
// sin(omega t) dir (eq. phi), in closed form: with sin^2(x) = (1 - cos 2x) / 2
// and Omega = 2 pi / Tp the integrand is (A0 / 2)(sin(omega s) - (sin((omega +
// Omega) s) + sin((omega - Omega) s)) / 2), and int_0^t sin(a s) ds =
// 2 sin^2(a t / 2) / a (0 for a = 0; no cancellation for small a).
__device__ __forceinline__ double int_sin(double a, double t) {
    if (a == 0.0) return 0.0;
    const double s = sin(0.5 * a * t);
    return 2.0 * s * s / a;
}

__global__ void k_pulse_phi(double* phi, int ntf, int d, double hs, double A0, double omega, double Om,
                            double dir0, double dir1, double dir2) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < ntf; m += gridDim.x * blockDim.x) {
        const double t = (double)m * hs;
        const double v = 0.5 * A0 * (int_sin(omega, t) - 0.5 * (int_sin(omega + Om, t) + int_sin(omega - Om, t)));
        phi[m] = v * dir0;
        if (d >= 2) phi[(size_t)ntf + m] = v * dir1;
        if (d == 3) phi[2 * (size_t)ntf + m] = v * dir2;
    }
}

cudaError_t launch_pulse_phi(double* phi, int ntf, int d, double hs, double A0, double omega, double Tp,
                             const double* dir, cudaStream_t s) {
    const double Om = 2.0 * 3.14159265358979323846 / Tp;
    k_pulse_phi<<<grid_for((size_t)ntf, 256), 256, 0, s>>>(phi, ntf, d, hs, A0, omega, Om, dir[0],
                                                            d >= 2 ? dir[1] : 0.0, d == 3 ? dir[2] : 0.0);
    return cudaGetLastError();
}

cudaError_t launch_split_float(float2* hilo, const double* src, size_t n, cudaStream_t s) {
    k_split_float<<<grid_for(n, 256), 256, 0, s>>>(hilo, src, n);
    return cudaGetLastError();
}

cudaError_t launch_combine(void* state, const void* chains, size_t chain_stride, int L, const double* coef,
                           size_t n, bool ff, cudaStream_t s) {
    Coef4 co{};
    for (int c = 0; c < L && c < 4; ++c) co.c[c] = coef[c];
    if (ff)
        k_combine<float4><<<grid_for(n, 256), 256, 0, s>>>((float4*)state, (const float4*)chains, chain_stride, L,
                                                              co, n);
    else
        k_combine<double2><<<grid_for(n, 256), 256, 0, s>>>((double2*)state, (const double2*)chains, chain_stride,
                                                               L, co, n);
    return cudaGetLastError();
}

cudaError_t launch_copy_slot(void* dst, const void* ring, int ring_slots, int slot, int B, size_t NP,
                             size_t elem_bytes, cudaStream_t s) {
    const size_t bytes = NP * elem_bytes;   // multiple of 16 (NP >= 8, elem 8 or 16)
    size_t gx = (bytes / 16 + 255) / 256;
    if (gx > 64) gx = 64;
    k_copy_slot<<<dim3((unsigned)gx, B), 256, 0, s>>>((char*)dst, (const char*)ring, ring_slots, slot, bytes);
    return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(const void* x, size_t nwords, bool ff, int* count, cudaStream_t s) {
    k_count_nonfinite<<<grid_for(nwords, 256), 256, 0, s>>>((const double*)x, nwords, ff, count);
    return cudaGetLastError();
}

cudaError_t launch_to_interaction(const KArgs& a, int n, const int* slot_steps, const float* slot_z, int nslots,
                                  cudaStream_t s) {
    Steps8 st{};
    for (int q = 0; q < 8; ++q) {
        st.s[q] = q < nslots ? slot_steps[q] : -1;
        st.z[q][0] = q < nslots ? slot_z[2 * q] : 1.f;
        st.z[q][1] = q < nslots ? slot_z[2 * q + 1] : 0.f;
    }
    const int d = a.flat1d ? 1 : (a.tn2 > 0 ? 3 : (a.n1 > 1 ? 2 : 1));
    const int n0 = a.flat1d ? a.tn0 : (d == 3 ? a.tn0 : a.n0);
    const int n1 = a.flat1d ? 1 : (d == 3 ? a.tn1 : a.n1), n2 = d == 3 ? a.tn2 : 1;
    const size_t NP = (size_t)n0 * n1 * n2;
    size_t gx = (NP + 255) / 256;
    if (gx > 1024) gx = 1024;
    k_to_interaction<<<dim3((unsigned)gx, a.B), 256, 0, s>>>((float4*)a.uhat, (float2*)a.ring, a.ring_slots, a.phi,
                                                              a.ntf, d, n0, n1, n2, a.dt, n, st, nslots);
    return cudaGetLastError();
}

}  // namespace tdse
