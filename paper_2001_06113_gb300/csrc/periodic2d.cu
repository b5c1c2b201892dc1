// 2D periodic step as three shared-memory pass kernels over [B][n0][n1]
// (row-major, axis 1 contiguous).  Each pass holds LANES whole lines of the
// 2D array in shared memory, interleaved so that consecutive threads touch
// consecutive lanes:
//
//   col_begin (axis 0, LANES columns per CTA):
//       W = p_0 (u^ - i h S_1) per mode (eq. uadamsk), W -> u^'s slot,
//       inverse DFT along axis 0                       -> T1 [i0][k1]
//   row_mid   (axis 1, LANES rows per CTA):
//       inverse DFT along axis 1 -> y; u = y/(1 + i h mu_0 V); Vu;
//       forward DFT along axis 1 (1/n1)                 -> T2 [i0][k1]
//   col_end   (axis 0):
//       forward DFT along axis 0 (1/n0) -> R = (Vu)^; ring[out] <- R;
//       u^ <- W - i h mu_0 R
//
// MODE_REFRESH runs the same passes with no phase/history and beta = 0;
// MODE_INIT runs row_mid (u0 -> T1 = F1 u0, T2 = F1 V u0) and col_end
// (T1 -> u^, T2 -> ring[out]); MODE_READ runs col_begin (u^ -> T1) and
// row_mid (T1 -> u into aux2).
#include "step_common.cuh"

namespace tdse {

constexpr int LANES2D = 8;
constexpr int T2D = 256;

// ---------------------------------------------------------------- col_begin
template <class C, class RT, int N0>
__global__ void __launch_bounds__(T2D) k_col_begin(const KArgs a) {
    constexpr int L = LANES2D;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int b = blockIdx.y;
    const int c0 = blockIdx.x * L;
    const int n1 = a.n1;
    const size_t NP = (size_t)N0 * n1;
    double2* uh = a.uhat + (size_t)b * NP;
    const RT* ringb = reinterpret_cast<const RT*>(a.ring) + (size_t)b * a.ring_slots * NP;
    const C* tw;
    if constexpr (is_f64<C>::value) tw = a.tw64_0; else tw = a.tw32_0;
    const bool step = (a.mode == MODE_STEP);

    for (int item = threadIdx.x; item < N0 * L; item += T2D) {
        const int lane = item % L, m0 = item / L;
        const int m1 = c0 + lane;
        const size_t idx = (size_t)m0 * n1 + m1;
        double2 W = uh[idx];
        if (step) {
            Phase2D ph{a, b, m0, m1};
            W = recurrence_W<C, RT>(a, W, ringb, NP, idx, ph);
            uh[idx] = W;
        }
        buf[m0 * L + lane] = cvt<C>(W);
    }
    __syncthreads();
    fft_smem<C, N0, L, L, T2D, true>(buf, tw);
    C* T1 = reinterpret_cast<C*>(a.aux) + (size_t)b * NP;
    for (int item = threadIdx.x; item < N0 * L; item += T2D) {
        const int lane = item % L, i0 = item / L;
        T1[(size_t)i0 * n1 + c0 + lane] = buf[i0 * L + lane];
    }
}

// ------------------------------------------------------------------ row_mid
template <class C, int N1>
__global__ void __launch_bounds__(T2D) k_row_mid(const KArgs a) {
    constexpr int L = LANES2D;
    constexpr int LS = L + 1;
    using R = typename cx_traits<C>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int b = blockIdx.y;
    const int r0 = blockIdx.x * L;
    const int n0 = a.n0;
    const size_t NP = (size_t)n0 * N1;
    const C* tw;
    if constexpr (is_f64<C>::value) tw = a.tw64_1; else tw = a.tw32_1;
    const double vfac = a.tfac[(size_t)b * a.ntf + a.tf];
    const double* V0 = a.V0 + (size_t)b * NP;
    const float* V0f = a.V0f + (size_t)b * NP;
    auto Vat = [&](size_t idx) -> R {
        if constexpr (is_f64<C>::value) return vfac * V0[idx];
        else return (R)vfac * V0f[idx];
    };
    const R scale = (R)1 / (R)N1;

    if (a.mode == MODE_INIT) {
        // T2 = F1 (V u0), then T1 = F1 u0 (u0 is parked in u^'s slot).
        const double2* u0 = a.uhat + (size_t)b * NP;
        C* T1 = reinterpret_cast<C*>(a.aux) + (size_t)b * NP;
        C* T2 = reinterpret_cast<C*>(a.aux2) + (size_t)b * NP;
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            for (int item = threadIdx.x; item < N1 * L; item += T2D) {
                const int lane = item / N1, j1 = item % N1;
                const size_t idx = (size_t)(r0 + lane) * N1 + j1;
                const C u = cvt<C>(u0[idx]);
                buf[j1 * LS + lane] = pass == 0 ? cscale(u, Vat(idx)) : u;
            }
            __syncthreads();
            fft_smem<C, N1, L, LS, T2D, false>(buf, tw);
            C* dst = pass == 0 ? T2 : T1;
            for (int item = threadIdx.x; item < N1 * L; item += T2D) {
                const int lane = item / N1, k1 = item % N1;
                dst[(size_t)(r0 + lane) * N1 + k1] = cscale(buf[k1 * LS + lane], scale);
            }
            __syncthreads();
        }
        return;
    }

    const C* T1 = reinterpret_cast<const C*>(a.aux) + (size_t)b * NP;
    for (int item = threadIdx.x; item < N1 * L; item += T2D) {
        const int lane = item / N1, k1 = item % N1;
        buf[k1 * LS + lane] = T1[(size_t)(r0 + lane) * N1 + k1];
    }
    __syncthreads();
    fft_smem<C, N1, L, LS, T2D, true>(buf, tw);

    if (a.mode == MODE_READ) {
        double2* out = a.aux2 + (size_t)b * NP;
        for (int item = threadIdx.x; item < N1 * L; item += T2D) {
            const int lane = item / N1, j1 = item % N1;
            out[(size_t)(r0 + lane) * N1 + j1] = cvt<double2>(buf[j1 * LS + lane]);
        }
        return;
    }

    const R hmu0 = (a.mode == MODE_STEP) ? (R)(a.h * a.mu[0]) : (R)0;
    for (int item = threadIdx.x; item < N1 * L; item += T2D) {
        const int lane = item / N1, j1 = item % N1;
        const size_t idx = (size_t)(r0 + lane) * N1 + j1;
        buf[j1 * LS + lane] = implicit_solve_times_V(buf[j1 * LS + lane], Vat(idx), hmu0);
    }
    __syncthreads();
    fft_smem<C, N1, L, LS, T2D, false>(buf, tw);
    C* T2 = reinterpret_cast<C*>(a.aux2) + (size_t)b * NP;
    for (int item = threadIdx.x; item < N1 * L; item += T2D) {
        const int lane = item / N1, k1 = item % N1;
        T2[(size_t)(r0 + lane) * N1 + k1] = cscale(buf[k1 * LS + lane], scale);
    }
}

// ------------------------------------------------------------------ col_end
template <class C, class RT, int N0>
__global__ void __launch_bounds__(T2D) k_col_end(const KArgs a) {
    constexpr int L = LANES2D;
    using R = typename cx_traits<C>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int b = blockIdx.y;
    const int c0 = blockIdx.x * L;
    const int n1 = a.n1;
    const size_t NP = (size_t)N0 * n1;
    double2* uh = a.uhat + (size_t)b * NP;
    RT* ringb = reinterpret_cast<RT*>(a.ring) + (size_t)b * a.ring_slots * NP;
    const C* tw;
    if constexpr (is_f64<C>::value) tw = a.tw64_0; else tw = a.tw32_0;
    const R scale = (R)1 / (R)N0;
    const C* T2 = reinterpret_cast<const C*>(a.aux2) + (size_t)b * NP;

    for (int item = threadIdx.x; item < N0 * L; item += T2D) {
        const int lane = item % L, i0 = item / L;
        buf[i0 * L + lane] = T2[(size_t)i0 * n1 + c0 + lane];
    }
    __syncthreads();
    fft_smem<C, N0, L, L, T2D, false>(buf, tw);
    const bool step = (a.mode == MODE_STEP);
    const double hmu0 = a.h * a.mu[0];
    for (int item = threadIdx.x; item < N0 * L; item += T2D) {
        const int lane = item % L, m0 = item / L;
        const size_t idx = (size_t)m0 * n1 + c0 + lane;
        const RT r = cvt<RT>(cscale(buf[m0 * L + lane], scale));
        ringb[(size_t)a.out_slot * NP + idx] = r;
        if (step) uh[idx] = mode_update(uh[idx], cvt<double2>(r), hmu0);
    }
    if (a.mode == MODE_INIT) {
        __syncthreads();
        const C* T1 = reinterpret_cast<const C*>(a.aux) + (size_t)b * NP;
        for (int item = threadIdx.x; item < N0 * L; item += T2D) {
            const int lane = item % L, i0 = item / L;
            buf[i0 * L + lane] = T1[(size_t)i0 * n1 + c0 + lane];
        }
        __syncthreads();
        fft_smem<C, N0, L, L, T2D, false>(buf, tw);
        for (int item = threadIdx.x; item < N0 * L; item += T2D) {
            const int lane = item % L, m0 = item / L;
            uh[(size_t)m0 * n1 + c0 + lane] = cvt<double2>(cscale(buf[m0 * L + lane], scale));
        }
    }
}

// ---------------------------------------------------------------- launchers
template <class K>
static cudaError_t set_smem(K kern, size_t smem, bool& done) {
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done = true;
    return e;
}

template <class C, class RT, int N0>
static cudaError_t col_begin_n(const KArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)N0 * LANES2D * sizeof(C);
    static bool done = false;
    cudaError_t e = set_smem(k_col_begin<C, RT, N0>, smem, done);
    if (e != cudaSuccess) return e;
    k_col_begin<C, RT, N0><<<dim3(a.n1 / LANES2D, a.B), T2D, smem, s>>>(a);
    return cudaGetLastError();
}

template <class C, class RT, int N0>
static cudaError_t col_end_n(const KArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)N0 * LANES2D * sizeof(C);
    static bool done = false;
    cudaError_t e = set_smem(k_col_end<C, RT, N0>, smem, done);
    if (e != cudaSuccess) return e;
    k_col_end<C, RT, N0><<<dim3(a.n1 / LANES2D, a.B), T2D, smem, s>>>(a);
    return cudaGetLastError();
}

template <class C, int N1>
static cudaError_t row_mid_n(const KArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)N1 * (LANES2D + 1) * sizeof(C);
    static bool done = false;
    cudaError_t e = set_smem(k_row_mid<C, N1>, smem, done);
    if (e != cudaSuccess) return e;
    k_row_mid<C, N1><<<dim3(a.n0 / LANES2D, a.B), T2D, smem, s>>>(a);
    return cudaGetLastError();
}

#define TDSE_SWITCH_N(n, FN, ...)                   \
    switch (n) {                                    \
        case 8: return FN<__VA_ARGS__, 8>(a, s);    \
        case 16: return FN<__VA_ARGS__, 16>(a, s);  \
        case 32: return FN<__VA_ARGS__, 32>(a, s);  \
        case 64: return FN<__VA_ARGS__, 64>(a, s);  \
        case 128: return FN<__VA_ARGS__, 128>(a, s); \
        case 256: return FN<__VA_ARGS__, 256>(a, s); \
        case 512: return FN<__VA_ARGS__, 512>(a, s); \
        case 1024: return FN<__VA_ARGS__, 1024>(a, s); \
        default: return cudaErrorInvalidValue;      \
    }

template <class C, class RT> static cudaError_t col_begin(const KArgs& a, cudaStream_t s) { TDSE_SWITCH_N(a.n0, col_begin_n, C, RT) }
template <class C, class RT> static cudaError_t col_end(const KArgs& a, cudaStream_t s) { TDSE_SWITCH_N(a.n0, col_end_n, C, RT) }
template <class C> static cudaError_t row_mid(const KArgs& a, cudaStream_t s) { TDSE_SWITCH_N(a.n1, row_mid_n, C) }

template <class C, class RT>
static cudaError_t run2d(const KArgs& a, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    switch (a.mode) {
        case MODE_STEP:
        case MODE_REFRESH:
            if ((e = col_begin<C, RT>(a, s)) != cudaSuccess) return e;
            if ((e = row_mid<C>(a, s)) != cudaSuccess) return e;
            return col_end<C, RT>(a, s);
        case MODE_INIT:
            if ((e = row_mid<C>(a, s)) != cudaSuccess) return e;
            return col_end<C, RT>(a, s);
        case MODE_READ:
            if ((e = col_begin<C, RT>(a, s)) != cudaSuccess) return e;
            return row_mid<C>(a, s);
        default:
            return cudaErrorInvalidValue;
    }
}

bool periodic2d_supported(int n0, int n1) {
    auto ok = [](int n) { return n >= 8 && n <= 1024 && (n & (n - 1)) == 0; };
    return ok(n0) && ok(n1);
}

cudaError_t launch_periodic2d(const KArgs& a, int combo, cudaStream_t s) {
    if (!periodic2d_supported(a.n0, a.n1)) return cudaErrorInvalidValue;
    switch (combo) {
        case COMBO_F64: return run2d<double2, double2>(a, s);
        case COMBO_F32: return run2d<float2, float2>(a, s);
        case COMBO_F64_R32: return run2d<double2, float2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tdse
