// 1D periodic step: one CTA per instance, the whole transform in shared memory.
//
// MODE_STEP fuses, for an instance of N modes, in one launch:
//   history Horner sum + one-step phase (eq. uadamsk)  ->  W          [registers/global]
//   inverse DFT (no 1/N)                                ->  y          [shared memory]
//   u = y / (1 + i h mu_0 V), Vu                        (diagonal implicit solve)
//   forward DFT with 1/N                                ->  R = (Vu)^
//   u^ <- W - i h mu_0 R,  ring[out] <- R
// so that the mode arrays cross HBM once per step: read u^ and the history
// slots, write u^ and one slot.  W stays in registers when each thread owns
// at most 4 modes; otherwise it is parked in u^'s own slot (L2-resident).
#include "step_common.cuh"

namespace tdse {

constexpr int threads_1d(int N) { return N / 8 < 32 ? 32 : (N / 8 > 512 ? 512 : N / 8); }

template <class C, class RT, int N>
__global__ void __launch_bounds__(threads_1d(N)) k_periodic1d(const KArgs a) {
    constexpr int T = threads_1d(N);
    constexpr int PER = (N + T - 1) / T;
    constexpr bool KEEP = PER <= 4;
    using R = typename cx_traits<C>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);

    const int b = blockIdx.x;
    const size_t NP = N;
    double2* uh = a.uhat + (size_t)b * NP;
    RT* ringb = reinterpret_cast<RT*>(a.ring) + (size_t)b * a.ring_slots * NP;
    const C* tw;
    if constexpr (is_f64<C>::value) tw = a.tw64_0; else tw = a.tw32_0;
    const double vfac = a.tfac[(size_t)b * a.ntf + a.tf];
    const double* V0 = a.V0 + (size_t)b * NP;
    const float* V0f = a.V0f + (size_t)b * NP;
    const R scale = (R)1 / (R)N;

    auto Vat = [&](int j) -> R {
        if constexpr (is_f64<C>::value) return vfac * V0[j];
        else return (R)vfac * V0f[j];
    };

    if (a.mode == MODE_INIT) {
        // (V u0)^ -> ring[out]; u0 is read from u^'s slot, overwritten below.
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int j = threadIdx.x + p * T;
            if (N % T == 0 || j < N) buf[j] = cscale(cvt<C>(uh[j]), Vat(j));
        }
        __syncthreads();
        fft_smem<C, N, 1, 1, T, false>(buf, tw);
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int k = threadIdx.x + p * T;
            if (N % T == 0 || k < N) {
                ringb[(size_t)a.out_slot * NP + k] = cvt<RT>(cscale(buf[k], scale));
                buf[k] = cvt<C>(uh[k]);
            }
        }
        __syncthreads();
        fft_smem<C, N, 1, 1, T, false>(buf, tw);
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int k = threadIdx.x + p * T;
            if (N % T == 0 || k < N) uh[k] = cvt<double2>(cscale(buf[k], scale));
        }
        return;
    }

    if (a.mode == MODE_READ) {
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int k = threadIdx.x + p * T;
            if (N % T == 0 || k < N) buf[k] = cvt<C>(uh[k]);
        }
        __syncthreads();
        fft_smem<C, N, 1, 1, T, true>(buf, tw);
        double2* out = a.aux2 + (size_t)b * NP;
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int j = threadIdx.x + p * T;
            if (N % T == 0 || j < N) out[j] = cvt<double2>(buf[j]);
        }
        return;
    }

    const bool step = (a.mode == MODE_STEP);
    double2 Wk[KEEP ? PER : 1];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int k = threadIdx.x + p * T;
        if (N % T == 0 || k < N) {
            double2 W = uh[k];
            if (step) {
                Phase1D ph{a, b, k};
                W = recurrence_W<C, RT>(a, W, ringb, NP, (size_t)k, ph);
                if constexpr (KEEP) Wk[p]= W; else uh[k] = W;
            }
            buf[k] = cvt<C>(W);
        }
    }
    __syncthreads();
    fft_smem<C, N, 1, 1, T, true>(buf, tw);
    const R hmu0 = step ? (R)(a.h * a.mu[0]) : (R)0;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int j = threadIdx.x + p * T;
        if (N % T == 0 || j < N) buf[j] = implicit_solve_times_V(buf[j], Vat(j), hmu0);
    }
    __syncthreads();
    fft_smem<C, N, 1, 1, T, false>(buf, tw);
    const double hmu0d = a.h * a.mu[0];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int k = threadIdx.x + p * T;
        if (N % T == 0 || k < N) {
            const RT r = cvt<RT>(cscale(buf[k], scale));
            ringb[(size_t)a.out_slot * NP + k] = r;
            if (step) {
                const double2 W = KEEP ? Wk[p] : uh[k];
                uh[k] = mode_update(W, cvt<double2>(r), hmu0d);
            }
        }
    }
}

template <class C, class RT, int N>
static cudaError_t launch_n(const KArgs& a, cudaStream_t s) {
    constexpr int T = threads_1d(N);
    const size_t smem = (size_t)N * sizeof(C);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_periodic1d<C, RT, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    k_periodic1d<C, RT, N><<<a.B, T, smem, s>>>(a);
    return cudaGetLastError();
}

template <class C, class RT>
static cudaError_t dispatch_n(const KArgs& a, cudaStream_t s) {
    switch (a.n0) {
        case 8: return launch_n<C, RT, 8>(a, s);
        case 16: return launch_n<C, RT, 16>(a, s);
        case 32: return launch_n<C, RT, 32>(a, s);
        case 64: return launch_n<C, RT, 64>(a, s);
        case 128: return launch_n<C, RT, 128>(a, s);
        case 256: return launch_n<C, RT, 256>(a, s);
        case 512: return launch_n<C, RT, 512>(a, s);
        case 1024: return launch_n<C, RT, 1024>(a, s);
        case 2048: return launch_n<C, RT, 2048>(a, s);
        case 4096: return launch_n<C, RT, 4096>(a, s);
        case 8192: return launch_n<C, RT, 8192>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

bool periodic1d_supported(int n) { return n >= 8 && n <= 8192 && (n & (n - 1)) == 0; }

cudaError_t launch_periodic1d(const KArgs& a, int combo, cudaStream_t s) {
    if (!periodic1d_supported(a.n0)) return cudaErrorInvalidValue;
    switch (combo) {
        case COMBO_F64: return dispatch_n<double2, double2>(a, s);
        case COMBO_F32: return dispatch_n<float2, float2>(a, s);
        case COMBO_F64_R32: return dispatch_n<double2, float2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tdse
