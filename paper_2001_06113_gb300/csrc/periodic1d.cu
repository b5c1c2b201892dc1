// 1D periodic step: one CTA per instance, the whole transform in shared memory.
//
// MODE_STEP fuses, for an instance of N modes, in one launch:
//   history sum + phase (eq. uadamsk, lab frame or interaction picture) -> W
//   inverse DFT (no 1/N)                                                 -> y      [shared memory]
//   u = y / (1 + i h mu_0 V), Vu                         (diagonal implicit solve)
//   forward DFT with 1/N                                                 -> R = (Vu)^
//   state update and ring write
// so that the mode arrays cross HBM once per step: read the state and the
// history slots, write the state and one slot.  The pre-FFT state value (W or
// X) stays in registers when each thread owns at most 4 modes; otherwise it is
// parked in the state's own slot (L2-resident) and read back.  This unit
// builds the FP64-transform variants; periodic1d_f32.cu the FP32 ones.
#include "p1d_launch.cuh"

namespace tdse {

cudaError_t launch_periodic1d_f32(const KArgs& a, cudaStream_t s);
cudaError_t prepare_periodic1d_f32(int n);

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

template <class C, class RT>
static cudaError_t prepare_combo(int n) {
    switch (n) {
        case 8: return prepare_n<C, RT, 8>();
        case 16: return prepare_n<C, RT, 16>();
        case 32: return prepare_n<C, RT, 32>();
        case 64: return prepare_n<C, RT, 64>();
        case 128: return prepare_n<C, RT, 128>();
        case 256: return prepare_n<C, RT, 256>();
        case 512: return prepare_n<C, RT, 512>();
        case 1024: return prepare_n<C, RT, 1024>();
        case 2048: return prepare_n<C, RT, 2048>();
        case 4096: return prepare_n<C, RT, 4096>();
        case 8192: return prepare_n<C, RT, 8192>();
        default: return cudaErrorInvalidValue;
    }
}

bool periodic1d_supported(int n) { return n >= 8 && n <= 8192 && (n & (n - 1)) == 0; }

cudaError_t periodic1d_prepare(int n, int combo) {
    switch (combo) {
        case COMBO_F64: return prepare_combo<double2, double2>(n);
        case COMBO_F32: return prepare_periodic1d_f32(n);
        case COMBO_F64_R32: return prepare_combo<double2, float2>(n);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_periodic1d(const KArgs& a, int combo, cudaStream_t s) {
    if (combo == COMBO_F32) return launch_periodic1d_f32(a, s);
    if (!periodic1d_supported(a.n0)) return cudaErrorInvalidValue;
    switch (combo) {
        case COMBO_F64: return dispatch_n<double2, double2>(a, s);
        case COMBO_F64_R32: return dispatch_n<double2, float2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tdse
