// Free-space time step (Sec. 3.4, Remark highorderfs) in complex FP64.
//
// One step of eq. uadamsk on the contour modes, with zeta for k and
// zeta.zeta for |k|^2 (eq. uhatxirecur):
//   W   = p_0 (u^ - i h S_1),  S_j = mu_j R_j + p_j S_{j+1}       (mode space)
//   u   = inverse(W) / (1 + i h mu_0 V)                          (grid)
//   F   = forward(V u);   u^ <- W - i h mu_0 F;   ring <- F
// The trapezoidal sub-steps of the start-up are the same with nhist = 1 and
// mu = (1/2, 1/2) (eqs. utrapzfd, uhatzfd).
//
// Transforms (fsargs.h): each axis is split into the two equispaced blocks,
// done as R interleaved M-point FFTs with folded twiddles (eq. ssfftgen), and
// the dense block of Alpert and Gauss modes, done as a direct sum.  In shared
// memory the E buffer holds both blocks as 2R lines of length M:
// element (pos, line) at E[pos * LS + line], line = b R + s, LS = 2R + 1 (one
// pad slot against bank conflicts).  The mode i = s + R q of block b sits at
// pos q; the grid value j at pos j.
//
// Kernels:
//   k_fs_1d   one CTA per instance: the whole 1D step;
//   k_fs_row  (2D) one CTA per mode row k0: forward along axis 1 of the row
//             of the intermediate Z, mode update and ring write (end of a
//             step), then W of the next step and its inverse along axis 1
//             back into Z (begin of a step);
//   k_fs_phys (2D) one CTA per grid column j1: inverse along axis 0 of the
//             column of Z, implicit solve and V u on the grid, forward along
//             axis 0 back into the same column of Z.
#include <cuda_runtime.h>

#include "cplx.cuh"
#include "fsargs.h"

namespace tdse {
namespace {

__device__ __forceinline__ double2 zero2() { return make_double2(0.0, 0.0); }
// v * (-i c)
__device__ __forceinline__ double2 times_minus_i(double2 v, double c) { return make_double2(c * v.y, -c * v.x); }

template <int M, int R>
struct FsLine {
    static constexpr int L = 2 * R;
    static constexpr int LS = 2 * R + 1;
    static constexpr int NU = M * R;
    static constexpr int EBUF = M * LS;
    using FftF = CtaFft<double2, M, L, LS, FS_T, false>;
    using FftI = CtaFft<double2, M, L, LS, FS_T, true>;

    __device__ static __forceinline__ int epos(int b, int i) { return (i / R) * LS + b * R + (i % R); }

    // Forward transform of the M grid values f (shared, complete).  On return
    // E holds the block sums at epos(b, i) (before the post factor) and dv the
    // dense results.  Ends with a barrier.
    __device__ static void forward(const double2* f, double2* E, double2* dv, const FsAxis& ax) {
        for (int it = threadIdx.x; it < 2 * NU; it += FS_T) {
            const int b = it / NU, r = it - b * NU;
            const int j = r / R, s = r % R;
            E[j * LS + b * R + s] = cmul(f[j], __ldg(&ax.preF[it]));
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int dd = warp; dd < ax.ND; dd += FS_T / 32) {
            double2 acc = zero2();
            const double2* row = ax.Fd + (size_t)dd * M;
            for (int j = lane; j < M; j += 32) acc = acc + cmul(__ldg(&row[j]), f[j]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) dv[dd] = acc;
        }
        __syncthreads();
        FftF::run(E, ax.tw, nullptr);
    }

    // Forward result for mode m after forward().
    __device__ static __forceinline__ double2 fwd_value(int m, const double2* E, const double2* dv,
                                                        const FsAxis& ax) {
        const int NE = ax.NE, ND = ax.ND;
        if (m < NE) return cmul(E[epos(0, m)], __ldg(&ax.postF[m]));
        if (m < NE + ND) return dv[m - NE];
        const int i = m - NE - ND;
        return cmul(E[epos(1, i)], __ldg(&ax.postF[NE + i]));
    }

    // Place the mode value W_m as an input of the inverse transform.
    __device__ static __forceinline__ void stage_inv(int m, double2 W, double2* E, double2* dv, const FsAxis& ax) {
        const int NE = ax.NE, ND = ax.ND;
        if (m < NE) {
            E[epos(0, m)] = cmul(W, __ldg(&ax.preI[m]));
        } else if (m < NE + ND) {
            dv[m - NE] = W;
        } else {
            const int i = m - NE - ND;
            E[epos(1, i)] = cmul(W, __ldg(&ax.preI[NE + i]));
        }
    }

    // Zero the inputs NE..nu-1 of both blocks (the zero padding of eq. ssfftgen).
    __device__ static void zero_pad(double2* E, int NE) {
        const int per = NU - NE;
        for (int it = threadIdx.x; it < 2 * per; it += FS_T) {
            const int b = it / per, i = NE + (it - b * per);
            E[epos(b, i)] = zero2();
        }
    }

    // Inverse transform of the staged inputs into y (M values, shared).
    // Begins and ends with a barrier.
    __device__ static void inverse(double2* E, const double2* dv, double2* y, const FsAxis& ax) {
        __syncthreads();
        FftI::run(E, ax.tw, nullptr);
        for (int j = threadIdx.x; j < M; j += FS_T) {
            double2 acc = zero2();
            const double2* pj = ax.postI + (size_t)j * R;
#pragma unroll
            for (int s = 0; s < R; ++s) acc = acc + cmul(E[j * LS + s], __ldg(&pj[s]));
#pragma unroll
            for (int s = 0; s < R; ++s) acc = acc + cmul(E[j * LS + R + s], __ldg(&pj[NU + s]));
            for (int dd = 0; dd < ax.ND; ++dd) acc = acc + cmul(__ldg(&ax.Gd[(size_t)dd * M + j]), dv[dd]);
            y[j] = acc;
        }
        __syncthreads();
    }
};

// W = p_0 (u^ - i h S_1) with S_j = mu_j R_j + p_j S_{j+1} (Horner form of
// eq. uadamsk).  lag(j) returns R_j, phase(i) returns p_i.
template <class Lag, class Phase>
__device__ __forceinline__ double2 horner(const FsArgs& a, double2 uh, Lag lag, Phase phase) {
    double2 S = zero2();
#pragma unroll
    for (int j = FS_MAX_HIST; j >= 1; --j) {
        if (j <= a.nhist) {
            double2 t = cscale(lag(j), a.mu[j]);
            if (j < FS_MAX_HIST && j < a.nhist) t = t + cmul(phase(j), S);
            S = t;
        }
    }
    return cmul(phase(0), uh + times_minus_i(S, a.h));
}

// c R + b S with one rounding per fused multiply-add (complex).
__device__ __forceinline__ double2 cmul_add2(double2 c, double2 R, double2 b, double2 S) {
    return make_double2(fma(c.x, R.x, fma(-c.y, R.y, fma(b.x, S.x, -b.y * S.y))),
                        fma(c.x, R.y, fma(c.y, R.x, fma(b.x, S.y, b.y * S.x))));
}

// 2D form of the Horner recurrence with separable phases p_i = a_i b_i
// (a_i of the row, b_i of the mode):  S_j = c_j R_j + b_j S_{j+1} with the
// row constants c_j = mu_j a_1 .. a_{j-1}, so that S_1 equals the sum above;
// then W = a_0 b_0 (u^ - i h S_1).
template <class Lag, class PhaseB>
__device__ __forceinline__ double2 horner_sep(const FsArgs& a, double2 uh, const double2 (&c)[FS_MAX_HIST + 1],
                                              double2 a0, Lag lag, PhaseB phase_b) {
    double2 S = zero2();
#pragma unroll
    for (int j = FS_MAX_HIST; j >= 1; --j) {
        if (j <= a.nhist) {
            if (j < FS_MAX_HIST && j < a.nhist)
                S = cmul_add2(c[j], lag(j), phase_b(j), S);
            else
                S = cmul(c[j], lag(j));
        }
    }
    return cmul(cmul(a0, phase_b(0)), uh + times_minus_i(S, a.h));
}

// u = y / (1 + i c)
__device__ __forceinline__ double2 implicit_solve(double2 y, double c) {
    const double den = 1.0 + c * c;
    return make_double2((y.x + c * y.y) / den, (y.y - c * y.x) / den);
}

template <int M, int R>
__global__ void __launch_bounds__(FS_T) k_fs_1d(FsArgs a, int mode) {
    using Ln = FsLine<M, R>;
    extern __shared__ double2 sm[];
    double2* E = sm;
    double2* y = E + Ln::EBUF;
    double2* dv = y + M;
    const FsAxis& ax = a.ax[0];
    const int b = blockIdx.x, N = ax.N;
    const double vf = a.tfac[(size_t)b * a.ntf + a.tf];
    const double* V0 = a.V0 + (size_t)b * M;
    if (mode == FS_1D_FWD_ONLY) {
        for (int j = threadIdx.x; j < M; j += FS_T) {
            const double2 u = a.usrc[(size_t)b * M + j];
            y[j] = a.mulV ? cscale(u, vf * V0[j]) : u;
        }
        __syncthreads();
        Ln::forward(y, E, dv, ax);
        for (int m = threadIdx.x; m < N; m += FS_T) a.fdst[(size_t)b * a.fdst_bstride + m] = Ln::fwd_value(m, E, dv, ax);
        return;
    }
    double2* uh = a.uhat + (size_t)b * N;
    double2* ring = a.ring + (size_t)b * a.ring_slots * N;
    const double2* P = ax.P + (size_t)b * a.n_int * N;
    for (int m = threadIdx.x; m < N; m += FS_T) {
        const double2 W = horner(
            a, uh[m], [&](int j) { return ring[(size_t)a.hist_slot[j - 1] * N + m]; },
            [&](int i) { return __ldg(&P[(size_t)a.interval[i] * N + m]); });
        uh[m] = W;
        Ln::stage_inv(m, W, E, dv, ax);
    }
    Ln::zero_pad(E, ax.NE);
    Ln::inverse(E, dv, y, ax);
    const double hm0 = a.h * a.mu[0];
    for (int j = threadIdx.x; j < M; j += FS_T) {
        const double V = vf * V0[j];
        const double2 u = implicit_solve(y[j], hm0 * V);
        a.u[(size_t)b * M + j] = u;
        y[j] = cscale(u, V);
    }
    __syncthreads();
    Ln::forward(y, E, dv, ax);
    for (int m = threadIdx.x; m < N; m += FS_T) {
        const double2 F = Ln::fwd_value(m, E, dv, ax);
        uh[m] = uh[m] + times_minus_i(F, hm0);
        ring[(size_t)a.out_slot * N + m] = F;
    }
}

template <int M, int R>
__global__ void __launch_bounds__(FS_T) k_fs_row(FsArgs a, int flags) {
    using Ln = FsLine<M, R>;
    extern __shared__ double2 sm[];
    double2* E = sm;
    double2* f = E + Ln::EBUF;
    double2* dv = f + M;
    const FsAxis& ax = a.ax[1];
    const int k0 = blockIdx.x, b = blockIdx.y;
    const int N0 = a.ax[0].N, N1 = ax.N;
    const size_t NPm = (size_t)N0 * N1;
    double2* urow = a.uhat + (size_t)b * NPm + (size_t)k0 * N1;
    double2* zrow = a.Z + ((size_t)b * N0 + k0) * M;
    const bool end = flags & FS_ROW_END, begin = flags & FS_ROW_BEGIN;
    if (end || (flags & FS_ROW_FWD_ONLY)) {
        for (int j = threadIdx.x; j < M; j += FS_T) f[j] = zrow[j];
        __syncthreads();
        Ln::forward(f, E, dv, ax);
        if (flags & FS_ROW_FWD_ONLY) {
            double2* dst = a.fdst + (size_t)b * a.fdst_bstride + (size_t)k0 * N1;
            for (int m = threadIdx.x; m < N1; m += FS_T) dst[m] = Ln::fwd_value(m, E, dv, ax);
            return;
        }
    }
    const double2* P0 = a.ax[0].P + (size_t)b * a.n_int * N0;
    const double2* P1 = ax.P + (size_t)b * a.n_int * N1;
    double2 a0 = zero2(), cj[FS_MAX_HIST + 1];
    if (begin) {
        a0 = __ldg(&P0[(size_t)a.interval[0] * N0 + k0]);
        double2 A = make_double2(1.0, 0.0);
#pragma unroll
        for (int j = 1; j <= FS_MAX_HIST; ++j) {
            cj[j] = cscale(A, a.mu[j]);
            if (j < FS_MAX_HIST && j < a.nhist) A = cmul(A, __ldg(&P0[(size_t)a.interval[j] * N0 + k0]));
        }
    }
    const double hm0 = a.h * a.mu[0];
    double2* ring = a.ring + (size_t)b * a.ring_slots * NPm + (size_t)k0 * N1;
    for (int m = threadIdx.x; m < N1; m += FS_T) {
        double2 uh, F = zero2();
        if (end) {
            F = Ln::fwd_value(m, E, dv, ax);
            uh = urow[m] + times_minus_i(F, hm0);
            ring[(size_t)a.out_slot * NPm + m] = F;
            if (!begin) urow[m] = uh;
        } else {
            uh = urow[m];
        }
        if (begin) {
            const double2 W = horner_sep(
                a, uh, cj, a0,
                [&](int j) {
                    const int slot = a.hist_slot[j - 1];
                    return (end && slot == a.out_slot) ? F : ring[(size_t)slot * NPm + m];
                },
                [&](int i) { return __ldg(&P1[(size_t)a.interval[i] * N1 + m]); });
            urow[m] = W;
            Ln::stage_inv(m, W, E, dv, ax);
        }
    }
    if (!begin) return;
    Ln::zero_pad(E, ax.NE);
    Ln::inverse(E, dv, f, ax);
    for (int j = threadIdx.x; j < M; j += FS_T) zrow[j] = f[j];
}

template <int M, int R>
__global__ void __launch_bounds__(FS_T) k_fs_phys(FsArgs a, int from_usrc) {
    using Ln = FsLine<M, R>;
    extern __shared__ double2 sm[];
    double2* E = sm;
    double2* y = E + Ln::EBUF;
    double2* dv = y + M;
    const FsAxis& ax = a.ax[0];
    const int j1 = blockIdx.x, b = blockIdx.y;
    const int M1 = a.ax[1].M, N0 = ax.N;
    double2* zcol = a.Z + (size_t)b * N0 * M1 + j1;
    const size_t NX = (size_t)M * M1;
    const double vf = a.tfac[(size_t)b * a.ntf + a.tf];
    const double* V0 = a.V0 + (size_t)b * NX;
    if (!from_usrc) {
        for (int m = threadIdx.x; m < N0; m += FS_T) Ln::stage_inv(m, zcol[(size_t)m * M1], E, dv, ax);
        Ln::zero_pad(E, ax.NE);
        Ln::inverse(E, dv, y, ax);
        const double hm0 = a.h * a.mu[0];
        for (int j0 = threadIdx.x; j0 < M; j0 += FS_T) {
            const size_t g = (size_t)j0 * M1 + j1;
            const double V = vf * V0[g];
            const double2 u = implicit_solve(y[j0], hm0 * V);
            a.u[(size_t)b * NX + g] = u;
            y[j0] = cscale(u, V);
        }
    } else {
        for (int j0 = threadIdx.x; j0 < M; j0 += FS_T) {
            const size_t g = (size_t)j0 * M1 + j1;
            const double2 u = a.usrc[(size_t)b * NX + g];
            y[j0] = a.mulV ? cscale(u, vf * V0[g]) : u;
        }
    }
    __syncthreads();
    Ln::forward(y, E, dv, ax);
    for (int m = threadIdx.x; m < N0; m += FS_T) zcol[(size_t)m * M1] = Ln::fwd_value(m, E, dv, ax);
}

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

template <int M, int R>
constexpr size_t smem_of() {
    return (size_t)(FsLine<M, R>::EBUF + M + FS_MAX_ND) * sizeof(double2);
}

template <int M, int R>
cudaError_t launch_mr(const FsArgs& a, int which, int flag, cudaStream_t s) {
    constexpr size_t sm = smem_of<M, R>();
    cudaError_t e;
    if (which == 0) {
        e = cudaFuncSetAttribute(k_fs_1d<M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_fs_1d<M, R><<<a.B, FS_T, sm, s>>>(a, flag);
    } else if (which == 1) {
        e = cudaFuncSetAttribute(k_fs_row<M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_fs_row<M, R><<<dim3(a.ax[0].N, a.B), FS_T, sm, s>>>(a, flag);
    } else {
        e = cudaFuncSetAttribute(k_fs_phys<M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_fs_phys<M, R><<<dim3(a.ax[1].M, a.B), FS_T, sm, s>>>(a, flag);
    }
    return cudaGetLastError();
}

// (M, R) pairs built: M = 32..512, R = 4, 8, 16, nu = M R <= 4096.
#define FS_FOR_R(M_)                                                      \
    if (R == 4) return launch_mr<M_, 4>(a, which, flag, s);             \
    if (R == 8) return launch_mr<M_, 8>(a, which, flag, s);             \
    if (R == 16 && M_ * 16 <= 4096) return launch_mr<M_, (M_ * 16 <= 4096 ? 16 : 8)>(a, which, flag, s);

cudaError_t dispatch(const FsArgs& a, const FsAxis& ax, int which, int flag, cudaStream_t s) {
    const int M = ax.M, R = ax.R;
    switch (M) {
        case 32: { FS_FOR_R(32) break; }
        case 64: { FS_FOR_R(64) break; }
        case 128: { FS_FOR_R(128) break; }
        case 256: { FS_FOR_R(256) break; }
        case 512: { FS_FOR_R(512) break; }
        default: break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool fs_supported(int M, int R) {
    const bool m_ok = M == 32 || M == 64 || M == 128 || M == 256 || M == 512;
    const bool r_ok = R == 4 || R == 8 || R == 16;
    return m_ok && r_ok && M * R <= 4096;
}

size_t fs_smem_bytes(int M, int R) { return (size_t)(M * (2 * R + 1) + M + FS_MAX_ND) * sizeof(double2); }

cudaError_t launch_fs_1d(const FsArgs& a, int mode, cudaStream_t s) { return dispatch(a, a.ax[0], 0, mode, s); }
cudaError_t launch_fs_row(const FsArgs& a, int flags, cudaStream_t s) { return dispatch(a, a.ax[1], 1, flags, s); }
cudaError_t launch_fs_phys(const FsArgs& a, int from_usrc, cudaStream_t s) {
    return dispatch(a, a.ax[0], 2, from_usrc, s);
}

cudaError_t launch_fs_phase(double2* P, const double2* zeta, int N, const int2* intervals, int n_int,
                            const double* phi, double dt, cudaStream_t s) {
    if (n_int <= 0) return cudaSuccess;
    const unsigned gy = n_int < 65535 ? (unsigned)n_int : 65535u;
    k_fs_phase<<<dim3((N + 255) / 256, gy), 256, 0, s>>>(P, zeta, N, intervals, n_int, phi, dt / 8.0);
    return cudaGetLastError();
}

}  // namespace tdse
