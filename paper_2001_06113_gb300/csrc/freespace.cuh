// Free-space time step (Sec. 3.4, Remark highorderfs), templated on the
// transform type: complex FP64 (double2) or the FP32-transform variant
// (float2: transforms, V u and the history sum in FP32; the mode state, its
// one-step phase p_0 and the update in FP64).
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
//   k_fs_row  (2D, 3D) one CTA per mode row (k0 in 2D, (k0, k1) in 3D):
//             forward along the last axis of the row of the intermediate Z,
//             mode update and ring write (end of a step), then W of the next
//             step and its inverse along the last axis back into Z (begin of
//             a step);
//   k_fs_mid  (3D) one CTA per line (k0, j2) along axis 1: inverse from the
//             N1 modes in Z to the M1 grid values in Y, or forward back;
//   k_fs_phys (2D, 3D) one CTA per grid column (j1 in 2D, (j1, j2) in 3D):
//             inverse along axis 0 of the column of Z (3D: Y), implicit solve
//             and V u on the grid, forward along axis 0 back into the same
//             column.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "cplx.cuh"
#include "fsargs.h"

namespace tdse {
namespace fs {

// Resident CTAs per SM the register allocation is sized for: the FP64
// kernels keep the FP64 pipe busy at two CTAs (left to itself the compiler
// takes 152 registers for the row pass: one CTA per SM, 2.46 against 2.26 ms
// per 256^2 step); the FP32 ones wait on memory latency and need more warps in
// flight (per 256^2 step: 2 or 3 CTAs 0.45 ms, 4 CTAs (64 registers) 0.430,
// 5 CTAs (51 registers, more spilled) 0.400, 6 CTAs 0.426 ms).
#ifndef FS_MINB32
#define FS_MINB32 5
#endif
// The same budget for the short-line kernels (FsThr below), in 256-thread
// CTA equivalents: measured at 4.
#ifndef FS_MINB32_SMALL
#define FS_MINB32_SMALL 4
#endif
template <class C> struct MinBlocks { static constexpr int value = 2; };   // FP64: 128 registers, 2 CTAs/SM
template <> struct MinBlocks<float2> { static constexpr int value = FS_MINB32; };
// Threads per CTA: FS_T for the FP64 kernels, FS_T32 for the FP32 ones (512
// threads at two CTAs per SM measured slower than 256 at four: 0.467 against
// 0.409 ms per 256^2 step).
#ifndef FS_T32
#define FS_T32 FS_T
#endif
template <class C> struct FsThreads { static constexpr int value = FS_T; };
template <> struct FsThreads<float2> { static constexpr int value = FS_T32; };
// Lines of at most 64 points (the 3D axes of the 64^3 workload): FS_T_SMALL
// threads per CTA and proportionally more resident CTAs, since the FFT, the
// dense-row and the grid phases of such a line keep only 64 threads busy and
// the CTA's barriers then stall the rest.  Per 64^3 Adams step (nu = 256):
// 256 / 128 / 64 threads 4.99 / 3.19 / 2.30 ms with FP32 transforms,
// 18.1 / 14.3 / 13.7 ms in FP64 (same results).  Not for longer lines: the
// 256-point lines of the 2D 256^2 step (nu = 2048) with 128 / 64 threads
// 0.634 / 1.204 ms against 0.438 ms (FP32 transforms), 2.26 / 3.24 against
// 2.25 ms (FP64).
#ifndef FS_T_SMALL
#define FS_T_SMALL 64
#endif
#ifndef FS_SMALL_M
#define FS_SMALL_M 64
#endif
template <class C, int M> struct FsThr {
    static constexpr int value =
        M <= FS_SMALL_M && FS_T_SMALL < FsThreads<C>::value ? FS_T_SMALL : FsThreads<C>::value;
};
template <class C, int M> struct FsMinB {
    static constexpr bool SMALL = FsThr<C, M>::value < FsThreads<C>::value;
    static constexpr int base = (SMALL && std::is_same<C, float2>::value) ? FS_MINB32_SMALL : MinBlocks<C>::value;
    static constexpr int value = base * FsThreads<C>::value / FsThr<C, M>::value;
};

__device__ __forceinline__ double2 zero2() { return make_double2(0.0, 0.0); }
template <class C> __device__ __forceinline__ C zeroc() { return czero<C>(); }
// v * (-i c)
__device__ __forceinline__ double2 times_minus_i(double2 v, double c) { return make_double2(c * v.y, -c * v.x); }

// Tables of an axis in the transform type C.
template <class C> struct Tab;
template <> struct Tab<double2> {
    static __device__ __forceinline__ const double2* preI(const FsAxis& a) { return a.preI; }
    static __device__ __forceinline__ const double2* postI(const FsAxis& a) { return a.postI; }
    static __device__ __forceinline__ const double2* preF(const FsAxis& a) { return a.preF; }
    static __device__ __forceinline__ const double2* postF(const FsAxis& a) { return a.postF; }
    static __device__ __forceinline__ const double2* Gd(const FsAxis& a) { return a.Gd; }
    static __device__ __forceinline__ const double2* Fd(const FsAxis& a) { return a.Fd; }
    static __device__ __forceinline__ const double2* tw(const FsAxis& a) { return a.tw; }
    static __device__ __forceinline__ const double2* P(const FsAxis& a) { return a.P; }
    static __device__ __forceinline__ const double2* Lf(const FsAxis& a) { return a.Lf; }
    static __device__ __forceinline__ const double2* Li(const FsAxis& a) { return a.Li; }
    static __device__ __forceinline__ const double* Tc(const FsAxis& a) { return a.Tc; }
    static __device__ __forceinline__ const double2* TcW(const FsAxis& a) { return a.TcW; }
};
template <> struct Tab<float2> {
    static __device__ __forceinline__ const float2* preI(const FsAxis& a) { return a.preI_f; }
    static __device__ __forceinline__ const float2* postI(const FsAxis& a) { return a.postI_f; }
    static __device__ __forceinline__ const float2* preF(const FsAxis& a) { return a.preF_f; }
    static __device__ __forceinline__ const float2* postF(const FsAxis& a) { return a.postF_f; }
    static __device__ __forceinline__ const float2* Gd(const FsAxis& a) { return a.Gd_f; }
    static __device__ __forceinline__ const float2* Fd(const FsAxis& a) { return a.Fd_f; }
    static __device__ __forceinline__ const float2* tw(const FsAxis& a) { return a.tw_f; }
    static __device__ __forceinline__ const float2* P(const FsAxis& a) { return a.P_f; }
    static __device__ __forceinline__ const float2* Lf(const FsAxis& a) { return a.Lf_f; }
    static __device__ __forceinline__ const float2* Li(const FsAxis& a) { return a.Li_f; }
    static __device__ __forceinline__ const float* Tc(const FsAxis& a) { return a.Tc_f; }
    static __device__ __forceinline__ const float2* TcW(const FsAxis& a) { return a.TcW_f; }
};

template <class C, int M, int R>
struct FsLine {
    using T = Tab<C>;
    static constexpr int L = 2 * R;
    static constexpr int LS = 2 * R + 1;
    static constexpr int NU = M * R;
    static constexpr int EBUF = M * LS;
    using FftF = CtaFft<C, M, L, LS, FsThr<C, M>::value, false>;
    using FftI = CtaFft<C, M, L, LS, FsThr<C, M>::value, true>;

    __device__ static __forceinline__ int epos(int b, int i) { return (i / R) * LS + b * R + (i % R); }

    // Forward transform of the M grid values f (shared, complete).  On return
    // E holds the block sums at epos(b, i) (before the post factor) and dv the
    // dense results.  Ends with a barrier.
    __device__ static void forward(const C* f, C* E, C* dv, const FsAxis& ax) {
        const C* preF = T::preF(ax);
        for (int it = threadIdx.x; it < 2 * NU; it += FsThr<C, M>::value) {
            const int b = it / NU, r = it - b * NU;
            const int j = r / R, s = r % R;
            E[j * LS + b * R + s] = cmul(f[j], __ldg(&preF[it]));
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const bool cheb = ax.NT > 0;
        // one warp per row: the dense rows by direct sums (the C rows too
        // unless they go through the interpolant), then the NT interpolant rows
        const int nrow = ax.ND + (cheb ? ax.NT : 0);
        for (int rr = warp; rr < nrow; rr += FsThr<C, M>::value / 32) {
            if (cheb && rr >= ax.p && rr < ax.p + ax.NC) continue;
            const bool crow = rr >= ax.ND;
            const C* row = crow ? T::Lf(ax) + (size_t)(rr - ax.ND) * M : T::Fd(ax) + (size_t)rr * M;
            C acc = zeroc<C>();
            for (int j = lane; j < M; j += 32) acc = acc + cmul(__ldg(&row[j]), f[j]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            }
            if (lane == 0) {
                if (crow) dv[FS_MAX_ND + rr - ax.ND] = acc;      // g_l = sum_j (2/M) lambda_l(x_j) f_j
                else dv[rr] = acc;
            }
        }
        __syncthreads();
        if (cheb) {   // C rows: f^_k = sum_l T_l(tau_k / H) g_l
            for (int k = threadIdx.x; k < ax.NC; k += FsThr<C, M>::value) {
                const auto* tc = T::Tc(ax) + (size_t)k * ax.NT;
                C acc = zeroc<C>();
                for (int l = 0; l < ax.NT; ++l) acc = acc + cscale(dv[FS_MAX_ND + l], __ldg(&tc[l]));
                dv[ax.p + k] = acc;
            }
        }
        FftF::run(E, T::tw(ax), nullptr);   // begins with reads of E only; ends with a barrier
    }

    // Forward result for mode m after forward().
    __device__ static __forceinline__ C fwd_value(int m, const C* E, const C* dv, const FsAxis& ax) {
        const int NE = ax.NE, ND = ax.ND;
        if (m < NE) return cmul(E[epos(0, m)], __ldg(&T::postF(ax)[m]));
        if (m < NE + ND) return dv[m - NE];
        const int i = m - NE - ND;
        return cmul(E[epos(1, i)], __ldg(&T::postF(ax)[NE + i]));
    }

    // Place the mode value W_m as an input of the inverse transform.
    __device__ static __forceinline__ void stage_inv(int m, C W, C* E, C* dv, const FsAxis& ax) {
        const int NE = ax.NE, ND = ax.ND;
        if (m < NE) {
            E[epos(0, m)] = cmul(W, __ldg(&T::preI(ax)[m]));
        } else if (m < NE + ND) {
            dv[m - NE] = W;
        } else {
            const int i = m - NE - ND;
            E[epos(1, i)] = cmul(W, __ldg(&T::preI(ax)[NE + i]));
        }
    }

    // Zero the inputs NE..nu-1 of both blocks (the zero padding of eq. ssfftgen).
    __device__ static void zero_pad(C* E, int NE) {
        const int per = NU - NE;
        for (int it = threadIdx.x; it < 2 * per; it += FsThr<C, M>::value) {
            const int b = it / per, i = NE + (it - b * per);
            E[epos(b, i)] = zeroc<C>();
        }
    }

    // Inverse transform of the staged inputs into y (M values, shared).
    // Begins and ends with a barrier.
    __device__ static void inverse(C* E, const C* dv, C* y, const FsAxis& ax) {
        __syncthreads();
        const bool cheb = ax.NT > 0;
        if (cheb) {   // h_l = sum_k T_l(tau_k / H) (w_k / 2pi) f^_k (read after FftI's barriers)
            C* hb = const_cast<C*>(dv) + FS_MAX_ND;
            for (int l = threadIdx.x; l < ax.NT; l += FsThr<C, M>::value) {
                const C* tw = T::TcW(ax) + (size_t)l * ax.NC;
                C acc = zeroc<C>();
                for (int k = 0; k < ax.NC; ++k) acc = acc + cmul(__ldg(&tw[k]), dv[ax.p + k]);
                hb[l] = acc;
            }
        }
        FftI::run(E, T::tw(ax), nullptr);
        for (int j = threadIdx.x; j < M; j += FsThr<C, M>::value) {
            C acc = zeroc<C>();
            const C* pj = T::postI(ax) + (size_t)j * R;
#pragma unroll
            for (int s = 0; s < R; ++s) acc = acc + cmul(E[j * LS + s], __ldg(&pj[s]));
#pragma unroll
            for (int s = 0; s < R; ++s) acc = acc + cmul(E[j * LS + R + s], __ldg(&pj[NU + s]));
            const C* gd = T::Gd(ax);
            if (!cheb) {
                for (int dd = 0; dd < ax.ND; ++dd) acc = acc + cmul(__ldg(&gd[(size_t)dd * M + j]), dv[dd]);
            } else {   // Alpert rows directly, the C rows as sum_l rho_l(x_j) h_l
                for (int dd = 0; dd < ax.p; ++dd) acc = acc + cmul(__ldg(&gd[(size_t)dd * M + j]), dv[dd]);
                for (int dd = ax.p + ax.NC; dd < ax.ND; ++dd)
                    acc = acc + cmul(__ldg(&gd[(size_t)dd * M + j]), dv[dd]);
                const C* li = T::Li(ax);
                for (int l = 0; l < ax.NT; ++l) acc = acc + cmul(__ldg(&li[(size_t)l * M + j]), dv[FS_MAX_ND + l]);
            }
            y[j] = acc;
        }
        __syncthreads();
    }
};

// c R + b S with one rounding per fused multiply-add (complex).
__device__ __forceinline__ double2 cmul_add2(double2 c, double2 R, double2 b, double2 S) {
    return make_double2(fma(c.x, R.x, fma(-c.y, R.y, fma(b.x, S.x, -b.y * S.y))),
                        fma(c.x, R.y, fma(c.y, R.x, fma(b.x, S.y, b.y * S.x))));
}
__device__ __forceinline__ float2 cmul_add2(float2 c, float2 R, float2 b, float2 S) {
    return make_float2(fmaf(c.x, R.x, fmaf(-c.y, R.y, fmaf(b.x, S.x, -b.y * S.y))),
                       fmaf(c.x, R.y, fmaf(c.y, R.x, fmaf(b.x, S.y, b.y * S.x))));
}

// History sum of eq. uadamsk in Horner form with separable phases p_i = a_i b_i
// (a_i of the row, b_i of the mode; 1D: a_i = 1):  S_j = c_j R_j + b_j S_{j+1},
// c_j = mu_j a_1 .. a_{j-1}, so that S_1 = sum_j mu_j p_1 .. p_{j-1} R_j.
// In the transform type C (FP32 in the FP32-transform variant).
template <class C, class Lag, class PhaseB>
__device__ __forceinline__ C history_sep(const FsArgs& a, const C (&c)[FS_MAX_HIST + 1], Lag lag, PhaseB phase_b) {
    C S = zeroc<C>();
#pragma unroll
    for (int j = FS_MAX_HIST; j >= 1; --j) {
        if (j <= a.nhist) {
            if (j < FS_MAX_HIST && j < a.nhist)
                S = cmul_add2(c[j], lag(j), phase_b(j), S);
            else
                S = cmul(c[j], lag(j));
        }
    }
    return S;
}

// W = p_0 (u^ - i h S_1) in FP64 (the state recurrence keeps FP64 in both variants).
__device__ __forceinline__ double2 begin_W(const FsArgs& a, double2 uh, double2 p0, double2 S) {
    return cmul(p0, uh + times_minus_i(S, a.h));
}

// u = y / (1 + i c)
template <class C, class Rl>
__device__ __forceinline__ C implicit_solve(C y, Rl c) {
    const Rl den = (Rl)1 + c * c;
    C u;
    u.x = (y.x + c * y.y) / den;
    u.y = (y.y - c * y.x) / den;
    return u;
}

template <class C>
__device__ __forceinline__ void store_fwd(const FsArgs& a, size_t idx, C F) {
    if (a.fdst_ring) reinterpret_cast<C*>(a.fdst)[idx] = F;
    else a.fdst[idx] = cvt<double2>(F);
}

template <class C, int M, int R>
__global__ void __launch_bounds__(FsThr<C, M>::value, FsMinB<C, M>::value) k_fs_1d(FsArgs a, int mode) {
    using Ln = FsLine<C, M, R>;
    using Rl = typename cx_traits<C>::real;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* E = reinterpret_cast<C*>(sm_raw);
    C* y = E + Ln::EBUF;
    C* dv = y + M;
    const FsAxis& ax = a.ax[0];
    const int b = blockIdx.x, N = ax.N;
    const double vf = a.tfac[(size_t)b * a.ntf + a.tf];
    const double* V0 = a.V0 + (size_t)b * a.vstride;
    if (mode == FS_1D_FWD_ONLY) {
        for (int j = threadIdx.x; j < M; j += FsThr<C, M>::value) {
            const double2 u = a.usrc[(size_t)b * M + j];
            y[j] = cvt<C>(a.mulV ? cscale(u, vf * V0[j]) : u);
        }
        __syncthreads();
        Ln::forward(y, E, dv, ax);
        for (int m = threadIdx.x; m < N; m += FsThr<C, M>::value)
            store_fwd(a, (size_t)b * a.fdst_bstride + m, Ln::fwd_value(m, E, dv, ax));
        return;
    }
    double2* uh = a.uhat + (size_t)b * N;
    C* ring = reinterpret_cast<C*>(a.ring) + (size_t)b * a.ring_slots * N;
    const double2* P = ax.P + (size_t)b * a.n_int * N;
    const C* Pc = Tab<C>::P(ax) + (size_t)b * a.n_int * N;
    C cj[FS_MAX_HIST + 1];
#pragma unroll
    for (int j = 0; j <= FS_MAX_HIST; ++j) cj[j] = cvt<C>(make_double2(a.mu[j], 0.0));
    for (int m = threadIdx.x; m < N; m += FsThr<C, M>::value) {
        const C S = history_sep<C>(
            a, cj, [&](int j) { return ring[(size_t)a.hist_slot[j - 1] * N + m]; },
            [&](int i) { return __ldg(&Pc[(size_t)a.interval[i] * N + m]); });
        const double2 W = begin_W(a, uh[m], __ldg(&P[(size_t)a.interval[0] * N + m]), cvt<double2>(S));
        uh[m] = W;
        Ln::stage_inv(m, cvt<C>(W), E, dv, ax);
    }
    Ln::zero_pad(E, ax.NE);
    Ln::inverse(E, dv, y, ax);
    const double hm0 = a.h * a.mu[0];
    for (int j = threadIdx.x; j < M; j += FsThr<C, M>::value) {
        const double V = vf * V0[j];
        const C u = implicit_solve(y[j], (Rl)(hm0 * V));
        a.u[(size_t)b * M + j] = cvt<double2>(u);
        y[j] = cscale(u, (Rl)V);
    }
    __syncthreads();
    Ln::forward(y, E, dv, ax);
    for (int m = threadIdx.x; m < N; m += FsThr<C, M>::value) {
        const C F = Ln::fwd_value(m, E, dv, ax);
        uh[m] = uh[m] + times_minus_i(cvt<double2>(F), hm0);
        ring[(size_t)a.out_slot * N + m] = F;
    }
}

template <class C, int M, int R>
__global__ void __launch_bounds__(FsThr<C, M>::value, FsMinB<C, M>::value) k_fs_row(FsArgs a, int flags) {
    using Ln = FsLine<C, M, R>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* E = reinterpret_cast<C*>(sm_raw);
    C* f = E + Ln::EBUF;
    C* dv = f + M;
    const bool d3 = a.d == 3;
    const FsAxis& ax = a.ax[d3 ? 2 : 1];                // the line axis (the last one)
    const int k0 = blockIdx.x, b = blockIdx.y;           // k0: the row (k0 N1 + k1 in 3D)
    const int N0 = a.ax[0].N, N1 = ax.N;
    const int nrows = d3 ? N0 * a.ax[1].N : N0;
    const size_t NPm = (size_t)nrows * N1;
    double2* urow = a.uhat + (size_t)b * NPm + (size_t)k0 * N1;
    C* zrow = reinterpret_cast<C*>(a.Z) + ((size_t)b * nrows + k0) * M;
    const bool end = flags & FS_ROW_END, begin = flags & FS_ROW_BEGIN;
    if (end || (flags & FS_ROW_FWD_ONLY)) {
        for (int j = threadIdx.x; j < M; j += FsThr<C, M>::value) f[j] = zrow[j];
        __syncthreads();
        Ln::forward(f, E, dv, ax);
        if (flags & FS_ROW_FWD_ONLY) {
            const size_t base = (size_t)b * a.fdst_bstride + (size_t)k0 * N1;
            for (int m = threadIdx.x; m < N1; m += FsThr<C, M>::value) store_fwd(a, base + m, Ln::fwd_value(m, E, dv, ax));
            return;
        }
    }
    const double2* P0 = a.ax[0].P + (size_t)b * a.n_int * N0;
    const double2* P1 = ax.P + (size_t)b * a.n_int * N1;
    const C* P1c = Tab<C>::P(ax) + (size_t)b * a.n_int * N1;
    // phase of the row over interval iv: P0 (2D), P0 P1 of axes 0 and 1 (3D)
    auto row_phase = [&](int iv) -> double2 {
        if (!d3) return __ldg(&P0[(size_t)iv * N0 + k0]);
        const int NA = a.ax[1].N, i0 = k0 / NA, i1 = k0 - i0 * NA;
        const double2* PA = a.ax[1].P + (size_t)b * a.n_int * NA;
        return cmul(__ldg(&P0[(size_t)iv * N0 + i0]), __ldg(&PA[(size_t)iv * NA + i1]));
    };
    double2 a0 = zero2();
    C cj[FS_MAX_HIST + 1];
    if (begin) {
        a0 = row_phase(a.interval[0]);
        double2 A = make_double2(1.0, 0.0);
#pragma unroll
        for (int j = 1; j <= FS_MAX_HIST; ++j) {
            cj[j] = cvt<C>(cscale(A, a.mu[j]));
            if (j < FS_MAX_HIST && j < a.nhist) A = cmul(A, row_phase(a.interval[j]));
        }
    }
    const double hm0 = a.h * a.mu[0];
    C* ring = reinterpret_cast<C*>(a.ring) + (size_t)b * a.ring_slots * NPm + (size_t)k0 * N1;
    for (int m = threadIdx.x; m < N1; m += FsThr<C, M>::value) {
        double2 uh;
        C F = zeroc<C>();
        if (end) {
            F = Ln::fwd_value(m, E, dv, ax);
            uh = urow[m] + times_minus_i(cvt<double2>(F), hm0);
            ring[(size_t)a.out_slot * NPm + m] = F;
            if (!begin) urow[m] = uh;
        } else {
            uh = urow[m];
        }
        if (begin) {
            const C S = history_sep<C>(
                a, cj,
                [&](int j) {
                    const int slot = a.hist_slot[j - 1];
                    return (end && slot == a.out_slot) ? F : ring[(size_t)slot * NPm + m];
                },
                [&](int i) { return __ldg(&P1c[(size_t)a.interval[i] * N1 + m]); });
            const double2 p0 = cmul(a0, __ldg(&P1[(size_t)a.interval[0] * N1 + m]));
            const double2 W = begin_W(a, uh, p0, cvt<double2>(S));
            urow[m] = W;
            Ln::stage_inv(m, cvt<C>(W), E, dv, ax);
        }
    }
    if (!begin) return;
    Ln::zero_pad(E, ax.NE);
    Ln::inverse(E, dv, f, ax);
    for (int j = threadIdx.x; j < M; j += FsThr<C, M>::value) zrow[j] = f[j];
}

template <class C, int M, int R>
__global__ void __launch_bounds__(FsThr<C, M>::value, FsMinB<C, M>::value) k_fs_phys(FsArgs a, int from_usrc) {
    using Ln = FsLine<C, M, R>;
    using Rl = typename cx_traits<C>::real;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* E = reinterpret_cast<C*>(sm_raw);
    C* y = E + Ln::EBUF;
    C* dv = y + M;
    const FsAxis& ax = a.ax[0];
    const int j1 = blockIdx.x, b = blockIdx.y;          // j1: the column (j1 M2 + j2 in 3D)
    const bool d3 = a.d == 3;
    const int M1 = d3 ? a.ax[1].M * a.ax[2].M : a.ax[1].M, N0 = ax.N;
    C* zcol = reinterpret_cast<C*>(d3 ? a.Y : a.Z) + (size_t)b * N0 * M1 + j1;
    const size_t NX = (size_t)M * M1;
    const double vf = a.tfac[(size_t)b * a.ntf + a.tf];
    const double* V0 = a.V0 + (size_t)b * a.vstride;
    if (!from_usrc) {
        for (int m = threadIdx.x; m < N0; m += FsThr<C, M>::value) Ln::stage_inv(m, zcol[(size_t)m * M1], E, dv, ax);
        Ln::zero_pad(E, ax.NE);
        Ln::inverse(E, dv, y, ax);
        const double hm0 = a.h * a.mu[0];
        for (int j0 = threadIdx.x; j0 < M; j0 += FsThr<C, M>::value) {
            const size_t g = (size_t)j0 * M1 + j1;
            const double V = vf * V0[g];
            const C u = implicit_solve(y[j0], (Rl)(hm0 * V));
            a.u[(size_t)b * NX + g] = cvt<double2>(u);
            y[j0] = cscale(u, (Rl)V);
        }
    } else {
        for (int j0 = threadIdx.x; j0 < M; j0 += FsThr<C, M>::value) {
            const size_t g = (size_t)j0 * M1 + j1;
            const double2 u = a.usrc[(size_t)b * NX + g];
            y[j0] = cvt<C>(a.mulV ? cscale(u, vf * V0[g]) : u);
        }
    }
    __syncthreads();
    Ln::forward(y, E, dv, ax);
    for (int m = threadIdx.x; m < N0; m += FsThr<C, M>::value) zcol[(size_t)m * M1] = Ln::fwd_value(m, E, dv, ax);
}

// 3D, axis 1: line (k0, j2) between the N1 modes Z[b][k0][.][j2] and the M1
// grid values Y[b][k0][.][j2] (both with stride M2).
template <class C, int M, int R>
__global__ void __launch_bounds__(FsThr<C, M>::value, FsMinB<C, M>::value) k_fs_mid(FsArgs a, int dir) {
    using Ln = FsLine<C, M, R>;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* E = reinterpret_cast<C*>(sm_raw);
    C* f = E + Ln::EBUF;
    C* dv = f + M;
    const FsAxis& ax = a.ax[1];
    const int j2 = blockIdx.x, k0 = blockIdx.y, b = blockIdx.z;
    const int M2 = a.ax[2].M, N0 = a.ax[0].N, N1 = ax.N;
    C* zl = reinterpret_cast<C*>(a.Z) + ((size_t)b * N0 + k0) * N1 * M2 + j2;
    C* yl = reinterpret_cast<C*>(a.Y) + ((size_t)b * N0 + k0) * M * M2 + j2;
    if (dir == FS_MID_INV) {
        for (int m = threadIdx.x; m < N1; m += FsThr<C, M>::value) Ln::stage_inv(m, zl[(size_t)m * M2], E, dv, ax);
        Ln::zero_pad(E, ax.NE);
        Ln::inverse(E, dv, f, ax);
        for (int j = threadIdx.x; j < M; j += FsThr<C, M>::value) yl[(size_t)j * M2] = f[j];
    } else {
        for (int j = threadIdx.x; j < M; j += FsThr<C, M>::value) f[j] = yl[(size_t)j * M2];
        __syncthreads();
        Ln::forward(f, E, dv, ax);
        for (int m = threadIdx.x; m < N1; m += FsThr<C, M>::value) zl[(size_t)m * M2] = Ln::fwd_value(m, E, dv, ax);
    }
}

template <class C, int M, int R>
constexpr size_t smem_of() {
    return (size_t)(FsLine<C, M, R>::EBUF + M + FS_MAX_ND + FS_MAX_NT) * sizeof(C);
}

// Dynamic shared memory of the kernel and, for the FP32 kernels, the largest
// shared-memory carve-out (several CTAs per SM).
template <class C, class K>
cudaError_t prepare(K kernel, size_t sm) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess && MinBlocks<C>::value > 1)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

template <class C, int M, int R>
cudaError_t launch_mr(const FsArgs& a, int which, int flag, cudaStream_t s) {
    constexpr size_t sm = smem_of<C, M, R>();
    cudaError_t e;
    if (which == 0) {
        if ((e = prepare<C>(k_fs_1d<C, M, R>, sm)) != cudaSuccess) return e;
        k_fs_1d<C, M, R><<<a.B, FsThr<C, M>::value, sm, s>>>(a, flag);
    } else if (which == 1) {
        if ((e = prepare<C>(k_fs_row<C, M, R>, sm)) != cudaSuccess) return e;
        const unsigned rows = a.d == 3 ? (unsigned)(a.ax[0].N * a.ax[1].N) : (unsigned)a.ax[0].N;
        k_fs_row<C, M, R><<<dim3(rows, a.B), FsThr<C, M>::value, sm, s>>>(a, flag);
    } else if (which == 2) {
        if ((e = prepare<C>(k_fs_phys<C, M, R>, sm)) != cudaSuccess) return e;
        const unsigned cols = a.d == 3 ? (unsigned)(a.ax[1].M * a.ax[2].M) : (unsigned)a.ax[1].M;
        k_fs_phys<C, M, R><<<dim3(cols, a.B), FsThr<C, M>::value, sm, s>>>(a, flag);
    } else {
        if ((e = prepare<C>(k_fs_mid<C, M, R>, sm)) != cudaSuccess) return e;
        k_fs_mid<C, M, R><<<dim3(a.ax[2].M, a.ax[0].N, a.B), FsThr<C, M>::value, sm, s>>>(a, flag);
    }
    return cudaGetLastError();
}

// (M, R) pairs built: M = 32..512, R = 4, 8, 16, nu = M R <= 4096.
template <class C>
cudaError_t dispatch(const FsArgs& a, const FsAxis& ax, int which, int flag, cudaStream_t s) {
#define FS_FOR_R(M_)                                                                               \
    if (R == 4) return launch_mr<C, M_, 4>(a, which, flag, s);                                   \
    if (R == 8) return launch_mr<C, M_, 8>(a, which, flag, s);                                   \
    if (R == 16 && M_ * 16 <= 4096) return launch_mr<C, M_, (M_ * 16 <= 4096 ? 16 : 8)>(a, which, flag, s);
    const int M = ax.M, R = ax.R;
    switch (M) {
        case 32: { FS_FOR_R(32) break; }
        case 64: { FS_FOR_R(64) break; }
        case 128: { FS_FOR_R(128) break; }
        case 256: { FS_FOR_R(256) break; }
        case 512: { FS_FOR_R(512) break; }
        default: break;
    }
#undef FS_FOR_R
    return cudaErrorInvalidValue;
}

// which: 0 = 1D step, 1 = row pass (last axis), 2 = phys pass (axis 0), 3 = axis-1 pass (3D)
inline const FsAxis& axis_of(const FsArgs& a, int which) {
    return which == 1 ? a.ax[a.d - 1] : (which == 3 ? a.ax[1] : a.ax[0]);
}

}  // namespace fs
}  // namespace tdse
