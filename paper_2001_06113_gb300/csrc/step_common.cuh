// Per-mode and per-point arithmetic of one step of the periodic scheme,
// shared by the 1D fused kernel and the 2D pass kernels.
//
// Adams step (eq. uadamsk), written with one-step phases
//     p_i = exp(-i |k|^2 h + i k.(phi(t - i h) - phi(t - (i+1) h)))
// so that the lag-j phase of eq. uadamsk is p_0 p_1 ... p_{j-1}:
//     S_{m-1} = mu_{m-1} R_{m-1},   S_j = mu_j R_j + p_j S_{j+1}   (Horner)
//     W       = p_0 (u^(t-h) - i h S_1)
//             = P(t,h) u^(t-h) - i h sum_{j>=1} mu_j P(t, j h) (Vu)^(t - j h)
// with R_j = (Vu)^(t - j h) from the history ring.  Then
//     u = IDFT(W) / (1 + i mu_0 h V(t)),   R_0 = DFT(V(t) u),
//     u^(t) = W - i mu_0 h R_0,
// the last line being the mode-space form of "u^ + i mu_0 h (Vu)^ = W"
// (the diagonal implicit solve of Sec. 2.1, remark after eq. utrapkdisc).
// The trapezoidal rule (eq. utrapkdisc) is the case m = 2, mu = (1/2, 1/2).
//
// Precision: u^, W, p_0 and the update are FP64 in every mode.  The history
// sum S and the transforms run in the kernel's compute type C (FP64, or FP32
// in mixed mode, where only the O(h |V|) correction passes through FP32).
#pragma once
#include "cplx.cuh"
#include "kargs.h"

namespace tdse {

template <class C> struct is_f64 { static constexpr bool value = false; };
template <> struct is_f64<double2> { static constexpr bool value = true; };

// One-step phase of lag i at 1D mode index m of instance b.
struct Phase1D {
    const KArgs& a;
    int b, m;
    __device__ __forceinline__ const double2* adv64(int i) const {
        return a.adv64 + ((size_t)b * a.n_int + a.interval[i]) * (size_t)(a.nh + a.nl);
    }
    __device__ __forceinline__ const float2* adv32(int i) const {
        return a.adv32 + ((size_t)b * a.n_int + a.interval[i]) * (size_t)(a.nh + a.nl);
    }
    __device__ __forceinline__ double2 p64(int i) const {
        const double2* t = adv64(i);
        const double2 kin = __ldg(&a.kin64[(size_t)a.kin * a.n0 + m]);
        return cmul(kin, cmul(__ldg(&t[m >> a.lb]), __ldg(&t[a.nh + (m & (a.nl - 1))])));
    }
    template <class C> __device__ __forceinline__ C p(int i) const {
        if constexpr (is_f64<C>::value) {
            return p64(i);
        } else {
            const float2* t = adv32(i);
            const float2 kin = __ldg(&a.kin32[(size_t)a.kin * a.n0 + m]);
            return cmul(kin, cmul(__ldg(&t[m >> a.lb]), __ldg(&t[a.nh + (m & (a.nl - 1))])));
        }
    }
};

// One-step phase of lag i at 2D mode (m0, m1): separable product of per-axis tables.
struct Phase2D {
    const KArgs& a;
    int b, m0, m1;
    __device__ __forceinline__ size_t base(int i) const {
        return ((size_t)b * a.n_int + a.interval[i]) * (size_t)(a.n0 + a.n1);
    }
    __device__ __forceinline__ double2 p64(int i) const {
        const double2* q = a.q64 + base(i);
        return cmul(__ldg(&q[m0]), __ldg(&q[a.n0 + m1]));
    }
    template <class C> __device__ __forceinline__ C p(int i) const {
        if constexpr (is_f64<C>::value) {
            return p64(i);
        } else {
            const float2* q = a.q32 + base(i);
            return cmul(__ldg(&q[m0]), __ldg(&q[a.n0 + m1]));
        }
    }
};

// W = p_0 (u^ - i h S_1) for one mode; ringb points at instance b's ring.
template <class C, class RT, class Ph>
__device__ __forceinline__ double2 recurrence_W(const KArgs& a, double2 uh, const RT* __restrict__ ringb,
                                                size_t NP, size_t idx, const Ph& ph) {
    using R = typename cx_traits<C>::real;
    C S = czero<C>();
#pragma unroll 1
    for (int j = a.nhist; j >= 1; --j) {
        if (j < a.nhist) S = cmul(ph.template p<C>(j), S);
        const C r = cvt<C>(ringb[(size_t)a.hist_slot[j - 1] * NP + idx]);
        const R mu = (R)a.mu[j];
        S.x += mu * r.x;
        S.y += mu * r.y;
    }
    double2 X = uh;
    X.x += a.h * (double)S.y;
    X.y -= a.h * (double)S.x;
    return cmul(ph.p64(0), X);
}

// u = y / (1 + i beta), returns V u   (beta = h mu_0 V; beta = 0 for refresh)
template <class C>
__device__ __forceinline__ C implicit_solve_times_V(C y, typename cx_traits<C>::real V,
                                                    typename cx_traits<C>::real hmu0) {
    using R = typename cx_traits<C>::real;
    const R beta = hmu0 * V;
    const R inv = (R)1 / ((R)1 + beta * beta);
    C u;
    u.x = (y.x + beta * y.y) * inv;
    u.y = (y.y - beta * y.x) * inv;
    u.x *= V;
    u.y *= V;
    return u;
}

// u^(t) = W - i h mu_0 R
__device__ __forceinline__ double2 mode_update(double2 W, double2 R, double hmu0) {
    return make_double2(fma(hmu0, R.y, W.x), fma(-hmu0, R.x, W.y));
}

}  // namespace tdse
