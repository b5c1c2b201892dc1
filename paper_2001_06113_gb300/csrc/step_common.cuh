// Per-mode and per-point arithmetic of one step of the periodic scheme,
// shared by the 1D fused kernel and the 2D pass kernels.
//
// Lab-frame (relative-phase) form, used by FP64 mode and by the mixed-mode
// Richardson start-up.  With one-step phases
//     p_i = exp(-i |k|^2 h + i k.(phi(t - i h) - phi(t - (i+1) h)))
// the lag-j phase of eq. uadamsk is p_0 ... p_{j-1}, so
//     S_{m-1} = mu_{m-1} R_{m-1},   S_j = mu_j R_j + p_j S_{j+1}      (Horner)
//     W       = p_0 (u^(t-h) - i h S_1)
//             = P(t,h) u^(t-h) - i h sum_{j>=1} mu_j P(t, j h) (Vu)^(t - j h)
//     u = IDFT(W) / (1 + i mu_0 h V(t)),   R_0 = DFT(V(t) u),
//     u^(t) = W - i mu_0 h R_0
// (the last line is the mode-space form of "u^ + i mu_0 h (Vu)^ = W", the
// diagonal implicit solve; trapezoidal rule = the case m = 2, mu = (1/2, 1/2)).
//
// Interaction-picture form, used by the mixed-mode Adams steps.  With
// E_n = exp(-i |k|^2 t_n + i k.phi(t_n)) (so P(t_n, j h) = E_n / E_{n-j}),
// v^ = u^ / E_n and r^ = R / E_n, eq. uadamsk divided by E_n reads
//     X_n = v^_{n-1} - i h sum_{j>=1} mu_j r^_{n-j}
//     u = IDFT(E_n X_n) / (1 + i mu_0 h V),  R_n = DFT(V u),  r^_n = R_n / E_n,
//     v^_n = X_n - i h mu_0 r^_n .
// The history is a plain weighted sum (no per-lag phase products), and E_n,
// whose argument |k|^2 t_n is large, is computed in FP64 and rounded once.
//
// Precision: FP64 mode keeps everything in double.  Mixed mode keeps the state
// (u^, v^, W, X) in double-float (two FP32, 48-bit significand) and does the
// history sum, transforms and pointwise work in FP32; the weights mu_j, h and
// h mu_0 are split hi + lo so that no coefficient is rounded to FP32.  The
// mixed step therefore issues no FP64 instructions.
#pragma once
#include <type_traits>

#include "cplx.cuh"
#include "ff.cuh"
#include "kargs.h"

namespace tdse {

template <class C> struct is_f64 { static constexpr bool value = false; };
template <> struct is_f64<double2> { static constexpr bool value = true; };

template <class RT> using state_t = std::conditional_t<is_f64<RT>::value, double2, float4>;

// ---- state conversions
__device__ __forceinline__ double2 st_to_d(double2 v) { return v; }
__device__ __forceinline__ double2 st_to_d(float4 v) { return ffc_to_d(v); }
template <class ST> __device__ __forceinline__ ST d_to_st(double2 v);
template <> __device__ __forceinline__ double2 d_to_st<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float4 d_to_st<float4>(double2 v) { return d_to_ffc(v); }
template <class C> __device__ __forceinline__ C st_to_c(double2 v) { return cvt<C>(v); }
template <class C> __device__ __forceinline__ C st_to_c(float4 v);
template <> __device__ __forceinline__ float2 st_to_c<float2>(float4 v) { return make_float2(v.x, v.y); }
template <> __device__ __forceinline__ double2 st_to_c<double2>(float4 v) { return ffc_to_d(v); }

__device__ __forceinline__ float4 ff_from_d(double2 v) { return d_to_ffc(v); }

__device__ __forceinline__ double kmode(int m, int n) { return (double)(m < n / 2 ? m : m - n); }

// ---- one-step (relative) phases, lab-frame form
struct Phase1D {
    const KArgs& a;
    int b, m;
    __device__ __forceinline__ size_t base(int i) const {
        return ((size_t)b * a.n_int + a.interval[i]) * (size_t)(a.nh + a.nl);
    }
    __device__ __forceinline__ double2 p64(int i) const {
        const double2* t = a.adv64 + base(i);
        const double2 kin = __ldg(&a.kin64[(size_t)a.kin * a.tn0 + m]);
        return cmul(kin, cmul(__ldg(&t[m >> a.lb]), __ldg(&t[a.nh + (m & (a.nl - 1))])));
    }
    __device__ __forceinline__ float4 pff(int i) const {
        const float4* t = a.advff + base(i);
        const float4 kin = __ldg(&a.kinff[(size_t)a.kin * a.tn0 + m]);
        return ffc_mul(kin, ffc_mul(__ldg(&t[m >> a.lb]), __ldg(&t[a.nh + (m & (a.nl - 1))])));
    }
};

// Column index m1 of a 3D column pass ([n0][n1 n2]) -> (i1, i2); 2D: (m1, -1).
__device__ __forceinline__ void split12(const KArgs& a, int m1, int& i1, int& i2) {
    if (a.tn2 == 0) {
        i1 = m1;
        i2 = -1;
    } else {
        i1 = m1 / a.tn2;
        i2 = m1 - i1 * a.tn2;
    }
}

// Separable phases of the 2D (and 3D) steps: the product of one factor per axis.
struct Phase2D {
    const KArgs& a;
    int b, m0, m1;
    __device__ __forceinline__ size_t base(int i) const {
        return ((size_t)b * a.n_int + a.interval[i]) * (size_t)(a.tn0 + a.tn1 + a.tn2);
    }
    __device__ __forceinline__ double2 p64(int i) const {
        if (a.flat1d) return Phase1D{a, b, m0 * a.n1 + m1}.p64(i);
        const double2* q = a.q64 + base(i);
        if (a.tn2 == 0) return cmul(__ldg(&q[m0]), __ldg(&q[a.tn0 + m1]));
        int i1, i2;
        split12(a, m1, i1, i2);
        return cmul(cmul(__ldg(&q[m0]), __ldg(&q[a.tn0 + i1])), __ldg(&q[a.tn0 + a.tn1 + i2]));
    }
    __device__ __forceinline__ float4 pff(int i) const {
        if (a.flat1d) return Phase1D{a, b, m0 * a.n1 + m1}.pff(i);
        const float4* q = a.qff + base(i);
        if (a.tn2 == 0) return ffc_mul(__ldg(&q[m0]), __ldg(&q[a.tn0 + m1]));
        int i1, i2;
        split12(a, m1, i1, i2);
        return ffc_mul(ffc_mul(__ldg(&q[m0]), __ldg(&q[a.tn0 + i1])), __ldg(&q[a.tn0 + a.tn1 + i2]));
    }
};

__device__ __forceinline__ float2 e_1d(const KArgs& a, int b, int n, int m) {
    const float2 kin = cmul(__ldg(&a.k1d_hi[(size_t)(n / E1D_NLO) * a.tn0 + m]),
                            __ldg(&a.k1d_lo[(size_t)(n % E1D_NLO) * a.tn0 + m]));
    const float2* t = a.a1d + ((size_t)b * (a.ntf / 8 + 1) + n) * (size_t)(a.nh + a.nl);
    return cmul(kin, cmul(__ldg(&t[m >> a.lb]), __ldg(&t[a.nh + (m & (a.nl - 1))])));
}

// ---- absolute phases E_n (interaction picture), FP32
__device__ __forceinline__ float2 e_2d(const KArgs& a, int b, int n, int m0, int m1) {
    if (a.flat1d) return e_1d(a, b, n, m0 * a.n1 + m1);
    const float2* e = a.e2d + ((size_t)b * (a.ntf / 8 + 1) + n) * (size_t)(a.tn0 + a.tn1 + a.tn2);
    if (a.tn2 == 0) return cmul(__ldg(&e[m0]), __ldg(&e[a.tn0 + m1]));
    int i1, i2;
    split12(a, m1, i1, i2);
    return cmul(cmul(__ldg(&e[m0]), __ldg(&e[a.tn0 + i1])), __ldg(&e[a.tn0 + a.tn1 + i2]));
}
// E_n in FP64 from the phi table (read-out only): angle -|k|^2 t_n + k.phi(t_n)
__device__ __forceinline__ double2 e_exact(const KArgs& a, int b, int n, double k0, double k1, int d) {
    const double t = (double)n * a.dt;
    const double* ph = a.phi + (size_t)b * d * a.ntf;
    double arg = -(k0 * k0 + k1 * k1) * t + k0 * ph[8 * n];
    if (d == 2) arg += k1 * ph[a.ntf + 8 * n];
    double s, c;
    sincos(arg, &s, &c);
    return make_double2(c, s);
}
// The same in 3D for the flattened column index m1 of mode (m0, i1, i2).
__device__ __forceinline__ double2 e_exact3(const KArgs& a, int b, int n, int m0, int m1) {
    int i1, i2;
    split12(a, m1, i1, i2);
    const double k0 = kmode(m0, a.tn0), k1 = kmode(i1, a.tn1), k2 = kmode(i2, a.tn2);
    const double t = (double)n * a.dt;
    const double* ph = a.phi + (size_t)b * 3 * a.ntf;
    const double arg = -(k0 * k0 + k1 * k1 + k2 * k2) * t + k0 * ph[8 * n] + k1 * ph[a.ntf + 8 * n] +
                       k2 * ph[2 * (size_t)a.ntf + 8 * n];
    double s, c;
    sincos(arg, &s, &c);
    return make_double2(c, s);
}

__device__ __forceinline__ float2 conjf2(float2 z) { return make_float2(z.x, -z.y); }

// ---- mixed-mode history sum S = sum_{j=1}^{nhist} mu_j r_j (FP32, weights hi + lo).
// Fully unrolled over the (at most 7) lags so that every ring load of a mode is
// in flight at once.
__device__ __forceinline__ float2 history_sum_f32(const KArgs& a, const float2* __restrict__ ringb, size_t NP,
                                                   size_t idx) {
    float2 r[MAX_HIST];
#pragma unroll
    for (int j = 1; j <= MAX_HIST; ++j)
        r[j - 1] = (j <= a.nhist) ? ringb[(size_t)a.hist_slot[j - 1] * NP + idx] : make_float2(0.f, 0.f);
    float2 S = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = MAX_HIST; j >= 1; --j) {
        S.x = fmaf(a.mu_hi[j], r[j - 1].x, S.x);
        S.y = fmaf(a.mu_hi[j], r[j - 1].y, S.y);
        S.x = fmaf(a.mu_lo[j], r[j - 1].x, S.x);
        S.y = fmaf(a.mu_lo[j], r[j - 1].y, S.y);
    }
    return S;
}

// z - i (c_hi + c_lo) s, z double-float complex, s FP32 complex
__device__ __forceinline__ float4 ff_minus_i_times(float4 z, float c_hi, float c_lo, float2 s) {
    // -i c s = c s.y - i c s.x
    const float pr = c_hi * s.y, pi = c_hi * s.x;
    ffr ir{pr, fmaf(c_lo, s.y, fmaf(c_hi, s.y, -pr))};
    ffr ii{-pi, -fmaf(c_lo, s.x, fmaf(c_hi, s.x, -pi))};
    return ff_pack(ff_add(ff_re(z), ir), ff_add(ff_im(z), ii));
}

// Interaction-picture history sum S = sum_j c_j r~_{n-j}, c_j = mu_j / z_{n-j}
// (complex weights, hi + lo), all ring loads in flight together.
__device__ __forceinline__ float2 history_sum_ip(const KArgs& a, const float2* __restrict__ ringb, size_t NP,
                                                 size_t idx) {
    float2 r[MAX_HIST];
#pragma unroll
    for (int j = 1; j <= MAX_HIST; ++j)
        r[j - 1] = (j <= a.nhist) ? ringb[(size_t)a.hist_slot[j - 1] * NP + idx] : make_float2(0.f, 0.f);
    float2 S = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = MAX_HIST; j >= 1; --j) {
        const float2 q = r[j - 1];
        const float ch = a.c_hi[j][0], cih = a.c_hi[j][1], cl = a.c_lo[j][0], cil = a.c_lo[j][1];
        S.x = fmaf(cl, q.x, fmaf(-cil, q.y, S.x));
        S.y = fmaf(cl, q.y, fmaf(cil, q.x, S.y));
        S.x = fmaf(ch, q.x, fmaf(-cih, q.y, S.x));
        S.y = fmaf(ch, q.y, fmaf(cih, q.x, S.y));
    }
    return S;
}
__device__ __forceinline__ float4 ip_X(const KArgs& a, float4 st, const float2* __restrict__ ringb, size_t NP,
                                       size_t idx) {
    return ff_minus_i_times(st, a.h_hi, a.h_lo, history_sum_ip(a, ringb, NP, idx));
}
// v^ = X - i d r~,  d = h mu_0 / z_n (complex hi + lo)
__device__ __forceinline__ float4 ip_update(const KArgs& a, float4 X, float2 q) {
    float px = fmaf(a.d_lo[0], q.x, -a.d_lo[1] * q.y);
    float py = fmaf(a.d_lo[0], q.y, a.d_lo[1] * q.x);
    px = fmaf(a.d_hi[0], q.x, fmaf(-a.d_hi[1], q.y, px));
    py = fmaf(a.d_hi[0], q.y, fmaf(a.d_hi[1], q.x, py));
    return ffc_add_f(X, py, -px);
}

// X = st - i h S (mixed, double-float, real weights: lab-frame start-up)
__device__ __forceinline__ float4 mixed_X(const KArgs& a, float4 st, const float2* __restrict__ ringb, size_t NP,
                                          size_t idx) {
    return ff_minus_i_times(st, a.h_hi, a.h_lo, history_sum_f32(a, ringb, NP, idx));
}

// FP64 lab-frame W = p_0 (u^ - i h S_1) with the Horner history sum (ring
// loads issued together, lags beyond nhist contribute zero).
template <class Ph>
__device__ __forceinline__ double2 horner_W64(const KArgs& a, double2 uh, const double2* __restrict__ ringb,
                                              size_t NP, size_t idx, const Ph& ph) {
    double2 r[MAX_HIST];
#pragma unroll
    for (int j = 1; j <= MAX_HIST; ++j)
        r[j - 1] = (j <= a.nhist) ? ringb[(size_t)a.hist_slot[j - 1] * NP + idx] : make_double2(0.0, 0.0);
    double2 S = make_double2(0.0, 0.0);
#pragma unroll
    for (int j = MAX_HIST; j >= 1; --j) {
        if (j <= a.nhist) {
            if (j < a.nhist) S = cmul(ph.p64(j), S);
            S.x = fma(a.mu[j], r[j - 1].x, S.x);
            S.y = fma(a.mu[j], r[j - 1].y, S.y);
        }
    }
    double2 X = uh;
    X.x = fma(a.h, S.y, X.x);
    X.y = fma(-a.h, S.x, X.y);
    return cmul(ph.p64(0), X);
}

// u = y / (1 + i beta), beta = h mu_0 V, returns V u with V = Vhi + Vlo.
// 1/(1 + i beta) = (1 - c) - i beta (1 - c), c = beta^2 / (1 + beta^2), is
// applied as y - c y - i beta (1 - c) y so that no rounded factor close to 1 is
// reused identically every step (beta = O(h |V|) is small).
template <class C>
__device__ __forceinline__ C implicit_solve_times_V(C y, typename cx_traits<C>::real Vhi,
                                                    typename cx_traits<C>::real Vlo,
                                                    typename cx_traits<C>::real hmu0) {
    using R = typename cx_traits<C>::real;
    const R beta = hmu0 * Vhi;
    const R b2 = beta * beta;
    const R c = b2 / ((R)1 + b2);
    const R bc = beta - beta * c;
    C u;
    u.x = fma(bc, y.y, fma(-c, y.x, y.x));
    u.y = fma(-bc, y.x, fma(-c, y.y, y.y));
    C r;
    r.x = fma(u.x, Vhi, u.x * Vlo);
    r.y = fma(u.y, Vhi, u.y * Vlo);
    return r;
}

// u^(t) = W - i h mu_0 R
__device__ __forceinline__ double2 update64(double2 W, double2 R, double hmu0) {
    return make_double2(fma(hmu0, R.y, W.x), fma(-hmu0, R.x, W.y));
}
__device__ __forceinline__ float4 update_ff(const KArgs& a, float4 W, float2 R) {
    return ff_minus_i_times(W, a.hmu0_hi, a.hmu0_lo, R);
}

}  // namespace tdse
