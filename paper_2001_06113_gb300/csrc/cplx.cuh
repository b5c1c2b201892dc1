// Complex arithmetic on double2/float2 and a shared-memory Stockham FFT.
//
// The FFT computes, for each of L interleaved sequences of length N,
//     forward:  X_k = sum_j x_j e^{-2 pi i j k / N}
//     inverse:  x_j = sum_k X_k e^{+2 pi i j k / N}     (no 1/N)
// as a Stockham auto-sort sequence of passes.  In pass s with Ns = product of
// the earlier radices, butterfly j (0 <= j < N/R) reads x[j + r N/R], twiddles
// by e^{-+2 pi i (j mod Ns) r / (Ns R)}, takes an R-point DFT in registers and
// writes positions (j - j mod Ns) R + j mod Ns + r Ns.  The passes are radix 8
// plus one radix-2 or radix-4 pass when log2 N is not a multiple of 3 (second
// of three or more passes; with two passes first for forward transforms, last
// for inverse ones).  Then the last pass of a
// transform writes exactly the positions j + r N/R that the first pass of the
// next transform reads, so a transform's inputs and outputs stay in the
// registers of the thread that owns them: the first pass starts from
// registers, the last pass ends in registers, and the epilogue/prologue work of
// the step (history sum, implicit solve, mode update) runs there.  Shared
// memory holds element (pos, line) at buf[pos * PS + line], consecutive threads
// taking consecutive lines (interleaved columns).  Twiddles come from a global table
// tw[m] = e^{-2 pi i m / N} (read through the read-only cache); in FP32 a
// second table twlo = e^{-2 pi i m/N} - tw holds the rounding residual, used
// (v tw + v twlo) when TDSE_TWIDDLE_LO is set.
#pragma once
#include <cuda_runtime.h>

namespace tdse {

template <class C> struct cx_traits;
template <> struct cx_traits<double2> { using real = double; };
template <> struct cx_traits<float2> { using real = float; };

__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

template <class D> __device__ __forceinline__ D cvt(double2 a);
template <> __device__ __forceinline__ double2 cvt<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 cvt<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }
template <class D> __device__ __forceinline__ D cvt(float2 a);
template <> __device__ __forceinline__ double2 cvt<double2>(float2 a) { return make_double2(a.x, a.y); }
template <> __device__ __forceinline__ float2 cvt<float2>(float2 a) { return a; }

template <class C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

// multiply by -i (forward) or +i (inverse)
template <bool INV, class C> __device__ __forceinline__ C rot90(C a) {
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

// multiply by e^{-+ i pi/4} = (1 -+ i)/sqrt(2).  In FP32 the constant is
// applied as hi + lo so that the butterfly has no fixed rounding of 1/sqrt(2)
// (a rounding repeated identically at every step would bias the transform).
template <bool INV> __device__ __forceinline__ double2 rot45(double2 a) {
    const double s = 0.70710678118654752440;
    double2 r;
    if (INV) { r.x = (a.x - a.y) * s; r.y = (a.x + a.y) * s; }
    else     { r.x = (a.x + a.y) * s; r.y = (a.y - a.x) * s; }
    return r;
}
template <bool INV> __device__ __forceinline__ float2 rot45(float2 a) {
    const float sh = 0.707106769084930419921875f;          // float(1/sqrt 2)
    const float sl = 1.2101617485882343317e-08f;           // 1/sqrt 2 - sh
    const float u = INV ? a.x - a.y : a.x + a.y;
    const float v = INV ? a.x + a.y : a.y - a.x;
    return make_float2(fmaf(u, sh, u * sl), fmaf(v, sh, v * sl));
}

template <bool INV, class C> __device__ __forceinline__ void dft2(C* v) {
    C t = v[0] - v[1]; v[0] = v[0] + v[1]; v[1] = t;
}

template <bool INV, class C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    C t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = rot90<INV>(a1 - a3);
    a0 = t0 + t2; a2 = t0 - t2; a1 = t1 + t3; a3 = t1 - t3;
}

template <bool INV, class C> __device__ __forceinline__ void dft8(C* v) {
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = rot45<INV>(o1);
    o2 = rot90<INV>(o2);
    o3 = rot90<INV>(rot45<INV>(o3));
    v[0] = e0 + o0; v[4] = e0 - o0;
    v[1] = e1 + o1; v[5] = e1 - o1;
    v[2] = e2 + o2; v[6] = e2 - o2;
    v[3] = e3 + o3; v[7] = e3 - o3;
}

template <int R, bool INV, class C> __device__ __forceinline__ void dft_r(C* v) {
    if constexpr (R == 2) dft2<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else dft8<INV>(v);
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }


template <int N, bool INV> struct FftPlan {
    static constexpr int P = ilog2(N);
    static constexpr int RS = (P % 3 == 0) ? 8 : (1 << (P % 3));
    static constexpr int NPASS = (P % 3 == 0) ? P / 3 : P / 3 + 1;
    // Boundary passes are radix 8 whenever possible (small radix in the second
    // pass), so that a thread owns 8 values per item at both ends; with only two
    // passes the small radix goes first (forward) / last (inverse).
    static constexpr int radix(int s) {
        return RS == 8 ? 8 : (NPASS >= 3 ? (s == 1 ? RS : 8) : ((INV ? (s == NPASS - 1) : (s == 0)) ? RS : 8));
    }
    static constexpr int ns(int s) { return s == 0 ? 1 : ns(s - 1) * radix(s - 1); }
};

// v * w (w from tw, conjugated for the inverse); FP32 adds the residual table.
template <bool INV> __device__ __forceinline__ double2 twiddle(double2 v, const double2* __restrict__ tw,
                                                               const double2*, int idx) {
    double2 w = __ldg(&tw[idx]);
    if (INV) w.y = -w.y;
    return cmul(v, w);
}
// TDSE_TWIDDLE_LO = 1 applies the FP32 twiddle as hi + lo.  Off by default:
// on the 512^2 mixed workload it lowers the 2000-step error from 5.1e-7 to
// 4.4e-7 at a 7% cost in step time.
#ifndef TDSE_TWIDDLE_LO
#define TDSE_TWIDDLE_LO 0
#endif
template <bool INV> __device__ __forceinline__ float2 twiddle(float2 v, const float2* __restrict__ tw,
                                                              const float2* __restrict__ twl, int idx) {
    float2 w = __ldg(&tw[idx]);
    if (!TDSE_TWIDDLE_LO) {
        if (INV) w.y = -w.y;
        return cmul(v, w);
    }
    float2 wl = __ldg(&twl[idx]);
    if (INV) { w.y = -w.y; wl.y = -wl.y; }
    float2 t = cmul(v, w);
    t.x = fmaf(v.x, wl.x, fmaf(-v.y, wl.y, t.x));
    t.y = fmaf(v.x, wl.y, fmaf(v.y, wl.x, t.y));
    return t;
}

// Barrier policies for a group of threads that runs one transform: the whole
// CTA, one warp, or a named barrier over n threads (a multiple of 32) when
// several groups share a CTA.
struct CtaSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct GroupSync {
    unsigned id, n;
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
};

// L interleaved length-N transforms by T threads (thread index tid in 0..T-1
// of the group, barrier `sync`); element (pos, line) at buf[pos * PS + line].
// Item it of a pass with NB butterflies is butterfly j = it / L of line it % L.
template <class C, int N, int L, int PS, int T, bool INV>
struct Fft {
    using Plan = FftPlan<N, INV>;
    static constexpr int NPASS = Plan::NPASS;
    static constexpr int RF = Plan::radix(0);
    static constexpr int RL = Plan::radix(NPASS - 1);
    static constexpr int NBF = N / RF;           // first pass: item (j, line) owns positions j + r NBF
    static constexpr int NBL = N / RL;           // last pass:  item (j, line) owns positions j + r NBL
    static constexpr int PF = (NBF * L + T - 1) / T;
    static constexpr int PL = (NBL * L + T - 1) / T;

    __device__ static __forceinline__ bool item(int p, int NB, int& j, int& line, int tid) {
        const int it = tid + p * T;
        line = it % L;
        j = it / L;
        return ((NB * L) % T == 0) || it < NB * L;
    }

    template <int S, class Sync>
    __device__ static __forceinline__ void mid_pass(C* buf, const C* __restrict__ tw, const C* __restrict__ twl,
                                                    int tid, const Sync& sync) {
        constexpr int R = Plan::radix(S);
        constexpr int Ns = Plan::ns(S);
        constexpr int NB = N / R;
        constexpr int PER = (NB * L + T - 1) / T;
        C v[PER][R];
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            int j, line;
            if (item(p, NB, j, line, tid)) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[p][r] = buf[(j + r * NB) * PS + line];
            }
        }
        sync();
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            int j, line;
            if (item(p, NB, j, line, tid)) {
                const int k = j & (Ns - 1);
                constexpr int stride = N / (Ns * R);
#pragma unroll
                for (int r = 1; r < R; ++r) v[p][r] = twiddle<INV>(v[p][r], tw, twl, k * r * stride);
                dft_r<R, INV>(v[p]);
                const int base = (j - k) * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) buf[(base + r * Ns) * PS + line] = v[p][r];
            }
        }
        sync();
    }

    template <int S, class Sync>
    __device__ static __forceinline__ void mids(C* buf, const C* __restrict__ tw, const C* __restrict__ twl, int tid,
                                                const Sync& sync) {
        if constexpr (S <= NPASS - 2) {
            mid_pass<S>(buf, tw, twl, tid, sync);
            mids<S + 1>(buf, tw, twl, tid, sync);
        }
    }

    // in[p][r]: value at position j + r NBF of the item (p); out[p][r]: result at
    // position j + r NBL.  buf must not be in use by any thread of the group on
    // entry; the call ends with a barrier (buf free again).
    template <class Sync>
    __device__ static __forceinline__ void run(C (&in)[PF][RF], C (&out)[PL][RL], C* buf,
                                               const C* __restrict__ tw, const C* __restrict__ twl, int tid,
                                               const Sync& sync) {
        if constexpr (NPASS == 1) {
#pragma unroll
            for (int p = 0; p < PF; ++p) {
                dft_r<RF, INV>(in[p]);
#pragma unroll
                for (int r = 0; r < RF; ++r) out[p][r] = in[p][r];
            }
        } else {
#pragma unroll
            for (int p = 0; p < PF; ++p) {
                int j, line;
                if (item(p, NBF, j, line, tid)) {
                    dft_r<RF, INV>(in[p]);
#pragma unroll
                    for (int r = 0; r < RF; ++r) buf[(j * RF + r) * PS + line] = in[p][r];
                }
            }
            sync();
            mids<1>(buf, tw, twl, tid, sync);
#pragma unroll
            for (int p = 0; p < PL; ++p) {
                int j, line;
                if (item(p, NBL, j, line, tid)) {
#pragma unroll
                    for (int r = 0; r < RL; ++r) out[p][r] = buf[(j + r * NBL) * PS + line];
#pragma unroll
                    for (int r = 1; r < RL; ++r) out[p][r] = twiddle<INV>(out[p][r], tw, twl, j * r);
                    dft_r<RL, INV>(out[p]);
                }
            }
            sync();
        }
    }

    // The same transform split for callers that produce the inputs / consume
    // the outputs one item at a time in a non-unrolled loop (NPASS > 1):
    //   first_item(p, v)  for every p, then  middle(...),  then either
    //   last_item(p, v)   for every p followed by  finish(sync)   (buf free again).
    __device__ static __forceinline__ void first_item(int p, C (&v)[RF], C* buf, int tid) {
        int j, line;
        if (item(p, NBF, j, line, tid)) {
            dft_r<RF, INV>(v);
#pragma unroll
            for (int r = 0; r < RF; ++r) buf[(j * RF + r) * PS + line] = v[r];
        }
    }
    template <class Sync>
    __device__ static __forceinline__ void middle(C* buf, const C* __restrict__ tw, const C* __restrict__ twl,
                                                  int tid, const Sync& sync) {
        sync();
        mids<1>(buf, tw, twl, tid, sync);
    }
    __device__ static __forceinline__ bool last_item(int p, C (&v)[RL], const C* buf, const C* __restrict__ tw,
                                                     const C* __restrict__ twl, int tid, int& j) {
        int line;
        if (!item(p, NBL, j, line, tid)) return false;
#pragma unroll
        for (int r = 0; r < RL; ++r) v[r] = buf[(j + r * NBL) * PS + line];
#pragma unroll
        for (int r = 1; r < RL; ++r) v[r] = twiddle<INV>(v[r], tw, twl, j * r);
        dft_r<RL, INV>(v);
        return true;
    }
    template <class Sync>
    __device__ static __forceinline__ void finish(const Sync& sync) { sync(); }
};

// ---------------------------------------------------------------------------
// L interleaved length-N transforms done in place by a whole CTA of T threads:
// element (pos, line) at buf[pos * LS + line], consecutive threads taking
// consecutive lines.  Each pass loads all butterflies of the thread into
// registers, synchronises, then writes (in place).  The caller must have
// synchronised after filling buf; the call ends with a barrier.
template <class C, int N, int L, int LS, int T, bool INV>
struct CtaFft {
    using Plan = FftPlan<N, INV>;
    template <int S>
    __device__ static __forceinline__ void pass(C* buf, const C* __restrict__ tw, const C* __restrict__ twl) {
        if constexpr (S < Plan::NPASS) {
            constexpr int R = Plan::radix(S);
            constexpr int Ns = Plan::ns(S);
            constexpr int NB = N / R;
            constexpr int ITEMS = NB * L;
            constexpr int PER = (ITEMS + T - 1) / T;
            C v[PER][R];
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int it = threadIdx.x + p * T;
                if (ITEMS % T == 0 || it < ITEMS) {
                    const int line = it % L, j = it / L;
#pragma unroll
                    for (int r = 0; r < R; ++r) v[p][r] = buf[(j + r * NB) * LS + line];
                }
            }
            __syncthreads();
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int it = threadIdx.x + p * T;
                if (ITEMS % T == 0 || it < ITEMS) {
                    const int line = it % L, j = it / L;
                    const int k = j & (Ns - 1);
                    constexpr int stride = N / (Ns * R);
                    if (Ns > 1) {
#pragma unroll
                        for (int r = 1; r < R; ++r) v[p][r] = twiddle<INV>(v[p][r], tw, twl, k * r * stride);
                    }
                    dft_r<R, INV>(v[p]);
                    const int base = (j - k) * R + k;
#pragma unroll
                    for (int r = 0; r < R; ++r) buf[(base + r * Ns) * LS + line] = v[p][r];
                }
            }
            __syncthreads();
            pass<S + 1>(buf, tw, twl);
        }
    }
    __device__ static __forceinline__ void run(C* buf, const C* __restrict__ tw, const C* __restrict__ twl) {
        pass<0>(buf, tw, twl);
    }
};

}  // namespace tdse
