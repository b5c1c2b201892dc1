// Complex arithmetic on double2/float2 and a shared-memory Stockham FFT.
//
// The FFT computes, for each of LANES interleaved sequences of length N held in
// shared memory at buf[pos * LS + lane],
//     forward:  X_k = sum_j x_j e^{-2 pi i j k / N}
//     inverse:  x_j = sum_k X_k e^{+2 pi i j k / N}     (no 1/N)
// in place, as a Stockham auto-sort sequence of radix-8 passes preceded by
// one radix-2 or radix-4 pass when log2(N) is not a multiple of 3.  In pass s
// with Ns = product of the earlier radices, butterfly j (0 <= j < N/R) reads
// x[j + r N/R], twiddles by e^{-+2 pi i (j mod Ns) r / (Ns R)}, takes an R-point
// DFT in registers and writes positions (j - j mod Ns) R + j mod Ns + r Ns.
// Consecutive threads take consecutive lanes, so interleaved columns give
// conflict-free shared-memory access.  Twiddles come from a global table
// tw[m] = e^{-2 pi i m / N} (read through the read-only cache).
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

// multiply by e^{-+ i pi/4} = (1 -+ i)/sqrt(2)
template <bool INV, class C> __device__ __forceinline__ C rot45(C a) {
    using R = typename cx_traits<C>::real;
    const R s = (R)0.70710678118654752440;
    C r;
    if (INV) { r.x = (a.x - a.y) * s; r.y = (a.x + a.y) * s; }
    else     { r.x = (a.x + a.y) * s; r.y = (a.y - a.x) * s; }
    return r;
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

template <class C, int R, int N, int LANES, int LS, int T, bool INV>
__device__ __forceinline__ void stockham_pass(C* buf, const C* __restrict__ tw, int Ns) {
    constexpr int NB = N / R;
    constexpr int ITEMS = NB * LANES;
    constexpr int PER = (ITEMS + T - 1) / T;
    C v[PER][R];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int item = threadIdx.x + p * T;
        if ((ITEMS % T == 0) || item < ITEMS) {
            const int lane = item % LANES, j = item / LANES;
#pragma unroll
            for (int r = 0; r < R; ++r) v[p][r] = buf[(j + r * NB) * LS + lane];
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int item = threadIdx.x + p * T;
        if ((ITEMS % T == 0) || item < ITEMS) {
            const int lane = item % LANES, j = item / LANES;
            const int k = j & (Ns - 1);
            if (Ns > 1) {
                const int stride = N / (Ns * R);
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    C w = __ldg(&tw[k * r * stride]);
                    if (INV) w.y = -w.y;
                    v[p][r] = cmul(v[p][r], w);
                }
            }
            dft_r<R, INV>(v[p]);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[(base + r * Ns) * LS + lane] = v[p][r];
        }
    }
    __syncthreads();
}

// Full in-place FFT of LANES interleaved sequences; the caller must have
// synchronised after writing buf.  Ends with a barrier.
template <class C, int N, int LANES, int LS, int T, bool INV>
__device__ __forceinline__ void fft_smem(C* buf, const C* __restrict__ tw) {
    constexpr int P = ilog2(N);
    constexpr int R0 = (P % 3 == 0) ? 8 : (1 << (P % 3));
    constexpr int NREST = (P - ilog2(R0)) / 3;
    stockham_pass<C, R0, N, LANES, LS, T, INV>(buf, tw, 1);
    int Ns = R0;
#pragma unroll 1
    for (int s = 0; s < NREST; ++s) {
        stockham_pass<C, 8, N, LANES, LS, T, INV>(buf, tw, Ns);
        Ns *= 8;
    }
}

}  // namespace tdse
