// FP64 transforms of 1D instances of length N = 128 x 128 in two passes
// (four-step factorisation), for the start (u^ = DFT(u0), (V u0)^) and the
// read-out (u = IDFT(u^)) of 1D mixed-precision instances whose FP64
// transform does not fit one CTA's shared memory.  The steps themselves run
// in FP32 in the one-CTA kernel.
//
// With n = n1 N2 + n2 and k = k1 + N1 k2 (N1 = N2 = 128, w = e^{-+2 pi i / N}):
//   X[k1 + N1 k2] = sum_n2 w_N2^{n2 k2} [ w^{n2 k1} sum_n1 x[n1 N2 + n2] w_N1^{n1 k1} ].
// Pass A transforms the columns (fixed n2) and applies w^{n2 k1}; pass B
// transforms the rows (fixed k1) into X.  Both use the CTA-wide Stockham FFT
// on 8 interleaved lines per CTA.
#include "step_common.cuh"

namespace tdse {
namespace {

constexpr int F4_N1 = 128, F4_N2 = 128, F4_N = F4_N1 * F4_N2, F4_L = 8, F4_T = 256;

enum F4Src : int { F4_SRC_U0 = 0, F4_SRC_VU0 = 1, F4_SRC_STATE = 2 };
enum F4Dst : int { F4_DST_STATE = 0, F4_DST_RING = 1, F4_DST_OUT = 2 };

// Pass A: Y[b][k1 N2 + n2] = w^{n2 k1} sum_n1 x[n1 N2 + n2] w_N1^{n1 k1}
template <bool INV>
__global__ void __launch_bounds__(F4_T) k_f4_cols(const KArgs a, const double2* tw128, double2* Y, int src) {
    __shared__ double2 buf[F4_N1 * F4_L];
    const int cg = blockIdx.x, b = blockIdx.y;
    const size_t off = (size_t)b * F4_N;
    const double2* u0 = reinterpret_cast<const double2*>(a.uhat) + off;   // parked u0 (start)
    const float4* st = reinterpret_cast<const float4*>(a.uhat) + off;     // double-float state (read-out)
    const double vfac = a.tfac[(size_t)b * a.ntf + a.tf];
    for (int it = threadIdx.x; it < F4_N1 * F4_L; it += F4_T) {
        const int n1 = it / F4_L, c = it % F4_L;
        const int n = n1 * F4_N2 + cg * F4_L + c;
        double2 x;
        if (src == F4_SRC_STATE) {
            x = st_to_d(st[n]);
            if (a.ip) x = cmul(e_exact(a, b, a.e_step, kmode(n, F4_N), 0.0, 1), x);
        } else {
            x = u0[n];
            if (src == F4_SRC_VU0) x = cscale(x, vfac * a.V0[(size_t)b * a.vstride + n]);
        }
        buf[n1 * F4_L + c] = x;
    }
    __syncthreads();
    CtaFft<double2, F4_N1, F4_L, F4_L, F4_T, INV>::run(buf, tw128, nullptr);
    for (int it = threadIdx.x; it < F4_N1 * F4_L; it += F4_T) {
        const int k1 = it / F4_L, c = it % F4_L;
        const int n2 = cg * F4_L + c;
        double2 w = __ldg(&a.tw64_0[(n2 * k1) % F4_N]);
        if (INV) w.y = -w.y;
        Y[off + (size_t)k1 * F4_N2 + n2] = cmul(buf[k1 * F4_L + c], w);
    }
}

// Pass B: X[k1 + N1 k2] = sum_n2 Y[k1 N2 + n2] w_N2^{n2 k2}, written to the
// state (scaled 1/N), a ring slot (scaled 1/N) or the read-out array.
template <bool INV>
__global__ void __launch_bounds__(F4_T) k_f4_rows(const KArgs a, const double2* tw128, const double2* Y, int dst) {
    __shared__ double2 buf[F4_N2 * F4_L];
    const int rg = blockIdx.x, b = blockIdx.y;
    const size_t off = (size_t)b * F4_N;
    for (int it = threadIdx.x; it < F4_N2 * F4_L; it += F4_T) {
        const int c = it / F4_N2, n2 = it % F4_N2;
        buf[n2 * F4_L + c] = Y[off + (size_t)(rg * F4_L + c) * F4_N2 + n2];
    }
    __syncthreads();
    CtaFft<double2, F4_N2, F4_L, F4_L, F4_T, INV>::run(buf, tw128, nullptr);
    const double scale = 1.0 / F4_N;
    for (int it = threadIdx.x; it < F4_N2 * F4_L; it += F4_T) {
        const int k2 = it / F4_L, c = it % F4_L;
        const int k = rg * F4_L + c + F4_N1 * k2;
        const double2 X = buf[k2 * F4_L + c];
        if (dst == F4_DST_STATE)
            reinterpret_cast<float4*>(a.uhat)[off + k] = d_to_st<float4>(cscale(X, scale));
        else if (dst == F4_DST_RING)
            reinterpret_cast<float2*>(a.ring)[((size_t)b * a.ring_slots + a.out_slot) * F4_N + k] =
                cvt<float2>(cscale(X, scale));
        else
            a.aux2[off + k] = X;
    }
}

__global__ void k_tw128(double2* tw) {
    const int m = threadIdx.x;
    double s, c;
    sincospi(-2.0 * m / F4_N1, &s, &c);
    tw[m] = make_double2(c, s);
}

}  // namespace

int four_step_n() { return F4_N; }

cudaError_t launch_four_step_tables(double2* tw128, cudaStream_t s) {
    k_tw128<<<1, F4_N1, 0, s>>>(tw128);
    return cudaGetLastError();
}

// Start of a mixed 1D instance set of length 128^2 (MODE_INIT): ring[out_slot]
// = DFT(V(t_tf) u0) / N and state = DFT(u0) / N, u0 parked in the state slots.
cudaError_t launch_four_step_init(const KArgs& a, const double2* tw128, cudaStream_t s) {
    const dim3 grid(F4_N2 / F4_L, a.B);
    k_f4_cols<false><<<grid, F4_T, 0, s>>>(a, tw128, a.aux, F4_SRC_VU0);
    k_f4_cols<false><<<grid, F4_T, 0, s>>>(a, tw128, a.aux2, F4_SRC_U0);
    k_f4_rows<false><<<grid, F4_T, 0, s>>>(a, tw128, a.aux, F4_DST_RING);
    k_f4_rows<false><<<grid, F4_T, 0, s>>>(a, tw128, a.aux2, F4_DST_STATE);
    return cudaGetLastError();
}

// Read-out (MODE_READ): aux2 = IDFT(E_n v^) (or IDFT(u^) in the lab frame), FP64.
cudaError_t launch_four_step_read(const KArgs& a, const double2* tw128, cudaStream_t s) {
    const dim3 grid(F4_N2 / F4_L, a.B);
    k_f4_cols<true><<<grid, F4_T, 0, s>>>(a, tw128, a.aux, F4_SRC_STATE);
    k_f4_rows<true><<<grid, F4_T, 0, s>>>(a, tw128, a.aux, F4_DST_OUT);
    return cudaGetLastError();
}

}  // namespace tdse
