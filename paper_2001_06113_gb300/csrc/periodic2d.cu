// 2D periodic step as shared-memory pass kernels over [B][n0][n1]
// (row-major, axis 1 contiguous):
//
//   col_begin (axis 0, 8 columns per CTA):
//       state -> W (lab frame) or X (interaction picture), stored back in the
//       state slot; inverse DFT along axis 0 of W or E_n X    -> T1 [i0][k1]
//   row_mid   (axis 1, 8 rows per CTA, one warp per row):
//       inverse DFT along axis 1 -> y; u = y/(1 + i h mu_0 V); V u;
//       forward DFT along axis 1 (1/n1)                        -> T2 [i0][k1]
//   col_end   (axis 0):
//       forward DFT along axis 0 (1/n0) -> R = (Vu)^; ring[out] <- R (lab
//       frame) or z_n R / E_n (interaction picture); state update
//   col_fused = col_end of step n followed by col_begin of step n+1 on the same
//       column block: consecutive Adams steps cost two launches each
//       (row_mid, col_fused), and the mode arrays cross HBM once per step.
//       For mixed interaction-picture steps (the hot path) k_col_fused_ip does
//       the same with the state and history reads staged by cp.async.
//
// Each CTA holds 8 whole lines (columns or rows) in shared memory, interleaved
// so that consecutive threads touch consecutive lines, and transforms them
// together (CtaFft).  The element phases read and write 8 consecutive columns
// per row (one 64/128-byte segment); the per-mode history work is done one
// mode at a time per thread with all of that mode's loads in flight.
//
// MODE_REFRESH runs the passes with no phase/history and beta = 0;
// MODE_INIT runs row_mid (u0 -> T1 = F1 u0, T2 = F1 V u0) and col_end
// (T1 -> state, T2 -> ring[out]); MODE_READ runs col_begin (state -> T1, after
// multiplying by E_n in FP64 if the state is in the interaction picture) and
// row_mid (T1 -> u into aux2).
#include <type_traits>

#include "step_common.cuh"

namespace tdse {

constexpr int LANES2D = 8;     // columns per column-pass CTA = rows per row-pass CTA
constexpr int T2D = 256;
#ifndef TDSE_MINB2D
#define TDSE_MINB2D 4          // resident CTAs per SM the register budget is sized for
#endif
// FP32 row pass (less shared memory per CTA): 5 or 6 CTAs per SM (48 / 40
// registers, 330 / 940 bytes spilled) measured slower than 4 (0.526 / 0.592
// against 0.519 ms per 64 x 512^2 step).
#ifndef TDSE_MINB2D_ROW
#define TDSE_MINB2D_ROW TDSE_MINB2D
#endif
// FP64 kernels: two CTAs per SM (up to 128 registers) instead of four (64
// registers and 0.6-1.9 KB of spills per thread): 0.494 -> 0.488 ms per
// 4 x 512^2 FP64 step (the FP64 pipe bounds it either way).
#ifndef TDSE_MINB2D64
#define TDSE_MINB2D64 2
#endif
template <class C>
constexpr int min_blocks_2d() { return std::is_same<C, float2>::value ? TDSE_MINB2D : TDSE_MINB2D64; }
template <class C>
constexpr int row_min_blocks() { return std::is_same<C, float2>::value ? TDSE_MINB2D_ROW : TDSE_MINB2D64; }

// 16-byte asynchronous global -> shared copies (no registers held while in flight)
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copy TOTAL elements with all loads of a thread (up to 16 of 8 bytes or 8 of
// 16 bytes) in flight before their stores: the loads are L2 hits of the other
// pass's output, and issuing them one element at a time left the passes
// waiting on L2 latency (0.181 -> 0.153 ms per 512^2 x16 mixed step).
template <class C, int TOTAL, class Load, class Store>
__device__ __forceinline__ void batched_copy(Load load, Store store) {
    constexpr int PER = (TOTAL + T2D - 1) / T2D;
    constexpr int LIM = sizeof(C) <= 8 ? 16 : 8;
    constexpr int G = PER < LIM ? PER : LIM;
#pragma unroll 1
    for (int k0 = 0; k0 < PER; k0 += G) {
        C v[G];
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int item = threadIdx.x + (k0 + k) * T2D;
            if (TOTAL % T2D == 0 || item < TOTAL) v[k] = load(item);
        }
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const int item = threadIdx.x + (k0 + k) * T2D;
            if (TOTAL % T2D == 0 || item < TOTAL) store(item, v[k]);
        }
    }
}

// Hint the L2 to fetch `bytes` from p (one request per 128-byte line).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const char* c = static_cast<const char*>(p);
    for (size_t off = (size_t)threadIdx.x * 128; off < bytes; off += (size_t)T2D * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// ------------------------------------------------------------ element helpers
// Start of a step at mode (m0, m1): returns the inverse-DFT input and updates
// the state slot (W or X) in MODE_STEP.
template <class C, class RT>
__device__ __forceinline__ C begin_elem(const KArgs& a, bool step, int b, state_t<RT>* st, const RT* ringb,
                                        size_t NP, size_t idx, int m0, int m1, int n_e) {
    using ST = state_t<RT>;
    constexpr bool FF = !is_f64<RT>::value;
    ST W = st[idx];
    if (step) {
        if constexpr (!FF) {
            Phase2D ph{a, b, m0, m1};
            W = horner_W64(a, W, ringb, NP, idx, ph);
            st[idx] = W;
            return cvt<C>(W);
        } else {
            if (a.ip) {
                W = ip_X(a, W, ringb, NP, idx);
                st[idx] = W;
                return cvt<C>(cmul(e_2d(a, b, n_e, m0, m1), make_float2(W.x, W.y)));
            }
            W = mixed_X(a, W, ringb, NP, idx);
            Phase2D ph{a, b, m0, m1};
            W = ffc_mul(ph.pff(0), W);
            st[idx] = W;
            return st_to_c<C>(W);
        }
    }
    if (a.mode == MODE_READ && a.ip) {
        const double2 E = a.flat1d ? e_exact(a, b, a.e_step, kmode(m0 * a.n1 + m1, a.tn0), 0.0, 1)
                          : a.tn2 ? e_exact3(a, b, a.e_step, m0, m1)
                                  : e_exact(a, b, a.e_step, kmode(m0, a.n0), kmode(m1, a.n1), 2);
        return cvt<C>(cmul(E, st_to_d(W)));
    }
    return st_to_c<C>(W);
}

// End of a step at mode (m0, m1) given R (already scaled): ring and state.
template <class C, class RT>
__device__ __forceinline__ void end_elem(const KArgs& a, bool step, int b, state_t<RT>* st, RT* ringb,
                                         size_t NP, size_t idx, int m0, int m1, C Rc, int n_e) {
    constexpr bool FF = !is_f64<RT>::value;
    RT r = cvt<RT>(Rc);
    if constexpr (FF) {
        if (step && a.ip) {
            r = cmul(make_float2(a.zr[0], a.zr[1]), cmul(conjf2(e_2d(a, b, n_e, m0, m1)), r));
            ringb[(size_t)a.out_slot * NP + idx] = r;
            st[idx] = ip_update(a, st[idx], r);
            return;
        }
    }
    ringb[(size_t)a.out_slot * NP + idx] = r;
    if (step) {
        if constexpr (FF) st[idx] = update_ff(a, st[idx], r);
        else st[idx] = update64(st[idx], r, a.h * a.mu[0]);
    }
}

// ---------------------------------------------------------------- col_begin
template <class C, class RT, int N0>
__global__ void __launch_bounds__(T2D, min_blocks_2d<C>()) k_col_begin(const KArgs a) {
    constexpr int L = LANES2D;
    using FI = CtaFft<C, N0, L, L, T2D, true>;
    using ST = state_t<RT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int b = blockIdx.y;
    const int c0 = blockIdx.x * L;
    const int n1 = a.n1;
    const size_t NP = (size_t)N0 * n1;
    ST* st = reinterpret_cast<ST*>(a.uhat) + (size_t)b * NP;
    const RT* ringb = reinterpret_cast<const RT*>(a.ring) + (size_t)b * a.ring_slots * NP;
    const C* tw;
    const C* twl;
    if constexpr (is_f64<C>::value) { tw = a.tw64_0; twl = tw; } else { tw = a.tw32_0; twl = a.tw32lo_0; }
    const bool step = (a.mode == MODE_STEP);

#pragma unroll 1
    for (int item = threadIdx.x; item < N0 * L; item += T2D) {
        const int lane = item % L, m0 = item / L;
        const int m1 = c0 + lane;
        buf[m0 * L + lane] = begin_elem<C, RT>(a, step, b, st, ringb, NP, (size_t)m0 * n1 + m1, m0, m1, a.e_step);
    }
    __syncthreads();
    FI::run(buf, tw, twl);
    C* T1 = reinterpret_cast<C*>(a.aux) + (size_t)b * NP;
    for (int item = threadIdx.x; item < N0 * L; item += T2D) {
        const int lane = item % L, i0 = item / L;
        T1[(size_t)i0 * n1 + c0 + lane] = buf[i0 * L + lane];
    }
}

// 1D grids through the passes: the four-step twiddle e^{-2 pi i r c / N} of
// row r, position c (conjugated before the inverse row transform).
template <bool CONJ>
__device__ __forceinline__ double2 tw1d(const KArgs& a, int r, int c, double2 v) {
    double2 w = __ldg(&a.tw1d64[(size_t)r * c]);
    if (CONJ) w.y = -w.y;
    return cmul(v, w);
}
template <bool CONJ>
__device__ __forceinline__ float2 tw1d(const KArgs& a, int r, int c, float2 v) {
    float2 w = __ldg(&a.tw1d32[(size_t)r * c]);
    if (CONJ) w.y = -w.y;
    return cmul(v, w);
}

// ------------------------------------------------------------------ row_mid
// V loads per thread in flight in the FP32 element phase: one at a time
// 0.4653, 4 or 8 0.4537 ms per 64 x 512^2 mixed step (4 instance groups).
#ifndef TDSE_ROW_VG
#define TDSE_ROW_VG 8
#endif
template <class C, int N1>
__global__ void __launch_bounds__(T2D, row_min_blocks<C>()) k_row_mid(const KArgs a) {
    constexpr int L = LANES2D;
    constexpr int LS = L + 1;
    using FI = CtaFft<C, N1, L, LS, T2D, true>;
    using FW = CtaFft<C, N1, L, LS, T2D, false>;
    using R = typename cx_traits<C>::real;
    constexpr bool F64 = is_f64<C>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int b = blockIdx.y;
    const int r0 = blockIdx.x * L;
    const int n0 = a.n0;
    const size_t NP = (size_t)n0 * N1;
    const C* tw;
    const C* twl;
    if constexpr (F64) { tw = a.tw64_1; twl = tw; } else { tw = a.tw32_1; twl = a.tw32lo_1; }
    const double vfac = a.tfac[(size_t)b * a.ntf + a.tf];
    const double* V0 = a.V0 + (size_t)b * a.vstride;
    const float2* V0f = a.V0f + (size_t)b * a.vstride;
    const float fh = (float)vfac, fl = (float)(vfac - (double)fh);
    const R scale = (R)1 / (R)N1;

    if (a.mode == MODE_INIT) {
        // T2 = F1 (V u0), then T1 = F1 u0 (u0 is parked as raw FP64 pairs in the state slot).
        const double2* u0 = reinterpret_cast<const double2*>(a.uhat) + (size_t)b * NP;
        C* T1 = reinterpret_cast<C*>(a.aux) + (size_t)b * NP;
        C* T2 = reinterpret_cast<C*>(a.aux2) + (size_t)b * NP;
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            for (int item = threadIdx.x; item < N1 * L; item += T2D) {
                const int lane = item / N1, j1 = item % N1;
                const size_t idx = (size_t)(r0 + lane) * N1 + j1;
                const C u = cvt<C>(u0[idx]);
                buf[j1 * LS + lane] = pass == 0 ? cscale(u, (R)(vfac * V0[idx])) : u;
            }
            __syncthreads();
            FW::run(buf, tw, twl);
            C* dst = pass == 0 ? T2 : T1;
            for (int item = threadIdx.x; item < N1 * L; item += T2D) {
                const int lane = item / N1, k1 = item % N1;
                C v = buf[k1 * LS + lane];
                if (a.flat1d) v = tw1d<false>(a, r0 + lane, k1, v);
                dst[(size_t)(r0 + lane) * N1 + k1] = cscale(v, scale);
            }
            __syncthreads();
        }
        return;
    }

    if (!F64 && a.mode == MODE_STEP) prefetch_l2(V0f + (size_t)r0 * N1, (size_t)L * N1 * sizeof(float2));
    const C* T1 = reinterpret_cast<const C*>(a.aux) + (size_t)b * NP;
    if (a.flat1d)
        batched_copy<C, N1 * L>([&](int item) { return T1[(size_t)(r0 + item / N1) * N1 + item % N1]; },
                                [&](int item, C v) {
                                    buf[(item % N1) * LS + item / N1] = tw1d<true>(a, r0 + item / N1, item % N1, v);
                                });
    else
        batched_copy<C, N1 * L>([&](int item) { return T1[(size_t)(r0 + item / N1) * N1 + item % N1]; },
                                [&](int item, C v) { buf[(item % N1) * LS + item / N1] = v; });
    __syncthreads();
    FI::run(buf, tw, twl);

    if (a.mode == MODE_READ) {
        double2* out = a.aux2 + (size_t)b * NP;
        for (int item = threadIdx.x; item < N1 * L; item += T2D) {
            const int lane = item / N1, j1 = item % N1;
            out[(size_t)(r0 + lane) * N1 + j1] = cvt<double2>(buf[j1 * LS + lane]);
        }
        return;
    }

    const R hmu0 = (a.mode == MODE_STEP) ? (R)(a.h * a.mu[0]) : (R)0;
    if constexpr (F64) {
        for (int item = threadIdx.x; item < N1 * L; item += T2D) {
            const int lane = item / N1, j1 = item % N1;
            const size_t idx = (size_t)(r0 + lane) * N1 + j1;
            buf[j1 * LS + lane] = implicit_solve_times_V(buf[j1 * LS + lane], (R)(vfac * V0[idx]), (R)0, hmu0);
        }
    } else {
        // V hi/lo of TDSE_ROW_VG points per thread in flight at a time (L2 hits after the prefetch)
        constexpr int PER = (N1 * L + T2D - 1) / T2D;
        constexpr int G = PER < TDSE_ROW_VG ? PER : TDSE_ROW_VG;
#pragma unroll 1
        for (int k0 = 0; k0 < PER; k0 += G) {
            float2 v2[G];
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int item = threadIdx.x + (k0 + k) * T2D;
                if ((N1 * L) % T2D == 0 || item < N1 * L)
                    v2[k] = __ldg(&V0f[(size_t)(r0 + item / N1) * N1 + item % N1]);
            }
#pragma unroll
            for (int k = 0; k < G; ++k) {
                const int item = threadIdx.x + (k0 + k) * T2D;
                if ((N1 * L) % T2D == 0 || item < N1 * L) {
                    const int lane = item / N1, j1 = item % N1;
                    const float vh = fh * v2[k].x;
                    const float vl = fmaf(fh, v2[k].x, -vh) + fmaf(fh, v2[k].y, fl * v2[k].x);
                    buf[j1 * LS + lane] = implicit_solve_times_V(buf[j1 * LS + lane], vh, vl, hmu0);
                }
            }
        }
    }
    __syncthreads();
    FW::run(buf, tw, twl);
    C* T2 = reinterpret_cast<C*>(a.aux2) + (size_t)b * NP;
    for (int item = threadIdx.x; item < N1 * L; item += T2D) {
        const int lane = item / N1, k1 = item % N1;
        C v = buf[k1 * LS + lane];
        if (a.flat1d) v = tw1d<false>(a, r0 + lane, k1, v);
        T2[(size_t)(r0 + lane) * N1 + k1] = cscale(v, scale);
    }
}

// ------------------------------------------------------ col_end / col_fused
template <class C, class RT, int N0, bool FUSED>
__global__ void __launch_bounds__(T2D, min_blocks_2d<C>()) k_col_end(const KArgs a) {
    constexpr int L = LANES2D;
    using FW = CtaFft<C, N0, L, L, T2D, false>;
    using FI = CtaFft<C, N0, L, L, T2D, true>;
    using R = typename cx_traits<C>::real;
    using ST = state_t<RT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int b = blockIdx.y;
    const int c0 = blockIdx.x * L;
    const int n1 = a.n1;
    const size_t NP = (size_t)N0 * n1;
    ST* st = reinterpret_cast<ST*>(a.uhat) + (size_t)b * NP;
    RT* ringb = reinterpret_cast<RT*>(a.ring) + (size_t)b * a.ring_slots * NP;
    const C* tw;
    const C* twl;
    if constexpr (is_f64<C>::value) { tw = a.tw64_0; twl = tw; } else { tw = a.tw32_0; twl = a.tw32lo_0; }
    const R scale = (R)1 / (R)N0;

    auto load_tile = [&](const C* src) {
        batched_copy<C, N0 * L>([&](int item) { return src[(size_t)(item / L) * n1 + c0 + item % L]; },
                                [&](int item, C v) { buf[item] = v; });
        __syncthreads();
        FW::run(buf, tw, twl);
    };
    load_tile(reinterpret_cast<const C*>(a.aux2) + (size_t)b * NP);

    if (a.mode == MODE_INIT) {
        for (int item = threadIdx.x; item < N0 * L; item += T2D) {
            const int lane = item % L, m0 = item / L;
            ringb[(size_t)a.out_slot * NP + (size_t)m0 * n1 + c0 + lane] = cvt<RT>(cscale(buf[m0 * L + lane], scale));
        }
        __syncthreads();
        load_tile(reinterpret_cast<const C*>(a.aux) + (size_t)b * NP);
        for (int item = threadIdx.x; item < N0 * L; item += T2D) {
            const int lane = item % L, m0 = item / L;
            st[(size_t)m0 * n1 + c0 + lane] = d_to_st<ST>(cvt<double2>(cscale(buf[m0 * L + lane], scale)));
        }
        return;
    }

    const bool step = (a.mode == MODE_STEP);
#pragma unroll 1
    for (int item = threadIdx.x; item < N0 * L; item += T2D) {
        const int lane = item % L, m0 = item / L;
        const int m1 = c0 + lane;
        const size_t idx = (size_t)m0 * n1 + m1;
        end_elem<C, RT>(a, step, b, st, ringb, NP, idx, m0, m1, cscale(buf[m0 * L + lane], scale), a.e_step);
        if constexpr (FUSED) buf[m0 * L + lane] = begin_elem<C, RT>(a, true, b, st, ringb, NP, idx, m0, m1, a.e_next);
    }
    if constexpr (FUSED) {
        __syncthreads();
        FI::run(buf, tw, twl);
        C* T1 = reinterpret_cast<C*>(a.aux) + (size_t)b * NP;
        for (int item = threadIdx.x; item < N0 * L; item += T2D) {
            const int lane = item % L, i0 = item / L;
            T1[(size_t)i0 * n1 + c0 + lane] = buf[i0 * L + lane];
        }
    }
}

// ------------------------------------- col_fused, mixed interaction-picture step
// Same work as k_col_end<float2, float2, N0, true> for MODE_STEP with the state
// in the interaction picture, with the mode-space reads staged: the state and
// the history slots of lags 2..nhist of each chunk of PF_ROWS rows are copied
// into shared memory with cp.async (16-byte copies, no registers held), two
// chunks ahead, so that the DRAM reads of the step overlap the column FFT
// and the element work of the previous chunk.  The intermediate v^_n is not
// stored (the state slot receives X_{n+1} directly).
#ifndef TDSE_PF_ROWS
#define TDSE_PF_ROWS 32
#endif
// 3D mixed chains use this kernel for their fused column pass as well
#ifndef TDSE_COL_IP_3D
#define TDSE_COL_IP_3D 1
#endif
// ... and 1D grids in the four-step layout
#ifndef TDSE_COL_IP_1D
#define TDSE_COL_IP_1D 1
#endif
constexpr int PF_ROWS = TDSE_PF_ROWS;

// VAR 0: 2D column blocks; 1: 3D (column index i1 n2 + i2); 2: a 1D grid in
// the four-step layout (flat1d: E_n of the flattened mode index).
template <int N0, int VAR>
__global__ void __launch_bounds__(T2D, TDSE_MINB2D) k_col_fused_ip(const KArgs a) {
    constexpr bool D3 = VAR == 1, FLAT = VAR == 2;
    constexpr int L = LANES2D;
    constexpr int RC = PF_ROWS < N0 ? PF_ROWS : N0;     // rows per chunk
    constexpr int NCH = N0 / RC;
    constexpr int NPF = MAX_HIST - 1;                  // lags 2..7 at most
    using FW = CtaFft<float2, N0, L, L, T2D, false>;
    using FI = CtaFft<float2, N0, L, L, T2D, true>;
    struct Chunk {
        float4 st[RC * L];
        float2 ring[NPF][RC * L];
    };
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);
    Chunk* pre = reinterpret_cast<Chunk*>(smem_raw + (size_t)N0 * L * sizeof(float2));
    const int b = blockIdx.y;
    const int c0 = blockIdx.x * L;
    const int n1 = a.n1;
    const size_t NP = (size_t)N0 * n1;
    float4* st = reinterpret_cast<float4*>(a.uhat) + (size_t)b * NP;
    float2* ringb = reinterpret_cast<float2*>(a.ring) + (size_t)b * a.ring_slots * NP;
    const int npf = a.nhist - 1;                      // slots to stage (lag 1 is the value written here)

    // stage chunk c into buffer c & 1: state rows (8 x 16 B) and ring rows (8 x 8 B) of the CTA's columns
    auto stage = [&](int c) {
        Chunk& ch = pre[c & 1];
        for (int it = threadIdx.x; it < RC * L; it += T2D) {          // state: one float4 per copy
            const int r = it / L, q = it % L;
            cp_async16(&ch.st[r * L + q], st + (size_t)(c * RC + r) * n1 + c0 + q);
        }
#pragma unroll
        for (int j = 0; j < NPF; ++j) {                                // lag j + 2: two float2 per copy
            if (j < npf) {
                const float2* src = ringb + (size_t)a.hist_slot[j + 1] * NP + c0;
                for (int it = threadIdx.x; it < RC * (L / 2); it += T2D) {
                    const int r = it / (L / 2), h = it % (L / 2);
                    cp_async16(&ch.ring[j][r * L + 2 * h], src + (size_t)(c * RC + r) * n1 + 2 * h);
                }
            }
        }
        cp_async_commit();
    };
    stage(0);
    if (NCH > 1) stage(1);

    const float2* T2 = reinterpret_cast<const float2*>(a.aux2) + (size_t)b * NP;
    batched_copy<float2, N0 * L>([&](int item) { return T2[(size_t)(item / L) * n1 + c0 + item % L]; },
                                 [&](int item, float2 v) { buf[item] = v; });
    __syncthreads();
    FW::run(buf, a.tw32_0, a.tw32lo_0);
    const float scale = 1.0f / (float)N0;
    const float2 z = make_float2(a.zr[0], a.zr[1]);
    // E_n(m0, m1) = e_n[m0] e_n[n0 + m1] (e_2d): the axis-1 factors of the
    // column a thread keeps (RC * L == T2D: one column per thread) are loaded once
    const size_t erow = (size_t)(a.tn0 + a.tn1 + a.tn2);
    const float2* en = FLAT ? nullptr : a.e2d + ((size_t)b * (a.ntf / 8 + 1) + a.e_step) * erow;
    const float2* en1 = FLAT ? nullptr : a.e2d + ((size_t)b * (a.ntf / 8 + 1) + a.e_next) * erow;
    constexpr bool ONE_COL = (RC * L == T2D);
    const int lane_t = threadIdx.x % L;
    float2 en_1 = make_float2(0.f, 0.f), en1_1 = en_1;
    if constexpr (!FLAT) {
        en_1 = __ldg(&en[a.tn0 + c0 + lane_t]);
        en1_1 = __ldg(&en1[a.tn0 + c0 + lane_t]);
    }
    // D3 (3D column blocks, column index i1 n2 + i2): E_n = (e[m0] e[n0 + i1]) e[n0 + n1 + i2] as in e_2d
    float2 e3_1 = en_1, e3_2 = en_1, e31_1 = en1_1, e31_2 = en1_1;
    if constexpr (D3) {
        int i1, i2;
        split12(a, c0 + lane_t, i1, i2);
        e3_1 = __ldg(&en[a.tn0 + i1]);
        e3_2 = __ldg(&en[a.tn0 + a.tn1 + i2]);
        e31_1 = __ldg(&en1[a.tn0 + i1]);
        e31_2 = __ldg(&en1[a.tn0 + a.tn1 + i2]);
    }
    float2* ring_out = ringb + (size_t)a.out_slot * NP;

#pragma unroll 1
    for (int c = 0; c < NCH; ++c) {
        if (c + 1 < NCH) cp_async_wait<1>(); else cp_async_wait<0>();
        __syncthreads();
        const Chunk& ch = pre[c & 1];
        for (int it = threadIdx.x; it < RC * L; it += T2D) {
            const int lane = it % L, r = it / L;
            const int m0 = c * RC + r, m1 = c0 + lane;
            const int pos = m0 * L + lane;
            const size_t idx = (size_t)m0 * n1 + m1;
            // end of step n: r~ = z_n R / E_n into the ring, v^_n
            const float2 R = cscale(buf[pos], scale);
            float2 rv;
            if constexpr (FLAT) {
                rv = cmul(z, cmul(conjf2(e_1d(a, b, a.e_step, m0 * n1 + m1)), R));
            } else if constexpr (D3) {
                if constexpr (!ONE_COL) {   // column factors of this element's column
                    int i1, i2;
                    split12(a, m1, i1, i2);
                    e3_1 = __ldg(&en[a.tn0 + i1]);
                    e3_2 = __ldg(&en[a.tn0 + a.tn1 + i2]);
                    e31_1 = __ldg(&en1[a.tn0 + i1]);
                    e31_2 = __ldg(&en1[a.tn0 + a.tn1 + i2]);
                }
                rv = cmul(z, cmul(conjf2(cmul(cmul(__ldg(&en[m0]), e3_1), e3_2)), R));
            } else {
                const float2 e1n = ONE_COL ? en_1 : __ldg(&en[a.tn0 + m1]);
                rv = cmul(z, cmul(conjf2(cmul(__ldg(&en[m0]), e1n)), R));
            }
            ring_out[idx] = rv;
            const float4 v = ip_update(a, ch.st[it], rv);
            // begin of step n+1: X = v^_n - i h sum_j c_j r~_{n+1-j}
            float2 S = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = MAX_HIST; j >= 1; --j) {        // same order and terms as history_sum_ip
                const float2 q = j > a.nhist ? make_float2(0.f, 0.f) : (j == 1 ? rv : ch.ring[j - 2][it]);
                const float hh = a.c_hi[j][0], hi = a.c_hi[j][1], lo = a.c_lo[j][0], li = a.c_lo[j][1];
                S.x = fmaf(lo, q.x, fmaf(-li, q.y, S.x));
                S.y = fmaf(lo, q.y, fmaf(li, q.x, S.y));
                S.x = fmaf(hh, q.x, fmaf(-hi, q.y, S.x));
                S.y = fmaf(hh, q.y, fmaf(hi, q.x, S.y));
            }
            const float4 X = ff_minus_i_times(v, a.h_hi, a.h_lo, S);
            st[idx] = X;
            if constexpr (FLAT) {
                buf[pos] = cmul(e_1d(a, b, a.e_next, m0 * n1 + m1), make_float2(X.x, X.y));
            } else if constexpr (D3) {
                buf[pos] = cmul(cmul(cmul(__ldg(&en1[m0]), e31_1), e31_2), make_float2(X.x, X.y));
            } else {
                const float2 e1n1 = ONE_COL ? en1_1 : __ldg(&en1[a.tn0 + m1]);
                buf[pos] = cmul(cmul(__ldg(&en1[m0]), e1n1), make_float2(X.x, X.y));
            }
        }
        __syncthreads();                               // buffer c & 1 free
        if (c + 2 < NCH) stage(c + 2);
    }
    FI::run(buf, a.tw32_0, a.tw32lo_0);
    float2* T1 = reinterpret_cast<float2*>(a.aux) + (size_t)b * NP;
    for (int item = threadIdx.x; item < N0 * L; item += T2D) {
        const int lane = item % L, i0 = item / L;
        T1[(size_t)i0 * n1 + c0 + lane] = buf[i0 * L + lane];
    }
}

// ---------------------------------------------------------------- launchers
template <class K>
static cudaError_t set_smem(K kern, size_t smem, bool& done) {
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
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

template <class C, class RT, int N0, bool FUSED>
static cudaError_t col_end_n(const KArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)N0 * LANES2D * sizeof(C);
    static bool done = false;
    cudaError_t e = set_smem(k_col_end<C, RT, N0, FUSED>, smem, done);
    if (e != cudaSuccess) return e;
    k_col_end<C, RT, N0, FUSED><<<dim3(a.n1 / LANES2D, a.B), T2D, smem, s>>>(a);
    return cudaGetLastError();
}

template <int N0, int VAR = 0>
static cudaError_t col_fused_ip_n(const KArgs& a, cudaStream_t s) {
    constexpr int RC = PF_ROWS < N0 ? PF_ROWS : N0;
    const size_t smem = (size_t)N0 * LANES2D * sizeof(float2) +
                        2 * (size_t)RC * LANES2D * (sizeof(float4) + (MAX_HIST - 1) * sizeof(float2));
    static bool done = false;
    cudaError_t e = set_smem(k_col_fused_ip<N0, VAR>, smem, done);
    if (e != cudaSuccess) return e;
    k_col_fused_ip<N0, VAR><<<dim3(a.n1 / LANES2D, a.B), T2D, smem, s>>>(a);
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

#define TDSE_SWITCH_N(n, ...)                                \
    switch (n) {                                             \
        case 8: return __VA_ARGS__(8)(a, s);                 \
        case 16: return __VA_ARGS__(16)(a, s);               \
        case 32: return __VA_ARGS__(32)(a, s);               \
        case 64: return __VA_ARGS__(64)(a, s);               \
        case 128: return __VA_ARGS__(128)(a, s);             \
        case 256: return __VA_ARGS__(256)(a, s);             \
        case 512: return __VA_ARGS__(512)(a, s);             \
        case 1024: return __VA_ARGS__(1024)(a, s);           \
        default: return cudaErrorInvalidValue;               \
    }
#define TDSE_CB(n) col_begin_n<C, RT, n>
#define TDSE_CE(n) col_end_n<C, RT, n, false>
#define TDSE_CF(n) col_end_n<C, RT, n, true>
#define TDSE_RM(n) row_mid_n<C, n>

template <class C, class RT> static cudaError_t col_begin(const KArgs& a, cudaStream_t s) { TDSE_SWITCH_N(a.n0, TDSE_CB) }
template <class C, class RT> static cudaError_t col_end(const KArgs& a, cudaStream_t s) { TDSE_SWITCH_N(a.n0, TDSE_CE) }
template <class C, class RT> static cudaError_t col_fused(const KArgs& a, cudaStream_t s) { TDSE_SWITCH_N(a.n0, TDSE_CF) }
template <class C> static cudaError_t row_mid(const KArgs& a, cudaStream_t s) { TDSE_SWITCH_N(a.n1, TDSE_RM) }

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

template <class C, class RT>
static cudaError_t part2d(const KArgs& a, int part, cudaStream_t s) {
    switch (part) {
        case PART_COL_BEGIN: return col_begin<C, RT>(a, s);
        case PART_ROW_MID: return row_mid<C>(a, s);
        case PART_COL_END: return col_end<C, RT>(a, s);
        case PART_COL_FUSED:
            if constexpr (std::is_same<C, float2>::value && std::is_same<RT, float2>::value) {
                if (a.mode == MODE_STEP && a.ip && a.tn2 == 0 && !a.flat1d) {
#define TDSE_CFI(n) col_fused_ip_n<n>
                    TDSE_SWITCH_N(a.n0, TDSE_CFI)
#undef TDSE_CFI
                }
                if (TDSE_COL_IP_1D && a.mode == MODE_STEP && a.ip && a.flat1d) {
#define TDSE_CFI1(n) col_fused_ip_n<n, 2>
                    TDSE_SWITCH_N(a.n0, TDSE_CFI1)
#undef TDSE_CFI1
                }
            }
            return col_fused<C, RT>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ 3D
// Transform along axis 1 of [B n0][N1][n2] (one CTA per 8 consecutive i2 of
// one (instance, i0) plane), in place in X: forward with 1/N1, or inverse.
template <class C, int N1, bool INV>
__global__ void __launch_bounds__(T2D, min_blocks_2d<C>()) k_axis1(const KArgs a, C* X) {
    constexpr int L = LANES2D;
    using F = CtaFft<C, N1, L, L, T2D, INV>;
    using R = typename cx_traits<C>::real;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int n2 = a.tn2;
    const size_t plane = (size_t)blockIdx.z * a.tn0 + blockIdx.y;
    C* base = X + plane * (size_t)N1 * n2 + (size_t)blockIdx.x * L;
    batched_copy<C, N1 * L>([&](int item) { return base[(size_t)(item / L) * n2 + item % L]; },
                            [&](int item, C v) { buf[item] = v; });
    __syncthreads();
    const C* tw;
    const C* twl;
    if constexpr (is_f64<C>::value) { tw = a.tw64_1; twl = tw; } else { tw = a.tw32_1; twl = a.tw32lo_1; }
    F::run(buf, tw, twl);
    const R scale = (R)1 / (R)N1;
    for (int item = threadIdx.x; item < N1 * L; item += T2D)
        base[(size_t)(item / L) * n2 + item % L] = INV ? buf[item] : cscale(buf[item], scale);
}

template <class C, int N1>
static cudaError_t axis1_n(const KArgs& a, bool inv, void* X, cudaStream_t s) {
    const size_t smem = (size_t)N1 * LANES2D * sizeof(C);
    static bool done_f = false, done_i = false;
    cudaError_t e = inv ? set_smem(k_axis1<C, N1, true>, smem, done_i) : set_smem(k_axis1<C, N1, false>, smem, done_f);
    if (e != cudaSuccess) return e;
    const dim3 grid(a.tn2 / LANES2D, a.tn0, a.B);
    if (inv) k_axis1<C, N1, true><<<grid, T2D, smem, s>>>(a, static_cast<C*>(X));
    else k_axis1<C, N1, false><<<grid, T2D, smem, s>>>(a, static_cast<C*>(X));
    return cudaGetLastError();
}

template <class C>
static cudaError_t axis1(const KArgs& a, bool inv, void* X, cudaStream_t s) {
    switch (a.tn1) {
        case 8: return axis1_n<C, 8>(a, inv, X, s);
        case 16: return axis1_n<C, 16>(a, inv, X, s);
        case 32: return axis1_n<C, 32>(a, inv, X, s);
        case 64: return axis1_n<C, 64>(a, inv, X, s);
        case 128: return axis1_n<C, 128>(a, inv, X, s);
        case 256: return axis1_n<C, 256>(a, inv, X, s);
        default: return cudaErrorInvalidValue;
    }
}

// Launch geometry of the 3D passes: the column pass over the n1 n2 columns of
// [n0][n1 n2], the row pass over the n0 n1 rows of [n0 n1][n2] with the axis-2
// twiddles.
static KArgs col3(const KArgs& a) {
    KArgs c = a;
    c.n0 = a.tn0;
    c.n1 = a.tn1 * a.tn2;
    return c;
}
static KArgs row3(const KArgs& a) {
    KArgs r = a;
    r.n0 = a.tn0 * a.tn1;
    r.n1 = a.tn2;
    r.tw64_1 = a.tw64_2;
    r.tw32_1 = a.tw32_2;
    r.tw32lo_1 = a.tw32lo_2;
    return r;
}

// The fused column pass of a 3D chain: the staged interaction-picture kernel
// for mixed steps (3D column blocks), the generic one otherwise.
template <class C, class RT>
static cudaError_t col_fused_3d(const KArgs& a, cudaStream_t s) {
    if constexpr (std::is_same<C, float2>::value && std::is_same<RT, float2>::value) {
        if (TDSE_COL_IP_3D && a.mode == MODE_STEP && a.ip) {
#define TDSE_CFI3(n) col_fused_ip_n<n, 1>
            TDSE_SWITCH_N(a.n0, TDSE_CFI3)
#undef TDSE_CFI3
        }
    }
    return col_fused<C, RT>(a, s);
}

template <class C, class RT>
static cudaError_t part3d(const KArgs& a, int part, cudaStream_t s) {
    const KArgs c = col3(a), r = row3(a);
    cudaError_t e = cudaSuccess;
    switch (part) {
        case PART_COL_BEGIN:
            if ((e = col_begin<C, RT>(c, s)) != cudaSuccess) return e;
            return axis1<C>(a, true, a.aux, s);
        case PART_ROW_MID: return row_mid<C>(r, s);
        case PART_COL_END:
            if ((e = axis1<C>(a, false, a.aux2, s)) != cudaSuccess) return e;
            return col_end<C, RT>(c, s);
        case PART_COL_FUSED:
            if ((e = axis1<C>(a, false, a.aux2, s)) != cudaSuccess) return e;
            if ((e = col_fused_3d<C, RT>(c, s)) != cudaSuccess) return e;
            return axis1<C>(a, true, a.aux, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class C, class RT>
static cudaError_t run3d(const KArgs& a, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    switch (a.mode) {
        case MODE_STEP:
        case MODE_REFRESH:
            if ((e = part3d<C, RT>(a, PART_COL_BEGIN, s)) != cudaSuccess) return e;
            if ((e = part3d<C, RT>(a, PART_ROW_MID, s)) != cudaSuccess) return e;
            return part3d<C, RT>(a, PART_COL_END, s);
        case MODE_INIT:   // T1 = F2 u0, T2 = F2 V u0, then axis 1 of both, then axis 0 into state and ring
            if ((e = row_mid<C>(row3(a), s)) != cudaSuccess) return e;
            if ((e = axis1<C>(a, false, a.aux, s)) != cudaSuccess) return e;
            if ((e = axis1<C>(a, false, a.aux2, s)) != cudaSuccess) return e;
            return col_end<C, RT>(col3(a), s);
        case MODE_READ:
            if ((e = part3d<C, RT>(a, PART_COL_BEGIN, s)) != cudaSuccess) return e;
            return row_mid<C>(row3(a), s);
        default:
            return cudaErrorInvalidValue;
    }
}

bool periodic3d_supported(int n0, int n1, int n2) {
    auto ok = [](int n, int hi) { return n >= 8 && n <= hi && (n & (n - 1)) == 0; };
    return ok(n0, 1024) && ok(n1, 256) && ok(n2, 1024) && (long long)n0 * n1 * n2 <= (1LL << 24);
}

cudaError_t launch_periodic3d(const KArgs& a, int combo, cudaStream_t s) {
    if (!periodic3d_supported(a.tn0, a.tn1, a.tn2)) return cudaErrorInvalidValue;
    switch (combo) {
        case COMBO_F64: return run3d<double2, double2>(a, s);
        case COMBO_F32: return run3d<float2, float2>(a, s);
        case COMBO_F64_R32: return run3d<double2, float2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_periodic3d_part(const KArgs& a, int combo, int part, cudaStream_t s) {
    if (!periodic3d_supported(a.tn0, a.tn1, a.tn2)) return cudaErrorInvalidValue;
    switch (combo) {
        case COMBO_F64: return part3d<double2, double2>(a, part, s);
        case COMBO_F32: return part3d<float2, float2>(a, part, s);
        case COMBO_F64_R32: return part3d<double2, float2>(a, part, s);
        default: return cudaErrorInvalidValue;
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

cudaError_t launch_periodic2d_part(const KArgs& a, int combo, int part, cudaStream_t s) {
    if (!periodic2d_supported(a.n0, a.n1)) return cudaErrorInvalidValue;
    switch (combo) {
        case COMBO_F64: return part2d<double2, double2>(a, part, s);
        case COMBO_F32: return part2d<float2, float2>(a, part, s);
        case COMBO_F64_R32: return part2d<double2, float2>(a, part, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tdse
