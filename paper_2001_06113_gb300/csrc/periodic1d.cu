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
// parked in the state's own slot (L2-resident) and read back.
#include "step_common.cuh"

namespace tdse {

constexpr int threads_1d(int N) { return N / 8 < 32 ? 32 : (N / 8 > 512 ? 512 : N / 8); }

// The step of one instance b by a group of T threads (index tid, barrier sync)
// with the N-element transform buffer buf in shared memory.
template <class C, class RT, int N, int T, class Sync>
__device__ __forceinline__ void step1d(const KArgs& a, const int b, const int tid, const Sync& sync, C* buf) {
    using FI = Fft<C, N, 1, 1, T, true>;     // inverse transform (modes -> grid)
    using FW = Fft<C, N, 1, 1, T, false>;    // forward transform (grid -> modes)
    static_assert(FI::RL == FW::RF && FI::PL == FW::PF, "inverse output regs feed forward input regs");
    static_assert(FW::RL == FI::RF && FW::PL == FI::PF, "forward output regs sit on the step's modes");
    constexpr int PB = FI::PF, RB = FI::RF;  // a thread's modes: j + r FI::NBF (= j + r FW::NBL)
    constexpr bool KEEP = PB * RB <= 8;
    constexpr bool F64 = is_f64<C>::value;
    constexpr bool FF = !is_f64<RT>::value;  // double-float state
    using ST = state_t<RT>;
    using R = typename cx_traits<C>::real;
    const size_t NP = N;
    ST* st = reinterpret_cast<ST*>(a.uhat) + (size_t)b * NP;
    RT* ringb = reinterpret_cast<RT*>(a.ring) + (size_t)b * a.ring_slots * NP;
    const C* tw;
    const C* twl;
    if constexpr (F64) { tw = a.tw64_0; twl = tw; } else { tw = a.tw32_0; twl = a.tw32lo_0; }
    const double vfac = a.tfac[(size_t)b * a.ntf + a.tf];
    const double* V0 = a.V0 + (size_t)b * NP;
    const float2* V0f = a.V0f + (size_t)b * NP;
    const R scale = (R)1 / (R)N;
    const float fh = (float)vfac, fl = (float)(vfac - (double)fh);

    // V(x_j, t) as hi + lo in the compute precision
    auto Vat = [&](int j, R& hi, R& lo) {
        if constexpr (F64) {
            hi = vfac * V0[j];
            lo = 0.0;
        } else {
            const float2 v2 = V0f[j];
            hi = fh * v2.x;
            lo = fmaf(fh, v2.x, -hi) + fmaf(fh, v2.y, fl * v2.x);
        }
    };

    if (a.mode == MODE_INIT) {
        // (V u0)^ -> ring[out]; u0 is parked as raw FP64 pairs in the state slot
        // (overwritten below by the state in its own format).
        const double2* u0 = reinterpret_cast<const double2*>(a.uhat) + (size_t)b * NP;
        C in[FW::PF][FW::RF], out[FW::PL][FW::RL];
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
            for (int p = 0; p < FW::PF; ++p) {
                int j, line;
                if (FW::item(p, FW::NBF, j, line, tid)) {
#pragma unroll
                    for (int r = 0; r < FW::RF; ++r) {
                        const int x = j + r * FW::NBF;
                        const C u = cvt<C>(u0[x]);
                        in[p][r] = pass == 0 ? cscale(u, (R)(vfac * V0[x])) : u;
                    }
                }
            }
            FW::run(in, out, buf, tw, twl, tid, sync);
#pragma unroll
            for (int p = 0; p < FW::PL; ++p) {
                int j, line;
                if (FW::item(p, FW::NBL, j, line, tid)) {
#pragma unroll
                    for (int r = 0; r < FW::RL; ++r) {
                        const int k = j + r * FW::NBL;
                        const C v = cscale(out[p][r], scale);
                        if (pass == 0) ringb[(size_t)a.out_slot * NP + k] = cvt<RT>(v);
                    }
                }
            }
            if (pass == 0) sync();   // every thread has read u0 before any state write
        }
        // the last forward result is still in registers: write the state
#pragma unroll
        for (int p = 0; p < FW::PL; ++p) {
            int j, line;
            if (FW::item(p, FW::NBL, j, line, tid)) {
#pragma unroll
                for (int r = 0; r < FW::RL; ++r)
                    st[j + r * FW::NBL] = d_to_st<ST>(cvt<double2>(cscale(out[p][r], scale)));
            }
        }
        return;
    }

    if (a.mode == MODE_READ) {
        C in[FI::PF][FI::RF], out[FI::PL][FI::RL];
#pragma unroll
        for (int p = 0; p < FI::PF; ++p) {
            int j, line;
            if (FI::item(p, FI::NBF, j, line, tid)) {
#pragma unroll
                for (int r = 0; r < FI::RF; ++r) {
                    const int k = j + r * FI::NBF;
                    double2 v = st_to_d(st[k]);
                    if (a.ip) v = cmul(e_exact(a, b, a.e_step, kmode(k, N), 0.0, 1), v);
                    in[p][r] = cvt<C>(v);
                }
            }
        }
        FI::run(in, out, buf, tw, twl, tid, sync);
        double2* outg = a.aux2 + (size_t)b * NP;
#pragma unroll
        for (int p = 0; p < FI::PL; ++p) {
            int j, line;
            if (FI::item(p, FI::NBL, j, line, tid)) {
#pragma unroll
                for (int r = 0; r < FI::RL; ++r) outg[j + r * FI::NBL] = cvt<double2>(out[p][r]);
            }
        }
        return;
    }

    const bool step = (a.mode == MODE_STEP);
    ST Wk[KEEP ? PB : 1][KEEP ? RB : 1];
    C in[PB][RB], mid[FI::PL][FI::RL], out[FW::PL][FW::RL];
#pragma unroll
    for (int p = 0; p < PB; ++p) {
        int j, line;
        if (FI::item(p, FI::NBF, j, line, tid)) {
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                const int k = j + r * FI::NBF;
                ST W = st[k];
                C x;
                if (step) {
                    if constexpr (!FF) {
                        Phase1D ph{a, b, k};
                        W = horner_W64(a, W, reinterpret_cast<const double2*>(ringb), NP, (size_t)k, ph);
                        x = cvt<C>(W);
                    } else {
                        if (a.ip) {
                            W = ip_X(a, W, reinterpret_cast<const float2*>(ringb), NP, (size_t)k);
                            x = cvt<C>(cmul(e_1d(a, b, a.e_step, k), make_float2(W.x, W.y)));
                        } else {
                            W = mixed_X(a, W, reinterpret_cast<const float2*>(ringb), NP, (size_t)k);
                            Phase1D ph{a, b, k};
                            W = ffc_mul(ph.pff(0), W);
                            x = st_to_c<C>(W);
                        }
                    }
                    if constexpr (KEEP) Wk[p][r] = W; else st[k] = W;
                } else {
                    x = st_to_c<C>(W);
                }
                in[p][r] = x;
            }
        }
    }
    FI::run(in, mid, buf, tw, twl, tid, sync);
    const R hmu0 = step ? (R)(a.h * a.mu[0]) : (R)0;
#pragma unroll
    for (int p = 0; p < FI::PL; ++p) {
        int j, line;
        if (FI::item(p, FI::NBL, j, line, tid)) {
#pragma unroll
            for (int r = 0; r < FI::RL; ++r) {
                R vh, vl;
                Vat(j + r * FI::NBL, vh, vl);
                mid[p][r] = implicit_solve_times_V(mid[p][r], vh, vl, hmu0);
            }
        }
    }
    FW::run(mid, out, buf, tw, twl, tid, sync);
#pragma unroll
    for (int p = 0; p < FW::PL; ++p) {
        int j, line;
        if (FW::item(p, FW::NBL, j, line, tid)) {
#pragma unroll
            for (int r = 0; r < FW::RL; ++r) {
                const int k = j + r * FW::NBL;
                RT rv = cvt<RT>(cscale(out[p][r], scale));
                bool done = false;
                if constexpr (FF) {
                    if (step && a.ip) {
                        rv = cmul(make_float2(a.zr[0], a.zr[1]), cmul(conjf2(e_1d(a, b, a.e_step, k)), rv));
                        ringb[(size_t)a.out_slot * NP + k] = rv;
                        st[k] = ip_update(a, KEEP ? Wk[p][r] : st[k], rv);
                        done = true;
                    }
                }
                if (!done) {
                    ringb[(size_t)a.out_slot * NP + k] = rv;
                    if (step) {
                        const ST W = KEEP ? Wk[p][r] : st[k];
                        if constexpr (FF) st[k] = update_ff(a, W, rv);
                        else st[k] = update64(W, rv, a.h * a.mu[0]);
                    }
                }
            }
        }
    }
}

template <class C, class RT, int N>
__global__ void __launch_bounds__(threads_1d(N)) k_periodic1d(const KArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step1d<C, RT, N, threads_1d(N)>(a, blockIdx.x, threadIdx.x, CtaSync{}, reinterpret_cast<C*>(smem_raw));
}

// One-time kernel attributes (shared memory above 48 KB); done before the
// first launch and, for stream capture, by periodic1d_prepare beforehand.
template <class C, class RT, int N>
static cudaError_t prepare_n() {
    static bool configured = false;
    if (configured) return cudaSuccess;
    const size_t smem = (size_t)N * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_periodic1d<C, RT, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_periodic1d<C, RT, N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) configured = true;
    return e;
}

template <class C, class RT, int N>
static cudaError_t launch_n(const KArgs& a, cudaStream_t s) {
    constexpr int T = threads_1d(N);
    const size_t smem = (size_t)N * sizeof(C);
    cudaError_t e = prepare_n<C, RT, N>();
    if (e != cudaSuccess) return e;
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

cudaError_t periodic1d_prepare(int n, int combo) {
    switch (combo) {
        case COMBO_F64: return prepare_combo<double2, double2>(n);
        case COMBO_F32: return n == P1D_MAX_F32 ? prepare_n<float2, float2, P1D_MAX_F32>() : prepare_combo<float2, float2>(n);
        case COMBO_F64_R32: return prepare_combo<double2, float2>(n);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Uneven batches: one persistent launch runs the mixed step of many contexts.
namespace {

struct Variant {
    int n, t;
};
__host__ __device__ constexpr Variant kVariants[MULTI_NVAR] = {
    {256, 32},  {512, 64},   {512, 32},    {1024, 128}, {1024, 64}, {2048, 256}, {2048, 128}, {4096, 512},
    {4096, 256}, {8192, 512}, {16384, 512}, {128, 32},   {64, 32},   {32, 32},    {16, 32},    {8, 32}};

// `count` instances b0.. of one context, each by a group of T threads with
// its own N-element slice of shared memory.
template <int N, int T>
__device__ __forceinline__ void run_group(const KArgs& a, int b0, int count, float2* smem) {
    const int g = threadIdx.x / T, tid = threadIdx.x % T;
    if (g >= count) return;
    float2* buf = smem + (size_t)g * N;
    if constexpr (T == MULTI_CTA)
        step1d<float2, float2, N, T>(a, b0, tid, CtaSync{}, buf);
    else if constexpr (T == 32)
        step1d<float2, float2, N, T>(a, b0 + g, tid, WarpSync{}, buf);
    else
        step1d<float2, float2, N, T>(a, b0 + g, tid, GroupSync{1u + (unsigned)g, (unsigned)T}, buf);
}

__global__ void __launch_bounds__(MULTI_CTA, 1) k_periodic1d_multi(const __grid_constant__ MultiArgs1D m) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int take;
    float2* smem = reinterpret_cast<float2*>(smem_raw);
    for (;;) {
        if (threadIdx.x == 0) take = atomicAdd(m.next, 1);
        __syncthreads();
        const int i = take;
        if (i >= m.nitems) break;
        const MultiItem it = m.items[i];
        const KArgs& a = m.args[it.g];
        switch (it.var) {
            case 0: run_group<256, 32>(a, it.b0, it.count, smem); break;
            case 1: run_group<512, 64>(a, it.b0, it.count, smem); break;
            case 2: run_group<512, 32>(a, it.b0, it.count, smem); break;
            case 3: run_group<1024, 128>(a, it.b0, it.count, smem); break;
            case 4: run_group<1024, 64>(a, it.b0, it.count, smem); break;
            case 5: run_group<2048, 256>(a, it.b0, it.count, smem); break;
            case 6: run_group<2048, 128>(a, it.b0, it.count, smem); break;
            case 7: run_group<4096, 512>(a, it.b0, it.count, smem); break;
            case 8: run_group<4096, 256>(a, it.b0, it.count, smem); break;
            case 9: run_group<8192, 512>(a, it.b0, it.count, smem); break;
            case 10: run_group<16384, 512>(a, it.b0, it.count, smem); break;
            case 11: run_group<128, 32>(a, it.b0, it.count, smem); break;
            case 12: run_group<64, 32>(a, it.b0, it.count, smem); break;
            case 13: run_group<32, 32>(a, it.b0, it.count, smem); break;
            case 14: run_group<16, 32>(a, it.b0, it.count, smem); break;
            case 15: run_group<8, 32>(a, it.b0, it.count, smem); break;
            default: break;
        }
        __syncthreads();   // shared memory and `take` free for the next item
    }
}

}  // namespace

int multi_variant_n(int var) { return var >= 0 && var < MULTI_NVAR ? kVariants[var].n : 0; }
int multi_variant_t(int var) { return var >= 0 && var < MULTI_NVAR ? kVariants[var].t : 0; }
int multi_variant(int n, int t) {
    for (int v = 0; v < MULTI_NVAR; ++v)
        if (kVariants[v].n == n && kVariants[v].t == t) return v;
    return -1;
}
size_t multi_item_smem(int var, int count) { return (size_t)count * multi_variant_n(var) * sizeof(float2); }

int multi_occupancy(size_t smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_periodic1d_multi, MULTI_CTA, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t multi_prepare(size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(k_periodic1d_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_periodic1d_multi, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t launch_periodic1d_multi(const MultiArgs1D& m, int grid, size_t smem, cudaStream_t s) {
    if (m.nitems <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(m.next, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_periodic1d_multi<<<grid, MULTI_CTA, smem, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_periodic1d(const KArgs& a, int combo, cudaStream_t s) {
    if (a.n0 == P1D_MAX_F32 && combo == COMBO_F32) return launch_n<float2, float2, P1D_MAX_F32>(a, s);
    if (!periodic1d_supported(a.n0)) return cudaErrorInvalidValue;
    switch (combo) {
        case COMBO_F64: return dispatch_n<double2, double2>(a, s);
        case COMBO_F32: return dispatch_n<float2, float2>(a, s);
        case COMBO_F64_R32: return dispatch_n<double2, float2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tdse
