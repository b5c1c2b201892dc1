// The 1D periodic step of one instance by a group of threads (used by the
// one-CTA-per-instance kernels and by the fused launch of uneven batches).
#pragma once
#include "step_common.cuh"

namespace tdse {

// n = 16384 (FP32 only): 1024 threads, 16 points each (64 registers, ~200
// bytes spilled), one CTA per SM either way (128 KB of shared memory): 0.233
// -> 0.201 ms per step at 3M points against 512 threads; same bits.
#ifndef P1D_T16384
#define P1D_T16384 1024
#endif
constexpr int threads_1d(int N) {
    return N >= 16384 ? P1D_T16384 : (N / 8 < 32 ? 32 : (N / 8 > 512 ? 512 : N / 8));
}

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
    const double* V0 = a.V0 + (size_t)b * a.vstride;
    const float2* V0f = a.V0f + (size_t)b * a.vstride;
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
    // Start of the step at mode k: the inverse-transform input; W (or X) is
    // returned for the update.
    auto input_of = [&](int k, ST& W) -> C {
        W = st[k];
        if (!step) return st_to_c<C>(W);
        if constexpr (!FF) {
            Phase1D ph{a, b, k};
            W = horner_W64(a, W, reinterpret_cast<const double2*>(ringb), NP, (size_t)k, ph);
            return cvt<C>(W);
        } else {
            if (a.ip) {
                W = ip_X(a, W, reinterpret_cast<const float2*>(ringb), NP, (size_t)k);
                return cvt<C>(cmul(e_1d(a, b, a.e_step, k), make_float2(W.x, W.y)));
            }
            W = mixed_X(a, W, reinterpret_cast<const float2*>(ringb), NP, (size_t)k);
            Phase1D ph{a, b, k};
            W = ffc_mul(ph.pff(0), W);
            return st_to_c<C>(W);
        }
    };
    // End of the step at mode k from the forward-transform output o and W.
    auto output_of = [&](int k, C o, const ST& W) {
        RT rv = cvt<RT>(cscale(o, scale));
        if constexpr (FF) {
            if (step && a.ip) {
                rv = cmul(make_float2(a.zr[0], a.zr[1]), cmul(conjf2(e_1d(a, b, a.e_step, k)), rv));
                ringb[(size_t)a.out_slot * NP + k] = rv;
                st[k] = ip_update(a, W, rv);
                return;
            }
        }
        ringb[(size_t)a.out_slot * NP + k] = rv;
        if (step) {
            if constexpr (FF) st[k] = update_ff(a, W, rv);
            else st[k] = update64(W, rv, a.h * a.mu[0]);
        }
    };
    const R hmu0 = step ? (R)(a.h * a.mu[0]) : (R)0;
    auto solve = [&](C (&m)[FI::PL][FI::RL]) {
#pragma unroll
        for (int p = 0; p < FI::PL; ++p) {
            int j, line;
            if (FI::item(p, FI::NBL, j, line, tid)) {
#pragma unroll
                for (int r = 0; r < FI::RL; ++r) {
                    R vh, vl;
                    Vat(j + r * FI::NBL, vh, vl);
                    m[p][r] = implicit_solve_times_V(m[p][r], vh, vl, hmu0);
                }
            }
        }
    };

    // Large n (several items per thread, W parked in the state slot): the
    // element phases run one item at a time in a rolled loop, which keeps the
    // kernel's code within the instruction cache.
    constexpr bool ROLLED = !KEEP && PB > 1 && FI::NPASS > 1 && FW::NPASS > 1;
    if constexpr (ROLLED) {
#pragma unroll 1
        for (int p = 0; p < PB; ++p) {
            int j, line;
            C x[RB];
            if (FI::item(p, FI::NBF, j, line, tid)) {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int k = j + r * FI::NBF;
                    ST W;
                    x[r] = input_of(k, W);
                    if (step) st[k] = W;
                }
            }
            FI::first_item(p, x, buf, tid);
        }
        FI::middle(buf, tw, twl, tid, sync);
        C mid[FI::PL][FI::RL];
#pragma unroll
        for (int p = 0; p < FI::PL; ++p) {
            int j;
            FI::last_item(p, mid[p], buf, tw, twl, tid, j);
        }
        FI::finish(sync);
        solve(mid);
#pragma unroll
        for (int p = 0; p < FW::PF; ++p) FW::first_item(p, mid[p], buf, tid);
        FW::middle(buf, tw, twl, tid, sync);
#pragma unroll 1
        for (int p = 0; p < FW::PL; ++p) {
            C o[FW::RL];
            int j;
            if (FW::last_item(p, o, buf, tw, twl, tid, j)) {
#pragma unroll
                for (int r = 0; r < FW::RL; ++r) {
                    const int k = j + r * FW::NBL;
                    output_of(k, o[r], st[k]);
                }
            }
        }
        FW::finish(sync);
        return;
    } else {
        ST Wk[KEEP ? PB : 1][KEEP ? RB : 1];
        C in[PB][RB], mid[FI::PL][FI::RL], out[FW::PL][FW::RL];
#pragma unroll
        for (int p = 0; p < PB; ++p) {
            int j, line;
            if (FI::item(p, FI::NBF, j, line, tid)) {
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const int k = j + r * FI::NBF;
                    ST W;
                    in[p][r] = input_of(k, W);
                    if (step) {
                        if constexpr (KEEP) Wk[p][r] = W; else st[k] = W;
                    }
                }
            }
        }
        FI::run(in, mid, buf, tw, twl, tid, sync);
        solve(mid);
        FW::run(mid, out, buf, tw, twl, tid, sync);
#pragma unroll
        for (int p = 0; p < FW::PL; ++p) {
            int j, line;
            if (FW::item(p, FW::NBL, j, line, tid)) {
#pragma unroll
                for (int r = 0; r < FW::RL; ++r) {
                    const int k = j + r * FW::NBL;
                    output_of(k, out[p][r], KEEP ? Wk[p][r] : st[k]);
                }
            }
        }
    }
}

}  // namespace tdse
