// 2D periodic mixed-precision Adams steps (eq. uadamsk in the interaction
// picture, see step_common.cuh) of 512 x 512 instances, one instance per
// cluster of 16 CTAs, several consecutive steps per launch.
//
// Per step the method needs, per mode, the state and the history of (Vu)^ from
// HBM, and between them two 2D transforms whose intermediates (the grid values
// after the axis-0 transform, and (Vu) after the axis-1 transform) need not
// leave the chip.  The two-pass kernels of periodic2d.cu send those
// intermediates through global memory; here they stay in shared memory:
//
//   slab     each CTA q (0..15, 1024 threads) of the cluster holds 1/16 of
//            the instance, 512 x 32 complex FP32 (128 KB): the 32 columns
//            32q.. in the column phase, the 32 rows 32q.. in the row phase;
//   transpose between the phases every CTA pulls its new slab out of the
//            other CTAs' slabs through distributed shared memory
//            (ld.shared::cluster), straight into the registers of the first
//            FFT pass, and writes it locally once every CTA has finished
//            reading (cluster barrier);
//   streams  the mode state, the history slots and V reach shared memory by TMA
//            (cp.async.bulk.tensor, completion on an mbarrier) in a 3-stage
//            pipeline of 32 KB stages that runs ahead across phases and steps;
//            the state and the new history slot go back with coalesced stores.
//
// One step of one instance (n = the step being finished):
//   column phase: gather the axis-1 transform of (Vu) (row slabs) -> forward
//      DFT along axis 0 (1/n0) = R = (Vu)^; per mode (16-row chunks): r~ =
//      z_n R / E_n into the history ring, v^_n = X_n - i d r~, then the next
//      step's X_{n+1} = v^_n - i h sum_j c_j r~_{n+1-j} into the state, and
//      E_{n+1} X_{n+1} into the slab -> inverse DFT along axis 0;
//   row phase (step n+1): gather -> inverse DFT along axis 1 -> u = y / (1 +
//      i h mu_0 V), V u (V by 8-row TMA chunks) -> forward DFT along axis 1
//      (1/n1).
// A run of k steps is begin(n+1), (row, column) x (k - 1), row, end(n+k),
// where begin forms X from the state and all history lags and end only updates
// the state.  The arithmetic is the same, operation for operation, as the
// two-pass kernels' (k_col_begin, k_row_mid, k_col_fused_ip, k_col_end), so
// both paths give the same bits.
//
// Shared memory layout of a slab: element (position p along the transformed
// axis, line l) at p * 32 + (l ^ g(p)), g(p) = (p ^ (p >> 4)) & 31; lines are
// the 32 columns (rows) a CTA owns.  The transform passes run one butterfly
// position across the 32 lines of a warp, pass 0 and the V product run 32
// positions of one line, and a remote gather reads the 32 lines of one
// position: with this swizzle none of these patterns has bank conflicts.
//
// Waits: every mbarrier wait is bounded; a wait that gives up records
// TDSE_ETIMEOUT in the error word, and the CTA runs on without waiting
// (results are then invalid, but every CTA reaches every cluster barrier, so
// the launch ends).  Before it exits, the CTA waits (bounded) for its last
// copies.  Distributed shared memory is only read between cluster barriers
// that every CTA of the cluster passes.
#include <cuda.h>

#include "step_common.cuh"
#include "tdse.h"

namespace tdse {
namespace cl2d {

constexpr int N = CL_N;                  // points per axis
constexpr int Q = CL_Q;                  // CTAs per cluster
constexpr int W = N / Q;                 // lines per CTA (32)
constexpr int T = 1024;                  // threads per CTA
constexpr int NB = N / 8;                // butterflies per line in a radix-8 pass
constexpr int PER = NB * W / T;          // butterflies per thread per pass (4)
constexpr int STAGES = 3;
constexpr int STAGE_BYTES = 32768;
constexpr int SLAB_BYTES = N * W * 8;    // 131072
constexpr int BAR_OFF = SLAB_BYTES + STAGES * STAGE_BYTES;
constexpr int WT_OFF = BAR_OFF + 64;     // per-step weights of the current phase
constexpr int SMEM_BYTES = WT_OFF + 2 * CL_TAB * 4;
static_assert(W == 32, "slab layout assumes 32 lines per CTA");
static_assert(PER * T == NB * W, "whole butterflies per thread");
static_assert(PER == 2, "two butterflies per thread and pass");
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");

// Loads of the per-instance sequence: BEGIN chunks of 8 rows, then per step
// 4 V chunks of 8 rows and 32 FUSED (or, in the last step, END) chunks of
// 16 rows.
constexpr int NBEGIN = N / 8;            // 64
constexpr int NVCH = W / 8;              // 4
constexpr int NCOL = N / 16;             // 32
constexpr int PER_STEP = NVCH + NCOL;    // 36
enum LoadKind { L_BEGIN = 0, L_V = 1, L_FUSED = 2, L_END = 3 };

constexpr unsigned long long WAIT_LIMIT = 1ull << 26;   // polls, with back-off: seconds

// --------------------------------------------------------------- PTX helpers
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned cta_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_index() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_count() {
    unsigned r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned map_rank(unsigned saddr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster(unsigned addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of phase `parity`; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (unsigned long long it = 0; it < WAIT_LIMIT; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (it > 16) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void tma2d(unsigned dst, const CUtensorMap* tm, int x, int y, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma3d(unsigned dst, const CUtensorMap* tm, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
// Order this thread's earlier global stores before later TMA (async-proxy) reads.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

__device__ __forceinline__ constexpr int swz(int p) { return (p & 31) ^ ((p >> 6) & 7) ^ (((p >> 4) & 1) << 3); }
__device__ __forceinline__ int sidx(int p, int l) { return p * W + (l ^ swz(p)); }
// Position p = item + c r with item and c r on disjoint bits (the positions of
// one butterfly): swz is XOR-linear, so the eight indices are one base index,
// an XOR with a constant and an offset.
__device__ __forceinline__ int sidx_base(int item, int l) { return item * W + (l ^ swz(item)); }
template <int C>
__device__ __forceinline__ int sidx_at(int base, int r) { return (base ^ swz(C * r)) + W * C * r; }
// digit reversal of a 512-point index in base 8 (the order in which an
// in-place transform leaves its result)
__device__ __forceinline__ int rev8(int m) { return 64 * (m & 7) + 8 * ((m >> 3) & 7) + (m >> 6); }

struct Params {
    KArgs a;
    ClArgs c;
};

__device__ __forceinline__ int ring_slot(int n, int RS) { return ((n % RS) + RS) % RS; }

// Row of the potential table holding V(t_n) (one row per Adams step after the
// 8 S + 1 rows of the start-up's fine times).
__device__ __forceinline__ long long vrow_of(const ClArgs& c, int n) {
    if (!c.vtable) return 0;
    const int tf = 8 * n, fine = 8 * c.S_eff;
    return tf <= fine ? tf : fine + (n - c.S_eff);
}

struct LoadDesc {
    int kind, b, n, chunk;
};
__device__ __forceinline__ LoadDesc decode(const ClArgs& c, int i) {
    const int per_inst = NBEGIN + PER_STEP * c.k;
    const int ii = i / per_inst;
    int w = i - ii * per_inst;
    LoadDesc d;
    d.b = (int)cluster_index() + ii * (int)cluster_count();
    if (w < NBEGIN) {
        d.kind = L_BEGIN;
        d.n = c.n_first;
        d.chunk = w;
        return d;
    }
    w -= NBEGIN;
    const int s = w / PER_STEP, u = w - s * PER_STEP;
    d.n = c.n_first + s;
    if (u < NVCH) {
        d.kind = L_V;
        d.chunk = u;
    } else {
        d.kind = s + 1 < c.k ? L_FUSED : L_END;
        d.chunk = u - NVCH;
    }
    return d;
}

// Issue load i of this CTA's sequence into its stage (one thread).
__device__ void issue_load(const Params& P, const CUtensorMap* tm_st, const CUtensorMap* tm_ring,
                           const CUtensorMap* tm_v, unsigned char* smem, int i, int q) {
    const KArgs& a = P.a;
    const ClArgs& c = P.c;
    const LoadDesc d = decode(c, i);
    const int stg = i % STAGES;
    const unsigned dst = smem_u32(smem + SLAB_BYTES + stg * STAGE_BYTES);
    const unsigned bar = smem_u32(smem + BAR_OFF + 8 * stg);
    const int RS = a.ring_slots;
    const int nh = a.nhist;
    if (d.kind == L_BEGIN) {
        mbar_expect_tx(bar, 4096 + nh * 2048);
        const int row = d.b * N + 8 * d.chunk;
        tma2d(dst, tm_st, q * 128, row, bar);
        for (int j = 1; j <= nh; ++j) {
            const int slot = ring_slot(d.n - j, RS);
            tma2d(dst + 4096 + (j - 1) * 2048, tm_ring, q * 64, (d.b * RS + slot) * N + 8 * d.chunk, bar);
        }
    } else if (d.kind == L_V) {
        mbar_expect_tx(bar, 32768);
        const long long base = (long long)(c.vshared ? 0 : d.b) * c.vrows * N + vrow_of(c, d.n) * N;
        tma3d(dst, tm_v, 0, 0, (int)(base + q * W + 8 * d.chunk), bar);
    } else {
        const int nl = d.kind == L_FUSED ? nh - 1 : 0;
        mbar_expect_tx(bar, 8192 + nl * 4096);
        const int row = d.b * N + 16 * d.chunk;
        tma2d(dst, tm_st, q * 128, row, bar);
        tma2d(dst + 4096, tm_st, q * 128, row + 8, bar);
        for (int j = 2; j <= nl + 1; ++j) {          // lags 2..nhist of step n + 1
            const int slot = ring_slot(d.n + 1 - j, RS);
            const unsigned o = dst + 8192 + (j - 2) * 4096;
            const int y = (d.b * RS + slot) * N + 16 * d.chunk;
            tma2d(o, tm_ring, q * 64, y, bar);
            tma2d(o + 2048, tm_ring, q * 64, y + 8, bar);
        }
    }
}

// --------------------------------------------------------------- transforms
// The 32 interleaved length-512 transforms run as three radix-8 passes with
// the butterflies of CtaFft (pass s: butterfly j takes logical positions
// j + 64 r, twiddles them by tw[k r N / (8 Ns)], k = j mod Ns, Ns = 8^s, and
// gives logical positions (j - k) 8 + k + r Ns), but every butterfly writes
// its outputs back into the slots it read.  The logical order then moves
// through base-8 digit permutations of the physical position:
//   from natural order (Q = id):   pass 1 at 64 jl + 8 r + jh, pass 2 at
//     64 jl + 8 jh + r, result in digit-reversed order;
//   from digit-reversed order (Q = rev): pass 0 at 64 jl + 8 jh + r, pass 1
//     at 64 jh + 8 r + jl, pass 2 at j + 64 r, result in natural order
// (j = 8 jh + jl).  Each slot belongs to one butterfly per pass, so a pass
// needs one barrier (after it) and a thread holds one butterfly at a time;
// the values and the arithmetic of every butterfly are those of CtaFft.
// Threads: lanes of a warp are the 32 lines, warp w takes j = w and w + 32.

template <bool INV, int S>
__device__ __forceinline__ void butterfly_math(float2 (&v)[8], int j, const float2* __restrict__ tw) {
    using Plan = FftPlan<N, INV>;
    static_assert(Plan::NPASS == 3 && Plan::radix(S) == 8, "512 = 8 x 8 x 8");
    constexpr int Ns = Plan::ns(S);
    constexpr int stride = N / (Ns * 8);
    if (Ns > 1) {
        const int k = j & (Ns - 1);
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = twiddle<INV>(v[r], tw, tw, k * r * stride);
    }
    dft8<INV>(v);
}

// One in-place pass.  QREV: the transform started from digit-reversed order.
// SCALE: outputs multiplied by `scale` as they are stored.
template <bool INV, int S, bool QREV, bool SCALE>
__device__ __forceinline__ void inplace_pass(float2* slab, const float2* __restrict__ tw, float scale) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int j = warp + 32 * p, jh = j >> 3, jl = j & 7;
        // item part and the stride of r in the physical position
        constexpr int C = !QREV ? (S == 1 ? 8 : 1) : (S == 0 ? 1 : (S == 1 ? 8 : 64));
        const int item = !QREV ? (S == 1 ? 64 * jl + jh : 64 * jl + 8 * jh)
                               : (S == 0 ? 64 * jl + 8 * jh : (S == 1 ? 64 * jh + jl : j));
        const int sb = sidx_base(item, lane);
        float2 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = slab[sidx_at<C>(sb, r)];
        butterfly_math<INV, S>(v, j, tw);
#pragma unroll
        for (int r = 0; r < 8; ++r) slab[sidx_at<C>(sb, r)] = SCALE ? cscale(v[r], scale) : v[r];
    }
    __syncthreads();
}

// Whole transform of data in digit-reversed order; result in natural order.
template <bool INV, bool SCALE_LAST>
__device__ __forceinline__ void transform_from_rev(float2* slab, const float2* __restrict__ tw, float scale) {
    inplace_pass<INV, 0, true, false>(slab, tw, 1.f);
    inplace_pass<INV, 1, true, false>(slab, tw, 1.f);
    inplace_pass<INV, 2, true, SCALE_LAST>(slab, tw, scale);
}

// Pull this thread's pass-0 inputs of the other orientation out of the
// cluster's slabs (which hold their lines in natural order): position pos of
// line L = q W + line of the new orientation is element (L, pos & 31) of the
// slab of CTA pos / 32.  For the gather the lanes of a warp take consecutive
// butterflies of one line (warp w: line w, j = lane + 32 x), so that each load
// of a warp reads one whole 256-byte line-run of one remote slab.
__device__ __forceinline__ void gather(float2 (&v)[PER][8], unsigned slab_s, int q) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned base = slab_s + (unsigned)sidx(q * W + warp, lane) * 8u;
#pragma unroll
    for (int x = 0; x < PER; ++x) {
#pragma unroll
        for (int r = 0; r < 8; ++r) v[x][r] = ld_cluster(map_rank(base, (unsigned)(x + 2 * r)));
    }
}

// Transpose + transform: gather from the other CTAs, pass-0 butterflies while
// the cluster barrier (every CTA done reading) completes, pass-0 results into
// the local slab (at positions j + 64 r), passes 1 and 2 in place.  Result in
// digit-reversed order.
template <bool INV>
__device__ __forceinline__ void gather_transform(float2* slab, unsigned slab_s, int q, const float2* __restrict__ tw) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2 v[PER][8];
    gather(v, slab_s, q);
    cluster_arrive();
#pragma unroll
    for (int x = 0; x < PER; ++x) dft8<INV>(v[x]);
    cluster_wait();
#pragma unroll
    for (int x = 0; x < PER; ++x) {
        const int sb = sidx_base(lane + 32 * x, warp);
#pragma unroll
        for (int r = 0; r < 8; ++r) slab[sidx_at<64>(sb, r)] = v[x][r];
    }
    __syncthreads();
    inplace_pass<INV, 1, false, false>(slab, tw, 1.f);
    inplace_pass<INV, 2, false, false>(slab, tw, 1.f);
}

// ------------------------------------------------------ per-mode arithmetic
// v^ = X - i d r~ (ip_update with d = wd[0..1] hi, wd[2..3] lo)
__device__ __forceinline__ float4 ip_update_w(const float* wd, float4 X, float2 qv) {
    float px = fmaf(wd[2], qv.x, -wd[3] * qv.y);
    float py = fmaf(wd[2], qv.y, wd[3] * qv.x);
    px = fmaf(wd[0], qv.x, fmaf(-wd[1], qv.y, px));
    py = fmaf(wd[0], qv.y, fmaf(wd[1], qv.x, py));
    return ffc_add_f(X, py, -px);
}
// S += c_j q (c_j = wc[0..1] hi, wc[2..3] lo), the order of history_sum_ip
__device__ __forceinline__ void hist_term(float2& S, const float* wc, float2 qv) {
    const float ch = wc[0], cih = wc[1], cl = wc[2], cil = wc[3];
    S.x = fmaf(cl, qv.x, fmaf(-cil, qv.y, S.x));
    S.y = fmaf(cl, qv.y, fmaf(cil, qv.x, S.y));
    S.x = fmaf(ch, qv.x, fmaf(-cih, qv.y, S.x));
    S.y = fmaf(ch, qv.y, fmaf(cih, qv.x, S.y));
}

// ------------------------------------------------------------------ kernel
__global__ void __launch_bounds__(T, 1)
    k_step2d_cluster(const __grid_constant__ Params P, const __grid_constant__ CUtensorMap tm_st,
                     const __grid_constant__ CUtensorMap tm_ring, const __grid_constant__ CUtensorMap tm_v) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float2* slab = reinterpret_cast<float2*>(smem);
    float* wt = reinterpret_cast<float*>(smem + WT_OFF);
    const KArgs& a = P.a;
    const ClArgs& c = P.c;
    const int q = (int)cta_rank();
    const int tid = threadIdx.x, lane = tid & 31;
    const unsigned slab_s = smem_u32(slab);
    const unsigned bar0 = smem_u32(smem + BAR_OFF);
    const int G = (int)cluster_count(), g = (int)cluster_index();
    const int ninst = g < a.B ? (a.B - g + G - 1) / G : 0;
    const int total = ninst * (NBEGIN + PER_STEP * c.k);
    int next = 0, issued = 0;
    bool bad = false;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (; issued < STAGES && issued < total; ++issued) issue_load(P, &tm_st, &tm_ring, &tm_v, smem, issued, q);

    // wait for the next load of the sequence; its stage
    auto acquire = [&]() -> const unsigned char* {
        const int stg = next % STAGES;
        if (!bad && !mbar_wait(bar0 + 8 * stg, (unsigned)((next / STAGES) & 1))) {
            bad = true;
            atomicExch(c.err, (int)TDSE_ETIMEOUT);
        }
        return smem + SLAB_BYTES + stg * STAGE_BYTES;
    };
    // every thread is done with the current load: its stage takes load next + STAGES
    auto release = [&]() {
        __syncthreads();
        ++next;
        if (tid == 0 && issued < total) {
            issue_load(P, &tm_st, &tm_ring, &tm_v, smem, issued, q);
            ++issued;
        }
    };
    // per-step weights: row n (z_n, d_n) at wt[0..], row m (c_j of step m) at wt[CL_TAB..]
    auto load_weights = [&](int n, int m) {
        __syncthreads();
        if (tid < CL_TAB) {
            wt[tid] = c.tab[(size_t)n * CL_TAB + tid];
            wt[CL_TAB + tid] = c.tab[(size_t)m * CL_TAB + tid];
        }
        __syncthreads();
    };
    const float* wn = wt;
    const float* wm = wt + CL_TAB;
    const float scale = 1.0f / (float)N;
    const float hmu0 = (float)(a.h * a.mu[0]);
    const size_t NP = (size_t)N * N;
    const int m1 = q * W + lane;             // this thread's column in the column phase

#pragma unroll 1
    for (int ii = 0; ii < ninst; ++ii) {
        const int b = g + ii * G;
        float4* st = reinterpret_cast<float4*>(a.uhat) + (size_t)b * NP;
        float2* ringb = reinterpret_cast<float2*>(a.ring) + (size_t)b * a.ring_slots * NP;

        // ---- begin of step n_first: X = v^ - i h sum_j c_j r~_{n-j}; slab <- E_n X
        load_weights(c.n_first, c.n_first);
#pragma unroll 1
        for (int ch = 0; ch < NBEGIN; ++ch) {
            const unsigned char* sg = acquire();
            if (tid < 8 * W) {
                const int r = tid >> 5;
                const int m0 = 8 * ch + r;
                const float4 v = reinterpret_cast<const float4*>(sg)[r * W + lane];
                float2 S = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = MAX_HIST; j >= 1; --j) {
                    const float2 qv = j > a.nhist
                                          ? make_float2(0.f, 0.f)
                                          : reinterpret_cast<const float2*>(sg + 4096 + (j - 1) * 2048)[r * W + lane];
                    hist_term(S, wm + 6 + 4 * (j - 1), qv);
                }
                const float4 X = ff_minus_i_times(v, a.h_hi, a.h_lo, S);
                st[(size_t)m0 * N + m1] = X;
                slab[sidx(rev8(m0), lane)] = cmul(e_2d(a, b, c.n_first, m0, m1), make_float2(X.x, X.y));
            }
            if (ch == NBEGIN - 1) fence_proxy_async_global();
            release();
        }
        transform_from_rev<true, false>(slab, a.tw32_0, 1.f);
        cluster_arrive();
        cluster_wait();

#pragma unroll 1
        for (int s = 0; s < c.k; ++s) {
            const int n = c.n_first + s;
            // ---- row phase of step n: inverse along axis 1, u = y / (1 + i h mu_0 V), V u, forward along axis 1
            gather_transform<true>(slab, slab_s, q, a.tw32_1);
            {
                const double vfac = a.tfac[(size_t)b * a.ntf + (size_t)8 * n];
                const float fh = (float)vfac, fl = (float)(vfac - (double)fh);
                const int mcol = tid & (N - 1), pcol = rev8(mcol);
#pragma unroll 1
                for (int u = 0; u < NVCH; ++u) {
                    const float2* Vs = reinterpret_cast<const float2*>(acquire());
#pragma unroll
                    for (int i = 0; i < 8 * N / T; ++i) {
                        const int rr = (tid >> 9) + (T / N) * i;        // row within the 8-row chunk
                        const float2 v2 = Vs[rr * N + mcol];
                        const float vh = fh * v2.x;
                        const float vl = fmaf(fh, v2.x, -vh) + fmaf(fh, v2.y, fl * v2.x);
                        float2& y = slab[sidx(pcol, 8 * u + rr)];
                        y = implicit_solve_times_V(y, vh, vl, hmu0);
                    }
                    release();
                }
            }
            transform_from_rev<false, true>(slab, a.tw32_1, scale);
            cluster_arrive();
            cluster_wait();

            // ---- column phase: forward along axis 0 -> R; end of step n (and begin of step n + 1)
            gather_transform<false>(slab, slab_s, q, a.tw32_0);
            const bool fused = s + 1 < c.k;
            load_weights(n, fused ? n + 1 : n);
            const int out_slot = ring_slot(n, a.ring_slots);
#pragma unroll 1
            for (int ch = 0; ch < NCOL; ++ch) {
                const unsigned char* sg = acquire();
                if (tid < 16 * W) {
                const int r = tid >> 5;
                const int m0 = 16 * ch + r;
                const size_t idx = (size_t)m0 * N + m1;
                const int sp = sidx(rev8(m0), lane);
                const float2 R = cscale(slab[sp], scale);
                const float2 z = make_float2(wn[0], wn[1]);
                const float2 rv = cmul(z, cmul(conjf2(e_2d(a, b, n, m0, m1)), R));
                ringb[(size_t)out_slot * NP + idx] = rv;
                const float4 v = ip_update_w(wn + 2, reinterpret_cast<const float4*>(sg)[r * W + lane], rv);
                if (fused) {
                    float2 S = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = MAX_HIST; j >= 1; --j) {
                        const float2 qv =
                            j > a.nhist ? make_float2(0.f, 0.f)
                                        : (j == 1 ? rv
                                                  : reinterpret_cast<const float2*>(sg + 8192 + (j - 2) * 4096)[r * W + lane]);
                        hist_term(S, wm + 6 + 4 * (j - 1), qv);
                    }
                    const float4 X = ff_minus_i_times(v, a.h_hi, a.h_lo, S);
                    st[idx] = X;
                    slab[sp] = cmul(e_2d(a, b, n + 1, m0, m1), make_float2(X.x, X.y));
                } else {
                    st[idx] = v;
                }
                }
                if (ch == NCOL - 1) fence_proxy_async_global();
                release();
            }
            if (fused) {
                transform_from_rev<true, false>(slab, a.tw32_0, 1.f);
                cluster_arrive();
                cluster_wait();
            }
        }
    }
    // copies still in flight only if a wait gave up: wait (bounded) for them before exiting
    if (tid == 0 && bad)
        for (int i = issued - STAGES < 0 ? 0 : issued - STAGES; i < issued; ++i)
            (void)mbar_wait(bar0 + 8 * (i % STAGES), (unsigned)((i / STAGES) & 1));
}

}  // namespace cl2d

// ---------------------------------------------------------------- host side
namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    }
    return fn;
}

// FP32 tensor of `rank` dimensions (dims[0] innermost, byte strides of the
// outer dimensions), box `box`.
bool encode(void* out, void* base, int rank, const cuuint64_t* dims, const cuuint64_t* strides,
            const cuuint32_t* box) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, base, dims,
              strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaLaunchConfig_t make_config(int clusters, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(clusters * cl2d::Q), 1, 1);
    cfg.blockDim = dim3(cl2d::T, 1, 1);
    cfg.dynamicSmemBytes = cl2d::SMEM_BYTES;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl2d::Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t kernel_attributes() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(cl2d::k_step2d_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         cl2d::SMEM_BYTES);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(cl2d::k_step2d_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) done = true;
    return e;
}
}  // namespace

bool step2d_cluster_supported(int n0, int n1) { return n0 == CL_N && n1 == CL_N; }
int step2d_cluster_threads() { return cl2d::T; }
int step2d_cluster_smem() { return cl2d::SMEM_BYTES; }

cudaError_t step2d_cluster_plan(ClPlan& p, void* uhat, void* ring, void* V0f, int B, int RS, long long vrows_total) {
    p.clusters = 0;
    cudaError_t e = kernel_attributes();
    if (e != cudaSuccess) return e;
    const int N = CL_N;
    {   // state: FP32 [B n0][4 n1] (double-float complex = 4 floats per mode)
        const cuuint64_t d[2] = {(cuuint64_t)4 * N, (cuuint64_t)B * N};
        const cuuint64_t st[1] = {(cuuint64_t)4 * N * 4};
        const cuuint32_t box[2] = {4 * cl2d::W, 8};
        if (!encode(p.tm[0], uhat, 2, d, st, box)) return cudaErrorInvalidValue;
    }
    {   // ring: FP32 [B RS n0][2 n1]
        const cuuint64_t d[2] = {(cuuint64_t)2 * N, (cuuint64_t)B * RS * N};
        const cuuint64_t st[1] = {(cuuint64_t)2 * N * 4};
        const cuuint32_t box[2] = {2 * cl2d::W, 8};
        if (!encode(p.tm[1], ring, 2, d, st, box)) return cudaErrorInvalidValue;
    }
    {   // V hi/lo: FP32 [rows][4][256] (a row of n1 float2 = 1024 floats), box = 8 rows
        const cuuint64_t d[3] = {256, (cuuint64_t)(2 * N / 256), (cuuint64_t)vrows_total};
        const cuuint64_t st[2] = {256 * 4, (cuuint64_t)2 * N * 4};
        const cuuint32_t box[3] = {256, (cuuint32_t)(2 * N / 256), 8};
        if (!encode(p.tm[2], V0f, 3, d, st, box)) return cudaErrorInvalidValue;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = make_config(1, nullptr, attr);
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, cl2d::k_step2d_cluster, &cfg);
    if (e != cudaSuccess) return e;
    p.clusters = n;
    return cudaSuccess;
}

cudaError_t launch_step2d_cluster(const KArgs& a, const ClArgs& c, const ClPlan& p, cudaStream_t s) {
    if (p.clusters < 1 || c.k < 1 || a.n0 != CL_N || a.n1 != CL_N || a.nhist < 1 || a.nhist > MAX_HIST)
        return cudaErrorInvalidValue;
    cudaError_t e = kernel_attributes();
    if (e != cudaSuccess) return e;
    cl2d::Params P;
    P.a = a;
    P.c = c;
    const int clusters = a.B < p.clusters ? a.B : p.clusters;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = make_config(clusters, s, attr);
    const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(p.tm[0]);
    return cudaLaunchKernelEx(&cfg, cl2d::k_step2d_cluster, P, tm[0], tm[1], tm[2]);
}

}  // namespace tdse
