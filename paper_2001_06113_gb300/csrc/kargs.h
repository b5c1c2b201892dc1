// Argument bundle shared by the host orchestrator (api.cpp) and the periodic
// kernels (periodic1d.cu, periodic2d.cu, tables.cu).  Plain data only.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace tdse {

// What one launch sequence of the step operator computes.
enum Mode : int {
    MODE_STEP = 0,      // W = p0 (u^ - i h S1);  u = IDFT(W)/(1 + i h mu0 V);  R = DFT(V u);
                        // u^ <- W - i h mu0 R;  ring[out] <- R      (eq. uadamsk / utrapkdisc)
    MODE_REFRESH = 1,   // R = DFT(V IDFT(u^)) -> ring[out]; u^ unchanged
    MODE_INIT = 2,      // u^ <- DFT(u0) (u0 stored in u^'s buffer); ring[out] <- DFT(V u0)
    MODE_READ = 3       // out <- IDFT(u^)
};

// Compute/storage precision combination of one kernel instantiation.
enum Combo : int {
    COMBO_F64 = 0,      // transforms complex FP64, ring complex FP64
    COMBO_F32 = 1,      // transforms complex FP32, ring complex FP32
    COMBO_F64_R32 = 2   // transforms complex FP64, ring complex FP32 (mixed-mode init/read)
};

constexpr int MAX_HIST = 7;

struct KArgs {
    int mode;
    int B;                    // instances in this launch
    int n0, n1;               // grid (n1 = 1 for 1D)
    // step description
    int nhist;                // history terms j = 1..nhist
    double h;                 // step size
    double mu[MAX_HIST + 1];  // mu_0 .. mu_nhist
    int hist_slot[MAX_HIST];  // ring slot of lag j (index j-1)
    int out_slot;             // ring slot receiving the new (Vu)^
    int interval[MAX_HIST];   // interval id of the one-step phase p_i, i = 0..nhist-1
    int kin;                  // 1D kinetic table index (h = dt / 2^kin)
    int tf;                   // fine time index of the new time (t = tf * dt / 8)
    // state
    double2* uhat;            // [B][NP] FP64 modes (in/out)
    void* ring;               // [B][ring_slots][NP] ring (double2 or float2)
    int ring_slots;
    double2* aux;             // MODE_READ output / 2D intermediate T1 (16 B per element)
    double2* aux2;            // 2D intermediate T2 (16 B per element)
    // problem tables
    const double* V0;         // [B][NP]
    const float* V0f;         // [B][NP]
    const double* tfac;       // [B][ntf]
    int ntf;
    int n_int;                // number of phase intervals per instance
    // 1D phase tables: p(k) = kin[c][m] * adv_hi[m >> lb] * adv_lo[m & (nl-1)]
    const double2* kin64;     // [L][N]
    const float2* kin32;
    const double2* adv64;     // [B][n_int][nh + nl]
    const float2* adv32;
    int nh, nl, lb;
    // 2D phase tables: p(k0, k1) = q[int][m0] * q[int][n0 + m1]
    const double2* q64;       // [B][n_int][n0 + n1]
    const float2* q32;
    // twiddles e^{-2 pi i m / n} for each axis length
    const double2* tw64_0;
    const double2* tw64_1;
    const float2* tw32_0;
    const float2* tw32_1;
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_periodic1d(const KArgs& a, int combo, cudaStream_t s);
cudaError_t launch_periodic2d(const KArgs& a, int combo, cudaStream_t s);
bool periodic1d_supported(int n);
bool periodic2d_supported(int n0, int n1);

// Table builders (tables.cu).
cudaError_t launch_twiddles(double2* tw64, float2* tw32, int n, cudaStream_t s);
cudaError_t launch_kin1d(double2* kin64, float2* kin32, int n, int L, double dt, cudaStream_t s);
// intervals: [n_int] pairs (a, b) of fine time indices; phi: [B][d][ntf]
cudaError_t launch_adv1d(double2* adv64, float2* adv32, const int2* intervals, int n_int,
                         const double* phi, int ntf, int B, int n, int nh, int nl, cudaStream_t s);
cudaError_t launch_q2d(double2* q64, float2* q32, const int2* intervals, int n_int,
                       const double* phi, int ntf, int B, int n0, int n1, double dt, cudaStream_t s);
cudaError_t launch_to_float(float* dst, const double* src, size_t n, cudaStream_t s);
// u^ <- sum_c coef[c] * chain[c] (chains laid out [L][B*NP])
cudaError_t launch_combine(double2* uhat, const double2* chains, size_t chain_stride, int L,
                           const double* coef, size_t n, cudaStream_t s);
// copy ring slot src_slot of every instance into a 1-slot ring (same precision)
cudaError_t launch_copy_slot(void* dst, const void* ring, int ring_slots, int slot, int B,
                             size_t NP, size_t elem_bytes, cudaStream_t s);
// count non-finite entries of x[0..n) into *count (device int, accumulated)
cudaError_t launch_count_nonfinite(const double* x, size_t n, int* count, cudaStream_t s);

}  // namespace tdse
