// Argument bundle shared by the host orchestrator (api.cpp) and the periodic
// kernels (periodic1d.cu, periodic2d.cu, tables.cu, noalloc.cu).  Plain data.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace tdse {

// What one launch sequence of the step operator computes.
enum Mode : int {
    MODE_STEP = 0,      // one step of eq. uadamsk (or eq. utrapkdisc): see step_common.cuh
    MODE_REFRESH = 1,   // R = DFT(V IDFT(u^)) -> ring[out]; state unchanged
    MODE_INIT = 2,      // u^ <- DFT(u0) (u0 parked in the state slot); ring[out] <- DFT(V u0)
    MODE_READ = 3       // out <- IDFT(u^)   (u^ = E_n v^ first when the state is in the interaction picture)
};

// Compute/storage precision combination of one kernel instantiation.
//   C  = transform type, RT = ring element type, ST = state element type.
enum Combo : int {
    COMBO_F64 = 0,      // C = double2, RT = double2, ST = double2  (FP64 mode)
    COMBO_F32 = 1,      // C = float2,  RT = float2,  ST = float4 double-float (mixed steps)
    COMBO_F64_R32 = 2   // C = double2, RT = float2,  ST = float4 (mixed-mode init / read-out)
};

constexpr int MAX_HIST = 7;
constexpr int E1D_NLO = 32;    // 1D absolute kinetic phase: e^{-i k^2 n dt} = Khi[n / 32] Klo[n % 32]

struct KArgs {
    int mode;
    int B;                    // instances in this launch
    int n0, n1;               // launch geometry: lines x line length (n1 = 1 for 1D); for 3D the
                              // column pass sees [n0][n1 n2] and the row pass [n0 n1][n2]
    int tn0, tn1, tn2;        // the grid per axis for the phase and E tables (tn2 = 0 below 3D)
    // 1D grid of N = n0 n1 points through the 2D passes (four-step transform):
    // grid point j = n0 c + r at [r][c] (the grid stored transposed), mode k at
    // [k / n1][k % n1] (natural FFT order); the row pass multiplies by the
    // twiddle e^{-+2 pi i r c / N} between its transform and the column pass's.
    // tn0 = N and the 1D phase tables apply to the flattened mode index.
    int flat1d;
    int shape1d;              // 1D one-CTA-per-instance kernels: 1 = the alternative launch shape
                              // (half the threads per instance, twice the points per thread)
    const double2* tw1d64;    // e^{-2 pi i m / N}, m < N
    const float2* tw1d32;
    // ---- step description
    int nhist;                // history terms j = 1..nhist
    double h;                 // step size
    double mu[MAX_HIST + 1];  // mu_0 .. mu_nhist
    float h_hi, h_lo;         // h split into two floats (double-float arithmetic)
    float hmu0_hi, hmu0_lo;   // h mu_0 split
    float mu_hi[MAX_HIST + 1], mu_lo[MAX_HIST + 1];
    int hist_slot[MAX_HIST];  // ring slot of lag j (index j-1)
    int out_slot;             // ring slot receiving the new (Vu)^
    int interval[MAX_HIST];   // interval id of the one-step phase p_i, i = 0..nhist-1
    int kin;                  // 1D kinetic table index (h = dt / 2^kin)
    int tf;                   // fine time index of the new time (t = tf * dt / 8)
    int ip;                   // 1: interaction-picture step (state v^ = u^ / E_n, ring r~ = z_n R / E_n)
    // interaction picture, mixed: the ring stores r~_n = z_n r^_n with a per-step
    // dither z_n (|z| ~ 1); the history uses c_j = mu_j / z_{n-j} and the update
    // d = h mu_0 / z_n, both split hi + lo (complex).
    float zr[2];              // z_n of the ring value written by this launch
    float c_hi[MAX_HIST + 1][2], c_lo[MAX_HIST + 1][2];
    float d_hi[2], d_lo[2];
    int e_step;               // n of E_n for an interaction-picture step / read-out
    int e_next;               // fused column pass: n of the next step's E
    // ---- state
    void* uhat;               // [B][NP] state (ST)
    void* ring;               // [B][ring_slots][NP] ring (RT)
    int ring_slots;
    double2* aux;             // 2D intermediate T1 (16 B per element)
    double2* aux2;            // 2D intermediate T2 / read-out output (16 B per element)
    // ---- problem tables
    const double* V0;         // instance b at V0 + b vstride: V(x, t_tf) on the grid (separable: V0(x))
    const float2* V0f;        // same layout (float(V), float(V - float(V)))
    size_t vstride;           // NP (separable) or rows x NP (potential table, V0 then points at this time's row)
    const double* tfac;       // [B][ntf]
    int ntf;
    int n_int;                // phase intervals per instance
    double dt;
    const double* phi;        // [B][d][ntf], phi at t = m dt / 8
    // 1D relative phases p(k) = kin[c][m] * adv[hi] * adv[lo]
    const double2* kin64;     // [L][N]
    const float4* kinff;
    const double2* adv64;     // [B][n_int][nh + nl]
    const float4* advff;
    int nh, nl, lb;
    // 2D relative phases p(k0,k1) = q[int][m0] * q[int][n0 + m1]
    const double2* q64;       // [B][n_int][n0 + n1]
    const float4* qff;
    // interaction-picture phases E_n(k) = exp(-i |k|^2 t_n + i k.phi(t_n)) in FP32
    const float2* e2d;        // [B][nsteps + 1][n0 + n1]   (2D: separable)
    const float2* k1d_lo;     // [E1D_NLO][N]               (1D: e^{-i k^2 n dt}, n < 32)
    const float2* k1d_hi;     // [nhi][N]                   (1D: e^{-i k^2 32 q dt})
    const float2* a1d;        // [B][nsteps + 1][nh + nl]   (1D: e^{i k phi(t_n)})
    // twiddles e^{-2 pi i m / n} for each axis length
    const double2* tw64_0;
    const double2* tw64_1;
    const float2* tw32_0;
    const float2* tw32_1;
    const float2* tw32lo_0;   // e^{-2 pi i m / n} - tw32 (rounding residual)
    const float2* tw32lo_1;
    const double2* tw64_2;    // axis 2 (3D)
    const float2* tw32_2;
    const float2* tw32lo_2;
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_periodic1d(const KArgs& a, int combo, cudaStream_t s);
// 2D: launch_periodic2d runs the whole mode (MODE_STEP: col_begin, row_mid,
// col_end); launch_periodic2d_part runs one pass kernel, which the host uses to
// chain consecutive Adams steps as col_begin, (row_mid, col_fused)..., row_mid, col_end.
cudaError_t launch_periodic2d(const KArgs& a, int combo, cudaStream_t s);
cudaError_t launch_periodic2d_part(const KArgs& a, int combo, int part, cudaStream_t s);
enum Part2D : int { PART_COL_BEGIN = 0, PART_ROW_MID = 1, PART_COL_END = 2, PART_COL_FUSED = 3 };
// 3D [n0][n1][n2] (a.tn0..tn2; a.n0/a.n1 ignored): the 2D column pass over the
// n1 n2 columns of axis 0, a transform pass along axis 1, and the 2D row pass
// over the n0 n1 rows of axis 2; the same parts as in 2D.
cudaError_t launch_periodic3d(const KArgs& a, int combo, cudaStream_t s);
cudaError_t launch_periodic3d_part(const KArgs& a, int combo, int part, cudaStream_t s);
bool periodic3d_supported(int n0, int n1, int n2);
bool periodic1d_supported(int n);
bool periodic2d_supported(int n0, int n1);
// One-time kernel attributes of the 1D step for n and combo (before stream capture).
cudaError_t periodic1d_prepare(int n, int combo);
// Threads per instance of the FP32 one-CTA-per-instance 1D kernel of n in
// launch shape `shape` (0 default, 1 alternative); 0 if that shape is not built.
int periodic1d_f32_threads(int n, int shape);

// ---- uneven 1D batches: one persistent launch for many contexts (mixed steps)
// A CTA of MULTI_CTA threads takes the next item from a global counter; an
// item runs `count` instances of one context with the launch variant `var`
// (N and T = threads per instance), count <= MULTI_CTA / T, side by side.
constexpr int MULTI_CTA = 512;
constexpr int MULTI_MAX_GROUPS = 16;
constexpr int MULTI_MAX_ITEMS = 1536;
struct MultiItem {
    unsigned char g;          // context (index into args)
    unsigned char var;        // launch variant (multi_variant_n / multi_variant_t)
    unsigned short count;     // instances in the item
    int b0;                   // first instance
};
struct MultiArgs1D {
    int nitems;
    int* next;                // work counter (zeroed before the launch): items are taken in order, as CTAs free up
    KArgs args[MULTI_MAX_GROUPS];
    MultiItem items[MULTI_MAX_ITEMS];
};
constexpr int MULTI_NVAR = 15;
int multi_variant_n(int var);
int multi_variant_t(int var);
int multi_variant(int n, int t);            // -1 if not built
size_t multi_item_smem(int var, int count);
cudaError_t multi_prepare(size_t smem);
int multi_occupancy(size_t smem);           // resident CTAs per SM (0 on error)
cudaError_t launch_periodic1d_multi(const MultiArgs1D& m, int grid, size_t smem, cudaStream_t s);
// FP64 residual check of the mixed implicit step (resid.cu).
struct ResArgs;
bool residual_supported(int dim, int n0, int n1);
cudaError_t launch_residual_check(const ResArgs& r, bool correct, cudaStream_t s);

// ---- 2D mixed Adams steps of 512^2 instances over CTA clusters (step2d_cluster.cu)
// One cluster of CL_Q CTAs per instance holds the transform intermediates in
// shared memory; a launch runs k consecutive interaction-picture steps
// (begin, (row, column) x (k - 1), row, end) of every instance.
constexpr int CL_N = 512;      // points per axis
constexpr int CL_Q = 16;       // CTAs per cluster
constexpr int CL_TAB = 36;     // floats per step in the weight table
// Weight table row m (floats): z_m (0, 1); d_m = h mu_0 / z_m hi (2, 3), lo (4, 5);
// c_j of the step m begun, mu_j / z_{m-j}: hi at 6 + 4 (j - 1) (2 floats), lo at 8 + 4 (j - 1).
struct ClArgs {
    int n_first;        // first step of the run
    int k;              // steps in the run (>= 1)
    int S_eff;          // start-up steps (row of V(t_n) in a potential table)
    int vrows;          // potential-table rows per instance (1: separable)
    int vtable, vshared;
    const float* tab;   // [nsteps + 1][CL_TAB]
    int* err;           // device error word (TDSE_ETIMEOUT if a bounded wait gave up)
};
struct ClPlan {
    alignas(64) unsigned char tm[3][128];   // TMA descriptors: state, ring, V hi/lo
    int clusters = 0;                        // clusters resident at once (0: path unavailable)
};
bool step2d_cluster_supported(int n0, int n1);
// Tensor maps over the context's buffers and the resident cluster count.
cudaError_t step2d_cluster_plan(ClPlan& p, void* uhat, void* ring, void* V0f, int B, int RS, long long vrows_total);
cudaError_t launch_step2d_cluster(const KArgs& a, const ClArgs& c, const ClPlan& p, cudaStream_t s);
int step2d_cluster_threads();
int step2d_cluster_smem();

// Largest n of the 1D FP32 step kernels (larger than periodic1d_supported's
// limit: FP64 init / read-out of such sizes go through launch_fft64_four_step).
constexpr int P1D_MAX_F32 = 16384;
int four_step_n();                                   // 128 * 128
cudaError_t launch_four_step_tables(double2* tw128, cudaStream_t s);
cudaError_t launch_four_step_init(const KArgs& a, const double2* tw128, cudaStream_t s);
cudaError_t launch_four_step_read(const KArgs& a, const double2* tw128, cudaStream_t s);

// Table builders (tables.cu).
cudaError_t launch_twiddles(double2* tw64, float2* tw32, float2* tw32lo, int n, cudaStream_t s);
cudaError_t launch_kin1d(double2* kin64, float4* kinff, int n, int L, double dt, cudaStream_t s);
cudaError_t launch_adv1d(double2* adv64, float4* advff, const int2* intervals, int n_int, const double* phi,
                         int ntf, int n, int nh, int nl, cudaStream_t s);
// 2D / 3D separable phase tables over the axes n0, n1 (and n2 > 0 for 3D): n0 + n1 + n2 entries per row
cudaError_t launch_q2d(double2* q64, float4* qff, const int2* intervals, int n_int, const double* phi, int ntf,
                       int n0, int n1, int n2, double dt, cudaStream_t s);
cudaError_t launch_e2d(float2* e, const double* phi, int ntf, int nsteps, int n0, int n1, int n2, double dt,
                       cudaStream_t s);
cudaError_t launch_k1d(float2* klo, float2* khi, int nhi, int n, double dt, cudaStream_t s);
cudaError_t launch_a1d(float2* a1d, const double* phi, int ntf, int nsteps, int n, int nh, int nl,
                       cudaStream_t s);
cudaError_t launch_split_float(float2* hilo, const double* src, size_t n, cudaStream_t s);
// 1D grids through the 2D passes: natural order (point j = n0 c + r) <-> the
// transposed layout [r][c] (r < n0, c < n1), B arrays of n0 n1 elements of
// elem_bytes (8 or 16); to_passes = 1: natural -> [r][c].
cudaError_t launch_transpose_1d(void* dst, const void* src, int n0, int n1, int B, int elem_bytes, int to_passes,
                                cudaStream_t s);
// phi(m dt/8), m = 0..ntf-1, of the built-in pulse in closed form into phi[d][ntf]
cudaError_t launch_pulse_phi(double* phi, int ntf, int d, double hs, double A0, double omega, double Tp,
                             const double* dir, cudaStream_t s);
// state <- sum_c coef[c] * chain[c] (chains laid out [L][n]); ff = state is double-float
cudaError_t launch_combine(void* state, const void* chains, size_t chain_stride, int L, const double* coef,
                           size_t n, bool ff, cudaStream_t s);
cudaError_t launch_copy_slot(void* dst, const void* ring, int ring_slots, int slot, int B, size_t NP,
                             size_t elem_bytes, cudaStream_t s);
// count non-finite doubles (ff = false) or floats (ff = true) in n 8-byte words
cudaError_t launch_count_nonfinite(const void* x, size_t nwords, bool ff, int* count, cudaStream_t s);
// Convert the double-float state at step n and the ring slots of steps
// slot_steps[0..nslots) to the interaction picture (divide by E in FP64).
cudaError_t launch_to_interaction(const KArgs& a, int n, const int* slot_steps, const float* slot_z, int nslots,
                                  cudaStream_t s);

}  // namespace tdse
