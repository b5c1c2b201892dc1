// Argument bundle of the free-space (complex contour) kernels, freespace.cu,
// shared with the host orchestrator fs_api.cpp.  Plain data.
//
// Free-space discretisation (Sec. 3.3-3.4, 4.1), one axis:
//   grid     x_j = -1 + 2 j / M, j = 0..M-1;
//   modes    zeta_m on the contour Gamma in the block order
//            E1 (NE equispaced, Gamma_1), A1 (p Alpert), C (Gauss panels on
//            Gamma_2), A3 (p Alpert), E3 (NE equispaced, Gamma_3), N in all;
//            the middle ND = 2p + NC modes are the "dense" block;
//   forward  f^_m = (2/M) sum_j e^{-i zeta_m x_j} f_j                  (eq. fzdft)
//   inverse  f_j  = (1/2pi) sum_m w_m e^{i zeta_m x_j} f^_m            (eq. uciftdisc)
// In 2D and 3D both are tensor products over the axes (row-major arrays, the
// last axis contiguous).
//
// An equispaced block has zeta_i = zeta0 + i h, i = 0..NE-1, weight h, with
// h = pi M / nu, so e^{i i h x_j} = e^{-i i h} e^{2 pi i i j / nu}: its sums are
// length-nu DFTs with NE nonzero inputs (inverse) or M nonzero inputs
// (forward), evaluated at M (resp. NE) points (eq. ssfftgen).  With nu = R M
// and i = s + R q each is R interleaved M-point FFTs plus a twiddle
// e^{+-2 pi i j s / nu}; the tables below fold that twiddle into the block's
// pre/post factors.
#pragma once
#include <cuda_runtime.h>

namespace tdse {

constexpr int FS_T = 256;         // threads per CTA of every free-space kernel
constexpr int FS_MAX_ND = 128;    // dense (Alpert + Gauss) modes per axis
constexpr int FS_MAX_HIST = 7;
constexpr int FS_MAX_NT = 64;     // terms of the Chebyshev interpolant of the C-type transforms

struct FsAxis {
    int M;        // physical points
    int R;        // nu / M
    int nu;       // equispaced FFT length
    int NE;       // modes per equispaced block
    int ND;       // dense modes (A1, C, A3)
    int N;        // all modes: 2 NE + ND
    const double2* preI;   // [2][NE]    inverse, block b: (h / 2pi) e^{-i i h}
    const double2* postI;  // [2][M][R]  inverse: e^{i zeta0_b x_j} e^{+2 pi i j s / nu}
    const double2* preF;   // [2][M][R]  forward: (2/M) e^{-i zeta0_b x_j} e^{-2 pi i j s / nu}
    const double2* postF;  // [2][NE]    forward: e^{+i i h}
    const double2* Gd;     // [ND][M]    inverse dense: (w_d / 2pi) e^{i zeta_d x_j}
    const double2* Fd;     // [ND][M]    forward dense: (2/M) e^{-i zeta_d x_j}
    const double2* tw;     // [M]        e^{-2 pi i m / M}
    const double2* P;      // [B][n_int][N] one-step phases e^{-i zeta^2 s + i zeta (phi(t1) - phi(t0))}
    // FP32 copies for the FP32-transform variant (TDSE_MIXED), same layouts
    const float2* preI_f;
    const float2* postI_f;
    const float2* preF_f;
    const float2* postF_f;
    const float2* Gd_f;
    const float2* Fd_f;
    const float2* tw_f;
    const float2* P_f;
    // C-type transforms by Chebyshev interpolation in tau on Gamma_2 (Sec. 4.1,
    // eqs. expintrpm, expintrpp): with zeta = (1 - i) tau, tau in [-H, H],
    //   e^{-i zeta x} = e^{-(1+i) tau x} ~ sum_l lambda_l(x) T_l(tau / H),
    //   e^{+i zeta x} = e^{+(1+i) tau x} ~ sum_l rho_l(x) T_l(tau / H),
    // the NC Gauss rows of the dense block become
    //   forward  f^_k = sum_l T_l(tau_k / H) [sum_j (2/M) lambda_l(x_j) f_j]
    //   inverse  f_j += sum_l rho_l(x_j) [sum_k T_l(tau_k / H) (w_k / 2pi) f^_k]
    // at O(NT (M + NC)) instead of O(NC M).  NT = 0: direct sums (Gd, Fd rows).
    int p;                 // Alpert modes per side: the C rows are dd = p .. p + NC - 1
    int NC;                // Gauss (C) modes
    int NT;                // interpolant terms, 0 = C rows by direct sums
    const double2* Lf;     // [NT][M]  (2/M) lambda_l(x_j)
    const double2* Li;     // [NT][M]  rho_l(x_j)
    const double* Tc;      // [NC][NT] T_l(tau_k / H)
    const double2* TcW;    // [NT][NC] T_l(tau_k / H) w_k / 2pi
    const float2* Lf_f;
    const float2* Li_f;
    const float* Tc_f;
    const float2* TcW_f;
};

struct FsArgs {
    int B;                 // instances in the launch
    int d;                 // 1, 2 or 3
    FsAxis ax[3];
    int n_int;             // phase intervals per instance
    // ---- step description (eq. uadamsk with zeta for k; eq. utrapzfd for nhist = 1)
    int nhist;             // history terms j = 1..nhist
    double h;              // step size
    double mu[FS_MAX_HIST + 1];
    int hist_slot[FS_MAX_HIST];   // ring slot of lag j (index j-1)
    int out_slot;          // ring slot receiving the new (Vu)^
    int interval[FS_MAX_HIST];    // interval id of the one-step phase p_i, i = 0..nhist-1
    int tf;                // fine time index of the new time (t = tf dt / 8)
    // ---- buffers
    double2* uhat;         // [B][N0 N1] mode state: u^ between steps, W inside a step (FP64 in both variants)
    double2* ring;         // [B][ring_slots][N0 N1] history of (Vu)^ (elements of the transform type)
    int ring_slots;
    double2* Z;            // 2D: [B][N0][M1]; 3D: [B][N0][N1][M2] (last axis on the grid; transform type)
    double2* Y;            // 3D: [B][N0][M1][M2] (axes 1 and 2 on the grid; transform type)
    double2* u;            // [B][M0 M1] physical state written by the implicit solve
    const double2* usrc;   // forward-only source on the grid
    double2* fdst;         // forward-only destination in mode space, instance b at fdst + b fdst_bstride
    size_t fdst_bstride;
    int fdst_ring;         // destination is a ring slot (transform type) rather than the FP64 state
    int mulV;              // forward-only: transform V(t) usrc instead of usrc
    const double* V0;      // instance b at V0 + b vstride (separable: [B][M0 M1]; table: this time's row)
    size_t vstride;
    const double* tfac;    // [B][ntf]
    int ntf;
};

// Row pass flags (2D, 3D), 1D modes, directions of the 3D axis-1 pass.
enum FsRow : int { FS_ROW_END = 1, FS_ROW_BEGIN = 2, FS_ROW_FWD_ONLY = 4 };
enum Fs1D : int { FS_1D_STEP = 0, FS_1D_FWD_ONLY = 1 };
enum FsMid : int { FS_MID_INV = 0, FS_MID_FWD = 1 };

bool fs_supported(int M, int R);
// 2D: row pass over the N0 mode rows (last axis, Z), phys pass over the M1
// grid columns (axis 0, Z).  3D: row pass over the N0 N1 mode rows (axis 2,
// Z), axis-1 pass between Z and Y over the N0 M2 lines, phys pass over the
// M1 M2 grid columns (axis 0, Y).  f32 = 1 selects the FP32-transform
// kernels (freespace_f32.cu).
cudaError_t launch_fs_row(const FsArgs& a, int flags, int f32, cudaStream_t s);
cudaError_t launch_fs_phys(const FsArgs& a, int from_usrc, int f32, cudaStream_t s);
cudaError_t launch_fs_mid(const FsArgs& a, int dir, int f32, cudaStream_t s);
cudaError_t launch_fs_1d(const FsArgs& a, int mode, int f32, cudaStream_t s);
cudaError_t launch_fs_f32(const FsArgs& a, int which, int flag, cudaStream_t s);   // freespace_f32.cu
// FP32 copy of n complex values
cudaError_t launch_fs_to_f32(float2* dst, const double2* src, size_t n, cudaStream_t s);

// FP64 residual check of the FP32-transform step (free space).  Per instance b
// (NM modes, ring slot R_n in FP32 at ring + b rstride):
//   prep:   W = u^ + i hm0 R_n  (FP64)
//   norms:  sums[b] = (sum |R64 - R_n|^2, sum |u^|^2)
//   decide: rho[b] = hm0 sqrt(s0 / s1); flag[b] = !(rho <= tol); ncorr[b] += flag
//   apply:  where flagged, u^ <- Wc, R_n <- R64 (FP32), u <- u64
cudaError_t launch_fs_res_prep(double2* W, const double2* uhat, const float2* ring, size_t rstride, size_t NM, int B,
                               double hm0, cudaStream_t s);
cudaError_t launch_fs_res_norms(const double2* R64, const float2* ring, size_t rstride, const double2* uhat, size_t NM,
                                int B, double* sums, cudaStream_t s);
cudaError_t launch_fs_res_decide(const double* sums, int B, double hm0, double tol, double* rho, int* flags, int* ncorr,
                                 cudaStream_t s);
cudaError_t launch_fs_res_apply(const int* flags, int B, size_t NM, size_t NX, double2* uhat, const double2* Wc,
                                float2* ring, size_t rstride, const double2* R64, double2* u, const double2* u64,
                                cudaStream_t s);
// P[iv][m] of one instance and axis: zeta [N] complex, phi_axis [ntf] = that
// component of phi at t = m dt / 8.
cudaError_t launch_fs_phase(double2* P, const double2* zeta, int N, const int2* intervals, int n_int,
                            const double* phi_axis, double dt, cudaStream_t s);

}  // namespace tdse
