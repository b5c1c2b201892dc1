// Private context of the C ABI (include/tdse.h), shared by the periodic
// orchestrator (api.cpp) and the free-space one (fs_api.cpp).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <string>
#include <vector>

#include "kargs.h"
#include "tdse.h"

namespace tdse {

constexpr int SUB = 8;   // fine time grid: t_m = m dt / 8 (Richardson sub-steps down to dt/8)
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// q-point Gauss-Legendre nodes/weights on [-1,1] (api.cpp).
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w);

// One axis of the free-space contour rule (Sec. 3.4, 4.1), host copy.
struct FsAxisHost {
    int M = 0, nu = 0, R = 0, NE = 0, ND = 0, NC = 0, N = 0, p = 0, kappa = 0, q = 0, n_r = 0;
    int NT = 0;                 // terms of the Chebyshev form of the C-type transforms (0: direct sums)
    double H = 0, K = 0, h = 0;
    std::vector<double> zeta;   // [N][2] nodes (complex)
    std::vector<double> w;      // [N][2] weights (complex)
};

struct FsState {
    FsAxisHost ax[3];
    size_t NM = 0;   // modes per instance (N0 N1 N2)
    size_t NX = 0;   // grid points per instance (M0 M1 M2)
    bool f32 = false;   // TDSE_MIXED: FP32 transforms, ring, intermediate and history sum
    struct {
        size_t uhat, ring, chain_uhat, chain_ring, chain_u, u, Z, Y, V0, tfac, phi, iv, scratch, end;
        size_t zeta[3], preI[3], postI[3], preF[3], postF[3], Gd[3], Fd[3], tw[3], P[3];
        // FP32 copies (f32 only; 0 otherwise)
        size_t preI_f[3], postI_f[3], preF_f[3], postF_f[3], Gd_f[3], Fd_f[3], tw_f[3], P_f[3];
        // FP64 residual check of the FP32 step (f32 only): W / corrected state, R64, u64, intermediates
        size_t res_W, res_R, res_u, Z64, Y64;
        // Chebyshev form of the C-type transforms (NT > 0 only)
        size_t Lf[3], Li[3], Tc[3], TcW[3], Lf_f[3], Li_f[3], Tc_f[3], TcW_f[3];
    } off{};
    int zero_iv = -1;   // f32: interval of zero length (one-step phase 1) for the FP64 re-evaluation
};

}  // namespace tdse

struct tdse_ctx {
    bool fs = false;            // free-space (bc = TDSE_FREE) context: state in F
    tdse::FsState F;
    tdse_config cfg{};
    int d = 1, n0 = 0, n1 = 1, n2 = 1;   // n2: axis 2 of 3D periodic grids
    size_t ntab = 0;            // entries per row of the separable phase tables (n0 + n1 (+ n2))
    // 1D grids beyond one CTA: N = n0 points through the 2D passes as fs0 x fs1
    // (four-step transform, grid stored transposed in the workspace)
    bool four1d = false;
    int shape1d = 0;            // 1D FP32 steps: launch shape chosen by the batch tuner (KArgs::shape1d)
    int fs0 = 0, fs1 = 0;
    size_t NP = 0;
    int B = 1, m = 8, L = 4, S = 7, S_eff = 7, RS = 7, ntf = 0, n_int = 0, n_int_startup = 0, nhi = 1;
    bool mixed = false;
    bool ip = false;            // mixed mode: state and ring are in the interaction picture
    int nh = 1, nl = 1, lb = 0;
    size_t rsz = 16;            // ring element bytes
    double mu[8] = {0};
    double rich[4] = {0};
    std::vector<int2> intervals;
    std::vector<float> zdither;   // [nsteps + 1][2]: FP32 ring dither z_n (interaction picture)
    // workspace
    char* ws = nullptr;
    size_t ws_need = 0;
    struct {
        size_t uhat, ring, chain_uhat, chain_ring, aux, aux2, V0, V0f, tfac, phi, kin64, kinff, adv64, advff,
            q64, qff, e2d, k1lo, k1hi, a1d, tw64_0, tw32_0, tw64_1, tw32_1, tw32lo_0, tw32lo_1, tw64_2, tw32_2,
            tw32lo_2, tw1d64, tw1d32, tw1d32lo, iv, tw128, res_sums,
            res_rho, res_flags, res_ncorr, cl_tab, err, scratch, end;
    } off{};
    // 2D mixed steps over CTA clusters (512^2): plan built at bind, used when
    // step_path allows it (TDSE_PATH_AUTO / TDSE_PATH_CLUSTER)
    tdse::ClPlan cl{};
    bool cl_ok = false;
    int step_path = TDSE_PATH_AUTO;
    // 2D pass kernels: the instances split into step_groups groups whose step
    // chains run on parallel streams (forked from and joined to the caller's
    // stream); 1 = one chain for the whole batch.  Default 4: measured on the
    // 64 x 512^2 mixed workload, 0.495 ms per step with one chain, 0.46 with
    // 2..16 groups.
    int step_groups = 4;
    std::vector<cudaStream_t> group_streams;
    std::vector<cudaEvent_t> group_join;
    cudaEvent_t group_fork = nullptr;
    ~tdse_ctx() {
        for (cudaStream_t g : group_streams)
            if (g) cudaStreamDestroy(g);
        for (cudaEvent_t e : group_join)
            if (e) cudaEventDestroy(e);
        if (group_fork) cudaEventDestroy(group_fork);
    }
    std::vector<char> have_V, have_u0;
    bool vtable = false;        // TDSE_V_TABLE(_SHARED): V(x, t_r) rows in V0 / V0f
    bool vshared = false;       // one table for every instance
    int vrows = 1;              // rows per instance (1 when separable)
    int res_every = 0;          // FP64 residual check after every res_every-th Adams step (mixed; 0 = off)
    double res_tol = 0.0;
    int res_checks = 0;
    int step = 0;
    bool inited = false;
    std::string err;

    template <class T> T* P(size_t o) const { return reinterpret_cast<T*>(ws + o); }
    tdse_status fail(tdse_status s, const std::string& msg) {
        err = msg;
        return s;
    }
};

inline tdse_status cuda_fail(tdse_ctx* c, cudaError_t e, const char* where) {
    return c->fail(TDSE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define TDSE_CK(ctx, expr)                                       \
    do {                                                         \
        cudaError_t e__ = (expr);                                \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, #expr); \
    } while (0)



inline int slot_of(const tdse_ctx* c, int n) { return ((n % c->RS) + c->RS) % c->RS; }

// Interval ids.  Start-up step s (1..S_eff) owns ids (s-1)(2^L - 1) .. s(2^L - 1) - 1:
// chain c, sub-step i at (s-1)(2^L - 1) + (2^c - 1) + i (chain 0 is the main
// interval t_{s-1} -> t_s).  Main intervals of later steps n follow from
// n_int_startup (FP64 mode only: mixed Adams steps use absolute phases).
inline int startup_interval(const tdse_ctx* c, int s, int chain, int i) {
    return (s - 1) * ((1 << c->L) - 1) + ((1 << chain) - 1) + i;
}
inline int main_interval(const tdse_ctx* c, int n) {
    return n <= c->S_eff ? startup_interval(c, n, 0, 0) : c->n_int_startup + (n - c->S_eff - 1);
}

// Row of the potential table holding V(t_tf), t_tf = tf dt / 8: every fine
// time of the start-up steps, then one row per Adams step (tf a multiple of 8).
inline size_t vrow(const tdse_ctx* c, int tf) {
    if (!c->vtable) return 0;
    const int fine = tdse::SUB * c->S_eff;
    return tf <= fine ? (size_t)tf : (size_t)fine + (size_t)(tf / tdse::SUB - c->S_eff);
}

// Free-space orchestration (fs_api.cpp), called by the entry points in api.cpp
// once the common fields of the context are set.
tdse_status fs_create(tdse_ctx* c);
tdse_status fs_bind(tdse_ctx* c, cudaStream_t s);
tdse_status fs_build_phase_tables(tdse_ctx* c, int b, cudaStream_t s);
tdse_status fs_set_initial(tdse_ctx* c, int b, const double* u0, cudaMemcpyKind kind, cudaStream_t s);
tdse_status fs_steps(tdse_ctx* c, int nsteps, cudaStream_t s);
tdse_status fs_read_u(tdse_ctx* c, int lo, int hi, double* out, cudaMemcpyKind kind, cudaStream_t s);
