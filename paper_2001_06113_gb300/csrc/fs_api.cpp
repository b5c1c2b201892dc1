// Free-space orchestration (bc = TDSE_FREE): the contour rule of Sec. 3.4 and
// 4.1, the transform and phase tables, the workspace layout and the launch
// sequence of the start-up (Richardson on u^ and u, Remark highorderfs) and
// of the Adams steps.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "alpert_rules.h"
#include "ctx.h"
#include "fsargs.h"
#include "kargs.h"

using namespace tdse;

namespace {

constexpr long double kPiL = 3.141592653589793238462643383279502884L;

const AlpertRule* find_alpert(int p) {
    for (const AlpertRule& r : kAlpertRules)
        if (r.p == p) return &r;
    return nullptr;
}

// e^{i theta} with theta reduced to [-pi, pi] in long double first, so that
// large phases (|theta| up to ~ K) lose no accuracy.
void cis(long double theta, double& c, double& s) {
    long double r = fmodl(theta, 2.0L * kPiL);
    if (r > kPiL) r -= 2.0L * kPiL;
    if (r < -kPiL) r += 2.0L * kPiL;
    c = std::cos((double)r);
    s = std::sin((double)r);
}

// Nodes and weights of one axis (Sec. 3.4): E1, A1, C, A3, E3.
bool build_rule(FsAxisHost& A, int M, int nu, int p, int q, int n_r, double H) {
    const AlpertRule* ar = find_alpert(p);
    if (!ar) return false;
    A.M = M;
    A.nu = nu;
    A.R = nu / M;
    A.p = p;
    A.kappa = ar->kappa;
    A.q = q;
    A.n_r = n_r;
    A.H = H;
    A.NE = nu / 2 - 2 * A.kappa + 1;                 // nu = 2 (NE + 2 kappa - 1)
    if (A.NE <= M / 2) return false;                 // the blocks must reach beyond |Re zeta| = pi M / 2 - ...
    A.K = H + M_PI * M / 2.0;
    A.h = (A.K - H) / (A.NE + 2 * A.kappa - 1);
    A.NC = q * (n_r == 0 ? 1 : 2 * n_r);
    A.ND = 2 * p + A.NC;
    A.N = 2 * A.NE + A.ND;
    if (A.ND > FS_MAX_ND) return false;
    A.zeta.clear();
    A.w.clear();
    auto push = [&](double zr, double zi, double wr, double wi) {
        A.zeta.push_back(zr);
        A.zeta.push_back(zi);
        A.w.push_back(wr);
        A.w.push_back(wi);
    };
    const double h = A.h;
    // E1: reflection of E3 (zeta -> -zeta), ascending real part
    for (int i = 0; i < A.NE; ++i) push(-((H + A.kappa * h) + (A.NE - 1 - i) * h), H, h, 0.0);
    // A1: reflection of the Alpert nodes on Gamma_3
    for (int k = p - 1; k >= 0; --k) push(-(H + ar->x[k] * h), H, h * ar->w[k], 0.0);
    // C: composite q-point Gauss-Legendre on Gamma_2, zeta = (1 - i) tau, d zeta = (1 - i) d tau,
    // panels [-H, H] (n_r = 0) or dyadic toward 0: edges +-H / 2^(n_r - k), k = 1..n_r, and 0
    std::vector<double> gx, gw;
    gauss_legendre(q, gx, gw);
    std::vector<int> order(q);
    for (int i = 0; i < q; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return gx[a] < gx[b]; });
    std::vector<double> edges;
    if (n_r == 0) {
        edges = {-H, H};
    } else {
        std::vector<double> pos = {0.0};
        for (int k = 1; k <= n_r; ++k) pos.push_back(H / std::ldexp(1.0, n_r - k));
        for (int k = (int)pos.size() - 1; k >= 1; --k) edges.push_back(-pos[k]);
        for (double v : pos) edges.push_back(v);
    }
    for (size_t e = 0; e + 1 < edges.size(); ++e) {
        const double a = edges[e], b = edges[e + 1];
        for (int i : order) {
            const double tau = 0.5 * (b - a) * gx[i] + 0.5 * (a + b);
            const double wt = 0.5 * (b - a) * gw[i];
            push(tau, -tau, wt, -wt);
        }
    }
    // A3 and E3 on Gamma_3: tau - iH
    for (int k = 0; k < p; ++k) push(H + ar->x[k] * h, -H, h * ar->w[k], 0.0);
    for (int i = 0; i < A.NE; ++i) push((H + A.kappa * h) + i * h, -H, h, 0.0);
    return (int)A.zeta.size() == 2 * A.N;
}

struct AxisTables {
    std::vector<double> zeta, preI, postI, preF, postF, Gd, Fd, tw;
    std::vector<double> Lf, Li, Tc, TcW;   // Chebyshev form of the C-type transforms (NT > 0)
};

// Chebyshev form of the C-type transforms (Sec. 4.1).  For a grid point x the
// function tau -> e^{s (1+i) tau x} (s = -1 forward: e^{-i zeta x}; s = +1
// inverse: e^{+i zeta x}, zeta = (1 - i) tau) on [-H, H] is replaced by its
// NT-point Chebyshev interpolant sum_l c_l T_l(tau / H), the coefficients from
// the values at the Chebyshev points tau_m = H cos(pi (m + 1/2) / NT):
//   c_l = (2 / NT) sum_m g(tau_m) cos(l pi (m + 1/2) / NT),  c_0 halved.
// Long double throughout, rounded once.
struct ChebPoints {
    int NT;
    std::vector<long double> u, cosl_;   // cos(th_m), cos(l th_m) [m][l]
    ChebPoints(int nt) : NT(nt), u(nt), cosl_((size_t)nt * nt) {
        for (int m = 0; m < nt; ++m) {
            const long double th = kPiL * (m + 0.5L) / nt;
            u[m] = cosl(th);
            for (int l = 0; l < nt; ++l) cosl_[(size_t)m * nt + l] = cosl(l * th);
        }
    }
};
void cheb_coeffs(long double x, int s, long double H, const ChebPoints& P, std::vector<long double>& cr,
                 std::vector<long double>& ci) {
    const int NT = P.NT;
    cr.assign(NT, 0.0L);
    ci.assign(NT, 0.0L);
    for (int m = 0; m < NT; ++m) {
        const long double tau = H * P.u[m];
        const long double mag = expl(s * tau * x), ang = s * tau * x;   // e^{s tau x} e^{i s tau x}
        const long double gr = mag * cosl(ang), gi = mag * sinl(ang);
        const long double* cl = &P.cosl_[(size_t)m * NT];
        for (int l = 0; l < NT; ++l) {
            cr[l] += gr * cl[l];
            ci[l] += gi * cl[l];
        }
    }
    for (int l = 0; l < NT; ++l) {
        cr[l] *= 2.0L / NT;
        ci[l] *= 2.0L / NT;
    }
    cr[0] *= 0.5L;
    ci[0] *= 0.5L;
}

// T_l(u), l = 0..NT-1, by the three-term recurrence
void cheb_T(long double u, int NT, std::vector<long double>& T) {
    T.assign(NT, 0.0L);
    T[0] = 1.0L;
    if (NT > 1) T[1] = u;
    for (int l = 2; l < NT; ++l) T[l] = 2.0L * u * T[l - 1] - T[l - 2];
}

// Smallest NT (8..FS_MAX_NT, even) whose interpolants reproduce e^{-+i zeta x}
// at every C node to 4 units of FP64 rounding of the largest value, checked
// at every 16th grid point and at both ends of the grid (the interpolation
// error of e^{a tau} grows with |a| = sqrt(2) |x|, largest at the ends); 0 if
// none does.
int choose_nt(const FsAxisHost& A) {
    const int p = A.p, NC = A.NC, M = A.M, NE = A.NE;
    const long double H = A.H;
    std::vector<long double> cr, ci, T;
    for (int NT = 8; NT <= FS_MAX_NT; NT += 2) {
        const ChebPoints P(NT);
        long double err = 0.0L, big = 0.0L;
        for (int j = 0; j < M; j = (j + 16 < M || j == M - 1) ? j + 16 : M - 1) {
            const long double x = -1.0L + 2.0L * j / M;
            for (int sg = -1; sg <= 1; sg += 2) {
                cheb_coeffs(x, sg, H, P, cr, ci);
                for (int k = 0; k < NC; ++k) {
                    const long double tau = A.zeta[2 * (NE + p + k)];
                    cheb_T(tau / H, NT, T);
                    long double vr = 0.0L, vi = 0.0L;
                    for (int l = 0; l < NT; ++l) {
                        vr += cr[l] * T[l];
                        vi += ci[l] * T[l];
                    }
                    const long double mag = expl(sg * tau * x), ang = sg * tau * x;
                    const long double gr = mag * cosl(ang), gi = mag * sinl(ang);
                    err = fmaxl(err, hypotl(vr - gr, vi - gi));
                    big = fmaxl(big, mag);
                }
            }
        }
        if (err <= 4.0L * 2.220446049250313e-16L * big) return NT;
    }
    return 0;
}

void make_cheb_tables(const FsAxisHost& A, AxisTables& T) {
    const int M = A.M, NT = A.NT, NC = A.NC, NE = A.NE, p = A.p;
    const long double H = A.H;
    std::vector<long double> cr, ci, Tl;
    const ChebPoints P(NT);
    T.Lf.assign((size_t)2 * NT * M, 0.0);
    T.Li.assign((size_t)2 * NT * M, 0.0);
    for (int j = 0; j < M; ++j) {
        const long double x = -1.0L + 2.0L * j / M;
        cheb_coeffs(x, -1, H, P, cr, ci);
        for (int l = 0; l < NT; ++l) {
            T.Lf[2 * ((size_t)l * M + j)] = (double)(cr[l] * 2.0L / M);
            T.Lf[2 * ((size_t)l * M + j) + 1] = (double)(ci[l] * 2.0L / M);
        }
        cheb_coeffs(x, +1, H, P, cr, ci);
        for (int l = 0; l < NT; ++l) {
            T.Li[2 * ((size_t)l * M + j)] = (double)cr[l];
            T.Li[2 * ((size_t)l * M + j) + 1] = (double)ci[l];
        }
    }
    T.Tc.assign((size_t)NC * NT, 0.0);
    T.TcW.assign((size_t)2 * NT * NC, 0.0);
    const long double inv2pi = 1.0L / (2.0L * kPiL);
    for (int k = 0; k < NC; ++k) {
        const int m = NE + p + k;
        cheb_T((long double)A.zeta[2 * m] / H, NT, Tl);
        const long double wr = A.w[2 * m] * inv2pi, wi = A.w[2 * m + 1] * inv2pi;
        for (int l = 0; l < NT; ++l) {
            T.Tc[(size_t)k * NT + l] = (double)Tl[l];
            T.TcW[2 * ((size_t)l * NC + k)] = (double)(Tl[l] * wr);
            T.TcW[2 * ((size_t)l * NC + k) + 1] = (double)(Tl[l] * wi);
        }
    }
}

// Host tables of one axis (fsargs.h FsAxis), in FP64 from long double phases.
AxisTables make_tables(const FsAxisHost& A) {
    AxisTables T;
    const int M = A.M, R = A.R, nu = A.nu, NE = A.NE, ND = A.ND;
    const long double h = A.h;
    T.zeta = A.zeta;
    auto put = [](std::vector<double>& v, double mag, long double theta) {
        double c, s;
        cis(theta, c, s);
        v.push_back(mag * c);
        v.push_back(mag * s);
    };
    const long double inv2pi = 1.0L / (2.0L * kPiL);
    // block origins zeta0 (E1: first node; E3: node NE + ND)
    const double z0r[2] = {A.zeta[0], A.zeta[2 * (NE + ND)]};
    const double z0i[2] = {A.zeta[1], A.zeta[2 * (NE + ND) + 1]};
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < NE; ++i) put(T.preI, (double)(h * inv2pi), -(long double)i * h);
    for (int b = 0; b < 2; ++b)
        for (int j = 0; j < M; ++j) {
            const double x = -1.0 + 2.0 * j / M;
            for (int s = 0; s < R; ++s) {
                const long double tw = 2.0L * kPiL * (long double)(((long long)j * s) % nu) / nu;
                // e^{i zeta0 x} = e^{-Im(zeta0) x} e^{i Re(zeta0) x}
                put(T.postI, std::exp(-z0i[b] * x), (long double)z0r[b] * x + tw);
                put(T.preF, (2.0 / M) * std::exp(z0i[b] * x), -(long double)z0r[b] * x - tw);
            }
        }
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < NE; ++i) put(T.postF, 1.0, (long double)i * h);
    for (int dd = 0; dd < ND; ++dd) {
        const int m = NE + dd;
        const double zr = A.zeta[2 * m], zi = A.zeta[2 * m + 1];
        const double wr = A.w[2 * m] / (2.0 * M_PI), wi = A.w[2 * m + 1] / (2.0 * M_PI);
        for (int j = 0; j < M; ++j) {
            const double x = -1.0 + 2.0 * j / M;
            double c, s;
            cis((long double)zr * x, c, s);
            const double e = std::exp(-zi * x);
            // (w / 2pi) e^{i zeta x}
            const double gr = e * c, gi = e * s;
            T.Gd.push_back(wr * gr - wi * gi);
            T.Gd.push_back(wr * gi + wi * gr);
            // (2/M) e^{-i zeta x} = (2/M) e^{zi x} (c - i s)
            const double f = (2.0 / M) / e;
            T.Fd.push_back(f * c);
            T.Fd.push_back(-f * s);
        }
    }
    for (int m = 0; m < M; ++m) put(T.tw, 1.0, -2.0L * kPiL * m / M);
    if (A.NT > 0) make_cheb_tables(A, T);
    return T;
}

FsArgs fs_base(const tdse_ctx* c) {
    const FsState& F = c->F;
    FsArgs a{};
    a.B = c->B;
    a.d = c->d;
    for (int x = 0; x < 3; ++x) {
        FsAxis& X = a.ax[x];
        if (x >= c->d) {
            X.M = 1;
            X.N = 1;
            continue;
        }
        const FsAxisHost& A = F.ax[x];
        X.M = A.M;
        X.R = A.R;
        X.nu = A.nu;
        X.NE = A.NE;
        X.ND = A.ND;
        X.N = A.N;
        X.preI = c->P<double2>(F.off.preI[x]);
        X.postI = c->P<double2>(F.off.postI[x]);
        X.preF = c->P<double2>(F.off.preF[x]);
        X.postF = c->P<double2>(F.off.postF[x]);
        X.Gd = c->P<double2>(F.off.Gd[x]);
        X.Fd = c->P<double2>(F.off.Fd[x]);
        X.tw = c->P<double2>(F.off.tw[x]);
        X.P = c->P<double2>(F.off.P[x]);
        X.p = A.p;
        X.NC = A.NC;
        X.NT = A.NT;
        if (A.NT > 0) {
            X.Lf = c->P<double2>(F.off.Lf[x]);
            X.Li = c->P<double2>(F.off.Li[x]);
            X.Tc = c->P<double>(F.off.Tc[x]);
            X.TcW = c->P<double2>(F.off.TcW[x]);
            if (F.f32) {
                X.Lf_f = c->P<float2>(F.off.Lf_f[x]);
                X.Li_f = c->P<float2>(F.off.Li_f[x]);
                X.Tc_f = c->P<float>(F.off.Tc_f[x]);
                X.TcW_f = c->P<float2>(F.off.TcW_f[x]);
            }
        }
        if (F.f32) {
            X.preI_f = c->P<float2>(F.off.preI_f[x]);
            X.postI_f = c->P<float2>(F.off.postI_f[x]);
            X.preF_f = c->P<float2>(F.off.preF_f[x]);
            X.postF_f = c->P<float2>(F.off.postF_f[x]);
            X.Gd_f = c->P<float2>(F.off.Gd_f[x]);
            X.Fd_f = c->P<float2>(F.off.Fd_f[x]);
            X.tw_f = c->P<float2>(F.off.tw_f[x]);
            X.P_f = c->P<float2>(F.off.P_f[x]);
        }
    }
    a.n_int = c->n_int;
    a.uhat = c->P<double2>(F.off.uhat);
    a.ring = c->P<double2>(F.off.ring);
    a.ring_slots = c->RS;
    a.Z = F.off.Z ? c->P<double2>(F.off.Z) : nullptr;
    a.Y = F.off.Y ? c->P<double2>(F.off.Y) : nullptr;
    a.u = c->P<double2>(F.off.u);
    a.V0 = c->P<double>(F.off.V0);
    a.vstride = c->vshared ? 0 : (size_t)c->vrows * F.NX;
    a.tfac = c->P<double>(F.off.tfac);
    a.ntf = c->ntf;
    return a;
}

// The launch evaluates V at t = tf dt / 8 (with a potential table: that row).
void set_time(const tdse_ctx* c, FsArgs& a, int tf) {
    a.tf = tf;
    a.V0 = c->P<double>(c->F.off.V0) + vrow(c, tf) * c->F.NX;
}

// Ring slot `slot` of a ring with rsz-byte elements (as the kernels' double2* field).
double2* ring_at(const tdse_ctx* c, size_t ring_off, size_t elems) {
    return reinterpret_cast<double2*>(c->P<char>(ring_off) + elems * c->rsz);
}

// Grid values usrc (times V(t_tf) if mulV) -> mode space: into the FP64 state
// (to_ring = 0) or a ring slot in the ring's element type (to_ring = 1), instance
// b at fdst + b bstride elements.
tdse_status forward_to(tdse_ctx* c, const double2* usrc, int mulV, int tf, double2* fdst, size_t bstride,
                       int to_ring, cudaStream_t s) {
    FsArgs a = fs_base(c);
    a.usrc = usrc;
    a.mulV = mulV;
    set_time(c, a, tf);
    a.fdst = fdst;
    a.fdst_bstride = bstride;
    a.fdst_ring = to_ring;
    const int f32 = c->F.f32 ? 1 : 0;
    if (c->d == 1) {
        TDSE_CK(c, launch_fs_1d(a, FS_1D_FWD_ONLY, f32, s));
    } else {
        TDSE_CK(c, launch_fs_phys(a, 1, f32, s));
        if (c->d == 3) TDSE_CK(c, launch_fs_mid(a, FS_MID_FWD, f32, s));
        TDSE_CK(c, launch_fs_row(a, FS_ROW_FWD_ONLY, f32, s));
    }
    return TDSE_OK;
}

// The part of a 2D / 3D step between the row passes: the grid work along
// axis 0 (3D: between the inverse and the forward transform along axis 1).
tdse_status grid_part(tdse_ctx* c, const FsArgs& a, int f32, cudaStream_t s) {
    if (c->d == 3) TDSE_CK(c, launch_fs_mid(a, FS_MID_INV, f32, s));
    TDSE_CK(c, launch_fs_phys(a, 0, f32, s));
    if (c->d == 3) TDSE_CK(c, launch_fs_mid(a, FS_MID_FWD, f32, s));
    return TDSE_OK;
}

// One step with the description in a: 1D fused kernel; 2D / 3D row begin,
// grid part, row end.
tdse_status one_step(tdse_ctx* c, const FsArgs& a, cudaStream_t s) {
    const int f32 = c->F.f32 ? 1 : 0;
    if (c->d == 1) {
        TDSE_CK(c, launch_fs_1d(a, FS_1D_STEP, f32, s));
    } else {
        TDSE_CK(c, launch_fs_row(a, FS_ROW_BEGIN, f32, s));
        tdse_status st = grid_part(c, a, f32, s);
        if (st != TDSE_OK) return st;
        TDSE_CK(c, launch_fs_row(a, FS_ROW_END, f32, s));
    }
    return TDSE_OK;
}

tdse_status fs_init(tdse_ctx* c, cudaStream_t s) {
    const FsState& F = c->F;
    double2* u = c->P<double2>(F.off.u);
    tdse_status st = forward_to(c, u, 0, 0, c->P<double2>(F.off.uhat), F.NM, 0, s);
    if (st != TDSE_OK) return st;
    st = forward_to(c, u, 1, 0, ring_at(c, F.off.ring, (size_t)slot_of(c, 0) * F.NM), (size_t)c->RS * F.NM, 1, s);
    if (st != TDSE_OK) return st;
    c->inited = true;
    return TDSE_OK;
}

// Start-up step n: L trapezoid chains with 1, 2, 4, .. sub-steps, Richardson
// combination of u^ and u, then (Vu)^(t_n) = forward(V(t_n) u).
tdse_status fs_startup_step(tdse_ctx* c, int n, cudaStream_t s) {
    const FsState& F = c->F;
    const size_t BM = (size_t)c->B * F.NM, BX = (size_t)c->B * F.NX;
    double2* cu = c->P<double2>(F.off.chain_uhat);
    double2* cx = c->P<double2>(F.off.chain_u);
    for (int ch = 0; ch < c->L; ++ch) {
        double2* cr = ring_at(c, F.off.chain_ring, ch * BM);
        TDSE_CK(c, cudaMemcpyAsync(cu + ch * BM, c->P<double2>(F.off.uhat), BM * 16, cudaMemcpyDeviceToDevice, s));
        TDSE_CK(c, launch_copy_slot(cr, c->P<void>(F.off.ring), c->RS, slot_of(c, n - 1), c->B, F.NM, c->rsz, s));
        const int len = SUB >> ch;
        for (int i = 0; i < (1 << ch); ++i) {
            FsArgs a = fs_base(c);
            a.uhat = cu + ch * BM;
            a.ring = cr;
            a.ring_slots = 1;
            a.u = cx + ch * BX;
            a.nhist = 1;
            a.h = c->cfg.dt / (double)(1 << ch);
            a.mu[0] = 0.5;
            a.mu[1] = 0.5;
            a.hist_slot[0] = 0;
            a.out_slot = 0;
            a.interval[0] = startup_interval(c, n, ch, i);
            set_time(c, a, SUB * (n - 1) + (i + 1) * len);
            tdse_status st = one_step(c, a, s);
            if (st != TDSE_OK) return st;
        }
    }
    TDSE_CK(c, launch_combine(c->P<void>(F.off.uhat), cu, BM, c->L, c->rich, BM, false, s));
    TDSE_CK(c, launch_combine(c->P<void>(F.off.u), cx, BX, c->L, c->rich, BX, false, s));
    return forward_to(c, c->P<double2>(F.off.u), 1, SUB * n, ring_at(c, F.off.ring, (size_t)slot_of(c, n) * F.NM),
                      (size_t)c->RS * F.NM, 1, s);
}

FsArgs adams_args(const tdse_ctx* c, int n) {
    FsArgs a = fs_base(c);
    a.nhist = c->m - 1;
    a.h = c->cfg.dt;
    for (int j = 0; j < c->m; ++j) a.mu[j] = c->mu[j];
    for (int j = 1; j <= a.nhist; ++j) a.hist_slot[j - 1] = slot_of(c, n - j);
    a.out_slot = slot_of(c, n);
    for (int i = 0; i < a.nhist; ++i) a.interval[i] = main_interval(c, n - i);
    set_time(c, a, SUB * n);
    return a;
}

// Adams steps n0+1 .. n0+k.  2D / 3D: row begin, (grid part, row end+begin)
// x (k-1), grid part, row end.
tdse_status fs_adams(tdse_ctx* c, int n0, int k, cudaStream_t s) {
    const int f32 = c->F.f32 ? 1 : 0;
    if (c->d == 1) {
        for (int n = n0 + 1; n <= n0 + k; ++n) TDSE_CK(c, launch_fs_1d(adams_args(c, n), FS_1D_STEP, f32, s));
        return TDSE_OK;
    }
    TDSE_CK(c, launch_fs_row(adams_args(c, n0 + 1), FS_ROW_BEGIN, f32, s));
    for (int n = n0 + 1; n < n0 + k; ++n) {
        tdse_status st = grid_part(c, adams_args(c, n), f32, s);
        if (st != TDSE_OK) return st;
        FsArgs f = adams_args(c, n + 1);
        f.out_slot = slot_of(c, n);
        TDSE_CK(c, launch_fs_row(f, FS_ROW_END | FS_ROW_BEGIN, f32, s));
    }
    const FsArgs last = adams_args(c, n0 + k);
    tdse_status st = grid_part(c, last, f32, s);
    if (st != TDSE_OK) return st;
    TDSE_CK(c, launch_fs_row(last, FS_ROW_END, f32, s));
    return TDSE_OK;
}

// FP64 residual of the implicit step just completed (step c->step, FP32
// transforms): W = u^ + i mu_0 h R_n, then the step's implicit part
// re-evaluated in FP64 (the FP64 kernels with no history term and a one-step
// phase of 1): u64 = inverse(W) / (1 + i mu_0 h V), R64 = forward(V u64),
// Wc = W - i mu_0 h R64; rho = mu_0 h ||R64 - R_n|| / ||u^||; where rho > tol
// (or is not finite) the step's results are replaced by the FP64 ones.
tdse_status fs_residual_check(tdse_ctx* c, cudaStream_t s) {
    const FsState& F = c->F;
    const int n = c->step;
    const double hm0 = c->cfg.dt * c->mu[0];
    const size_t rstride = (size_t)c->RS * F.NM;
    float2* ring_n = reinterpret_cast<float2*>(ring_at(c, F.off.ring, (size_t)slot_of(c, n) * F.NM));
    double2* uhat = c->P<double2>(F.off.uhat);
    double2* W = c->P<double2>(F.off.res_W);
    double2* R64 = c->P<double2>(F.off.res_R);
    double2* u64 = c->P<double2>(F.off.res_u);
    TDSE_CK(c, launch_fs_res_prep(W, uhat, ring_n, rstride, F.NM, c->B, hm0, s));
    FsArgs a = fs_base(c);
    a.uhat = W;                 // W in, W - i mu_0 h R64 out
    a.ring = R64;               // one FP64 slot: R64
    a.ring_slots = 1;
    a.u = u64;
    a.Z = F.off.Z64 ? c->P<double2>(F.off.Z64) : nullptr;
    a.Y = F.off.Y64 ? c->P<double2>(F.off.Y64) : nullptr;
    a.nhist = 0;
    a.h = c->cfg.dt;
    a.mu[0] = c->mu[0];
    a.out_slot = 0;
    a.interval[0] = F.zero_iv;
    set_time(c, a, SUB * n);
    if (c->d == 1) {
        TDSE_CK(c, launch_fs_1d(a, FS_1D_STEP, 0, s));
    } else {
        TDSE_CK(c, launch_fs_row(a, FS_ROW_BEGIN, 0, s));
        tdse_status st = grid_part(c, a, 0, s);
        if (st != TDSE_OK) return st;
        TDSE_CK(c, launch_fs_row(a, FS_ROW_END, 0, s));
    }
    double* sums = c->P<double>(c->off.res_sums);
    int* flags = c->P<int>(c->off.res_flags);
    TDSE_CK(c, launch_fs_res_norms(R64, ring_n, rstride, uhat, F.NM, c->B, sums, s));
    TDSE_CK(c, launch_fs_res_decide(sums, c->B, hm0, c->res_tol, c->P<double>(c->off.res_rho), flags,
                                    c->P<int>(c->off.res_ncorr), s));
    TDSE_CK(c, launch_fs_res_apply(flags, c->B, F.NM, F.NX, uhat, W, ring_n, rstride, R64, c->P<double2>(F.off.u),
                                   u64, s));
    ++c->res_checks;
    return TDSE_OK;
}

}  // namespace

tdse_status fs_create(tdse_ctx* c) {
    const tdse_config& g = c->cfg;
    FsState& F = c->F;
    const int p = g.alpert_p == 0 ? 8 : g.alpert_p;
    if (!find_alpert(p)) return c->fail(TDSE_EINVAL, "alpert_p must be 4 or 8");
    if (g.gauss_q < 1 || g.gauss_q > 32) return c->fail(TDSE_EINVAL, "gauss_q must be in 1..32");
    if (g.n_r < 0 || g.n_r > 4) return c->fail(TDSE_EINVAL, "n_r must be in 0..4");
    if (!(g.H > 0.0) || !std::isfinite(g.H)) return c->fail(TDSE_EINVAL, "H must be positive");
    if (g.c_transform < TDSE_CT_AUTO || g.c_transform > TDSE_CT_CHEBYSHEV)
        return c->fail(TDSE_EINVAL, "c_transform: TDSE_CT_AUTO, TDSE_CT_DIRECT or TDSE_CT_CHEBYSHEV");
    F.f32 = g.precision == TDSE_MIXED;
    F.NM = 1;
    F.NX = 1;
    for (int x = 0; x < c->d; ++x) {
        const int M = x < 2 ? g.n[x] : g.n_z, nu = x < 2 ? g.nu[x] : g.nu_z;
        if (M <= 0 || nu <= 0 || nu % M) return c->fail(TDSE_EINVAL, "nu must be a multiple of n");
        if (!fs_supported(M, nu / M)) return c->fail(TDSE_EUNSUPPORTED, "free space: n in 32..512, nu/n in {4,8,16}, nu <= 4096");
        if (!build_rule(F.ax[x], M, nu, p, g.gauss_q, g.n_r, g.H))
            return c->fail(TDSE_EINVAL, "contour rule: NE must exceed n/2 and the dense block 128 modes");
        F.ax[x].NT = 0;
        if (g.c_transform != TDSE_CT_DIRECT) {
            const int nt = choose_nt(F.ax[x]);
            if (g.c_transform == TDSE_CT_CHEBYSHEV && nt == 0)
                return c->fail(TDSE_EUNSUPPORTED, "C-type transforms: no Chebyshev interpolant of at most 64 terms "
                                                  "reaches FP64 rounding for this H");
            if (g.c_transform == TDSE_CT_CHEBYSHEV || (nt > 0 && nt < F.ax[x].NC)) F.ax[x].NT = nt;
        }
        F.NM *= (size_t)F.ax[x].N;
        F.NX *= (size_t)M;
    }
    // workspace
    const size_t B = c->B;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    F.off = {};
    F.off.uhat = take(B * F.NM * 16);
    F.off.ring = take(B * c->RS * F.NM * c->rsz);
    F.off.chain_uhat = take((size_t)c->L * B * F.NM * 16);
    F.off.chain_ring = take((size_t)c->L * B * F.NM * c->rsz);
    F.off.chain_u = take((size_t)c->L * B * F.NX * 16);
    F.off.u = take(B * F.NX * 16);
    // 2D: Z [N0][M1]; 3D: Z [N0][N1][M2] and Y [N0][M1][M2]
    const size_t zel = c->d == 2 ? (size_t)F.ax[0].N * F.ax[1].M
                                 : (c->d == 3 ? (size_t)F.ax[0].N * F.ax[1].N * F.ax[2].M : 0);
    const size_t yel = c->d == 3 ? (size_t)F.ax[0].N * F.ax[1].M * F.ax[2].M : 0;
    F.off.Z = zel ? take(B * zel * c->rsz) : 0;
    F.off.Y = yel ? take(B * yel * c->rsz) : 0;
    const size_t vcopies = c->vshared ? 1 : B;
    F.off.V0 = take(vcopies * c->vrows * F.NX * 8);
    const size_t V0f = take(vcopies * c->vrows * F.NX * 8);
    F.off.tfac = take(B * (size_t)c->ntf * 8);
    F.off.phi = take(B * (size_t)c->d * c->ntf * 8);
    F.off.iv = take((size_t)c->n_int * sizeof(int2));
    for (int x = 0; x < c->d; ++x) {
        const FsAxisHost& A = F.ax[x];
        F.off.zeta[x] = take((size_t)A.N * 16);
        F.off.preI[x] = take((size_t)2 * A.NE * 16);
        F.off.postI[x] = take((size_t)2 * A.nu * 16);
        F.off.preF[x] = take((size_t)2 * A.nu * 16);
        F.off.postF[x] = take((size_t)2 * A.NE * 16);
        F.off.Gd[x] = take((size_t)A.ND * A.M * 16);
        F.off.Fd[x] = take((size_t)A.ND * A.M * 16);
        F.off.tw[x] = take((size_t)A.M * 16);
        F.off.P[x] = take(B * (size_t)c->n_int * A.N * 16);
        if (A.NT > 0) {
            F.off.Lf[x] = take((size_t)A.NT * A.M * 16);
            F.off.Li[x] = take((size_t)A.NT * A.M * 16);
            F.off.Tc[x] = take((size_t)A.NC * A.NT * 8);
            F.off.TcW[x] = take((size_t)A.NT * A.NC * 16);
            if (F.f32) {
                F.off.Lf_f[x] = take((size_t)A.NT * A.M * 8);
                F.off.Li_f[x] = take((size_t)A.NT * A.M * 8);
                F.off.Tc_f[x] = take((size_t)A.NC * A.NT * 4);
                F.off.TcW_f[x] = take((size_t)A.NT * A.NC * 8);
            }
        }
        if (F.f32) {
            F.off.preI_f[x] = take((size_t)2 * A.NE * 8);
            F.off.postI_f[x] = take((size_t)2 * A.nu * 8);
            F.off.preF_f[x] = take((size_t)2 * A.nu * 8);
            F.off.postF_f[x] = take((size_t)2 * A.NE * 8);
            F.off.Gd_f[x] = take((size_t)A.ND * A.M * 8);
            F.off.Fd_f[x] = take((size_t)A.ND * A.M * 8);
            F.off.tw_f[x] = take((size_t)A.M * 8);
            F.off.P_f[x] = take(B * (size_t)c->n_int * A.N * 8);
        }
    }
    size_t res_sums = 0, res_rho = 0, res_flags = 0, res_ncorr = 0;
    if (F.f32) {   // FP64 residual check of the FP32 step
        F.off.res_W = take(B * F.NM * 16);
        F.off.res_R = take(B * F.NM * 16);
        F.off.res_u = take(B * F.NX * 16);
        F.off.Z64 = zel ? take(B * zel * 16) : 0;
        F.off.Y64 = yel ? take(B * yel * 16) : 0;
        res_sums = take(B * 16);
        res_rho = take(B * 8);
        res_flags = take(B * 4);
        res_ncorr = take(B * 4);
    }
    F.off.scratch = take(256);
    F.off.end = o;
    c->ws_need = o;
    // fields the shared entry points use
    c->off = {};
    c->off.uhat = F.off.uhat;
    c->off.V0 = F.off.V0;
    c->off.V0f = V0f;
    c->off.tfac = F.off.tfac;
    c->off.phi = F.off.phi;
    c->off.iv = F.off.iv;
    c->off.scratch = F.off.scratch;
    c->off.res_sums = res_sums;
    c->off.res_rho = res_rho;
    c->off.res_flags = res_flags;
    c->off.res_ncorr = res_ncorr;
    return TDSE_OK;
}

tdse_status fs_bind(tdse_ctx* c, cudaStream_t s) {
    FsState& F = c->F;
    for (int x = 0; x < c->d; ++x) {
        const AxisTables T = make_tables(F.ax[x]);
        auto up = [&](size_t off, const std::vector<double>& v) {
            return cudaMemcpyAsync(c->P<double>(off), v.data(), v.size() * 8, cudaMemcpyHostToDevice, s);
        };
        TDSE_CK(c, up(F.off.zeta[x], T.zeta));
        TDSE_CK(c, up(F.off.preI[x], T.preI));
        TDSE_CK(c, up(F.off.postI[x], T.postI));
        TDSE_CK(c, up(F.off.preF[x], T.preF));
        TDSE_CK(c, up(F.off.postF[x], T.postF));
        TDSE_CK(c, up(F.off.Gd[x], T.Gd));
        TDSE_CK(c, up(F.off.Fd[x], T.Fd));
        TDSE_CK(c, up(F.off.tw[x], T.tw));
        if (F.ax[x].NT > 0) {
            TDSE_CK(c, up(F.off.Lf[x], T.Lf));
            TDSE_CK(c, up(F.off.Li[x], T.Li));
            TDSE_CK(c, up(F.off.Tc[x], T.Tc));
            TDSE_CK(c, up(F.off.TcW[x], T.TcW));
        }
        // FP32 copies: each complex value rounded from the FP64 table
        std::vector<float> t32;
        auto up32 = [&](size_t off, const std::vector<double>& v) -> cudaError_t {
            t32.assign(v.begin(), v.end());
            const cudaError_t e = cudaMemcpyAsync(c->P<float>(off), t32.data(), t32.size() * 4, cudaMemcpyHostToDevice, s);
            return e != cudaSuccess ? e : cudaStreamSynchronize(s);   // t32 is reused
        };
        if (F.f32) {
            TDSE_CK(c, up32(F.off.preI_f[x], T.preI));
            TDSE_CK(c, up32(F.off.postI_f[x], T.postI));
            TDSE_CK(c, up32(F.off.preF_f[x], T.preF));
            TDSE_CK(c, up32(F.off.postF_f[x], T.postF));
            TDSE_CK(c, up32(F.off.Gd_f[x], T.Gd));
            TDSE_CK(c, up32(F.off.Fd_f[x], T.Fd));
            TDSE_CK(c, up32(F.off.tw_f[x], T.tw));
            if (F.ax[x].NT > 0) {
                TDSE_CK(c, up32(F.off.Lf_f[x], T.Lf));
                TDSE_CK(c, up32(F.off.Li_f[x], T.Li));
                TDSE_CK(c, up32(F.off.Tc_f[x], T.Tc));
                TDSE_CK(c, up32(F.off.TcW_f[x], T.TcW));
            }
        }
        TDSE_CK(c, cudaStreamSynchronize(s));    // T goes out of scope
    }
    return TDSE_OK;
}

tdse_status fs_build_phase_tables(tdse_ctx* c, int b, cudaStream_t s) {
    const FsState& F = c->F;
    const int2* iv = c->P<int2>(F.off.iv);
    for (int x = 0; x < c->d; ++x) {
        const FsAxisHost& A = F.ax[x];
        double2* P = c->P<double2>(F.off.P[x]) + (size_t)b * c->n_int * A.N;
        const double* phi = c->P<double>(F.off.phi) + ((size_t)b * c->d + x) * c->ntf;
        TDSE_CK(c, launch_fs_phase(P, c->P<double2>(F.off.zeta[x]), A.N, iv, c->n_int, phi, c->cfg.dt, s));
        if (F.f32)
            TDSE_CK(c, launch_fs_to_f32(c->P<float2>(F.off.P_f[x]) + (size_t)b * c->n_int * A.N, P,
                                        (size_t)c->n_int * A.N, s));
    }
    return TDSE_OK;
}

tdse_status fs_set_initial(tdse_ctx* c, int b, const double* u0, cudaMemcpyKind kind, cudaStream_t s) {
    const FsState& F = c->F;
    TDSE_CK(c, cudaMemcpyAsync(c->P<double2>(F.off.u) + (size_t)b * F.NX, u0, F.NX * 16, kind, s));
    return TDSE_OK;
}

tdse_status fs_steps(tdse_ctx* c, int nsteps, cudaStream_t s) {
    if (!c->inited) {
        tdse_status st = fs_init(c, s);
        if (st != TDSE_OK) return st;
    }
    int k = 0;
    while (k < nsteps) {
        const int n = c->step + 1;
        if (n <= c->S) {
            tdse_status st = fs_startup_step(c, n, s);
            if (st != TDSE_OK) return st;
            c->step = n;
            ++k;
            continue;
        }
        int run_len = nsteps - k;
        const bool check = c->F.f32 && c->res_every > 0;
        if (check) {   // stop at the next step to check
            const int to_check = c->res_every - c->step % c->res_every;
            if (to_check < run_len) run_len = to_check;
        }
        tdse_status st = fs_adams(c, c->step, run_len, s);
        if (st != TDSE_OK) return st;
        c->step += run_len;
        k += run_len;
        if (check && c->step % c->res_every == 0) {
            st = fs_residual_check(c, s);
            if (st != TDSE_OK) return st;
        }
    }
    return TDSE_OK;
}

tdse_status fs_read_u(tdse_ctx* c, int lo, int hi, double* out, cudaMemcpyKind kind, cudaStream_t s) {
    const FsState& F = c->F;
    TDSE_CK(c, cudaMemcpyAsync(out, c->P<double2>(F.off.u) + (size_t)lo * F.NX, (size_t)(hi - lo) * F.NX * 16, kind,
                               s));
    return TDSE_OK;
}

extern "C" tdse_status tdse_free_rule(const tdse_ctx* c, int axis, int* N, double* zeta, double* w) {
    if (!c || !N || !c->fs || axis < 0 || axis >= c->d) return TDSE_EINVAL;
    const FsAxisHost& A = c->F.ax[axis];
    *N = A.N;
    if (zeta) std::memcpy(zeta, A.zeta.data(), A.zeta.size() * 8);
    if (w) std::memcpy(w, A.w.data(), A.w.size() * 8);
    return TDSE_OK;
}

extern "C" tdse_status tdse_free_choose_H_prec(double eps, double vnorm, double phimax, int dim, int precision,
                                               double* H_out) {
    if (!H_out || dim < 1 || dim > 3 || !(eps > 0.0) || !(vnorm >= 0.0) || !(phimax >= 0.0)) return TDSE_EINVAL;
    if (precision != TDSE_FP64 && precision != TDSE_MIXED) return TDSE_EINVAL;
    // machine epsilon of the arithmetic that evaluates the contour sums
    const double eps_m = std::ldexp(1.0, precision == TDSE_FP64 ? -52 : -23);
    const double H = std::log(eps / ((1.0 + vnorm) * eps_m)) / (2.0 * dim * (1.0 + phimax));
    if (!(H > 0.0) || !std::isfinite(H)) return TDSE_EINVAL;
    *H_out = H;
    return TDSE_OK;
}

extern "C" tdse_status tdse_free_choose_H(double eps, double vnorm, double phimax, int dim, double* H_out) {
    return tdse_free_choose_H_prec(eps, vnorm, phimax, dim, TDSE_FP64, H_out);
}

extern "C" int tdse_free_cheb_terms(const tdse_ctx* c, int axis) {
    if (!c || !c->fs || axis < 0 || axis >= c->d) return -1;
    return c->F.ax[axis].NT;
}
