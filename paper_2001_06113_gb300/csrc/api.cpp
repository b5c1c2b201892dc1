// C ABI of the periodic TDSE solver (see include/tdse.h): context, workspace
// layout, host-side setup (Adams weights, phi(t), Richardson coefficients,
// interval schedule) and the launch sequence of each time step.
#include "tdse.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ctx.h"
#include "kargs.h"

namespace tdse {
struct ResArgs {
    KArgs a;
    int n;
    int slot;
    float z[2];
    double hmu0;
    double tol;
    double* sums;
    int* flags;
    double* rho;
    int* ncorr;
};
}  // namespace tdse

using namespace tdse;

namespace {

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Implicit Adams weights (Sec. 2.2): mu_j = int_0^1 l_j(theta) dtheta, l_j the
// Lagrange basis polynomial on the nodes theta = 0..n-1 (s = t - theta dt).
// Exact integer arithmetic: l_j = N_j(theta) / D_j with integer coefficients,
// int_0^1 theta^p = 1/(p+1) scaled by lcm(1..n).  The final quotient of two
// exact integers is correctly rounded.
bool adams_weights(int n, double* mu) {
    if (n < 1 || n > 12) return false;
    long long lcm = 1;
    for (long long q = 2; q <= n; ++q) {
        long long a = lcm, b = q;
        while (b) { long long t = a % b; a = b; b = t; }
        lcm = lcm / a * q;
    }
    for (int j = 0; j < n; ++j) {
        std::vector<long long> c(1, 1);       // coefficients of prod_{m != j} (theta - m), ascending
        long long D = 1;
        for (int m = 0; m < n; ++m) {
            if (m == j) continue;
            std::vector<long long> nc(c.size() + 1, 0);
            for (size_t p = 0; p < c.size(); ++p) {
                nc[p + 1] += c[p];
                nc[p] -= (long long)m * c[p];
            }
            c.swap(nc);
            D *= (long long)(j - m);
        }
        long long num = 0;
        for (size_t p = 0; p < c.size(); ++p) num += c[p] * (lcm / (long long)(p + 1));
        mu[j] = (double)num / ((double)lcm * (double)D);
    }
    return true;
}

}  // namespace

// q-point Gauss-Legendre nodes/weights on [-1,1] by Newton on P_q (long double).
void tdse::gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < q; ++i) {
        long double z = cosl(pi * (i + 0.75L) / (q + 0.5L));
        long double dp = 0;
        for (int it = 0; it < 100; ++it) {
            long double p0 = 1, p1 = z;
            for (int k = 2; k <= q; ++k) {
                long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = q * (z * p1 - p0) / (z * z - 1);
            long double dz = p1 / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        long double p0 = 1, p1 = z;
        for (int k = 2; k <= q; ++k) {
            long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = q * (z * p1 - p0) / (z * z - 1);
        x[i] = (double)z;
        w[i] = (double)(2.0L / ((1 - z * z) * dp * dp));
    }
}

static void plan_workspace(tdse_ctx* c) {
    const size_t NP = c->NP, B = c->B;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    c->off = {};
    c->off.uhat = take(B * NP * 16);
    c->off.ring = take(B * c->RS * NP * c->rsz);
    c->off.chain_uhat = take((size_t)c->L * B * NP * 16);
    c->off.chain_ring = take((size_t)c->L * B * NP * c->rsz);
    c->off.aux = take(B * NP * 16);
    c->off.aux2 = take(B * NP * 16);
    const size_t vcopies = c->vshared ? 1 : B;
    c->off.V0 = take(vcopies * c->vrows * NP * 8);
    c->off.V0f = take(vcopies * c->vrows * NP * 8);
    c->off.tfac = take(B * (size_t)c->ntf * 8);
    c->off.phi = take(B * (size_t)c->d * c->ntf * 8);
    const size_t nsp1 = (size_t)c->cfg.nsteps + 1;
    if (c->d == 1) {
        if (c->mixed) {
            c->off.kinff = take((size_t)c->L * c->n0 * 16);
            c->off.advff = take(B * (size_t)c->n_int * (c->nh + c->nl) * 16);
            c->off.k1lo = take((size_t)E1D_NLO * c->n0 * 8);
            c->off.k1hi = take((size_t)c->nhi * c->n0 * 8);
            c->off.a1d = take(B * nsp1 * (c->nh + c->nl) * 8);
        } else {
            c->off.kin64 = take((size_t)c->L * c->n0 * 16);
            c->off.adv64 = take(B * (size_t)c->n_int * (c->nh + c->nl) * 16);
        }
    } else {
        if (c->mixed) {
            c->off.qff = take(B * (size_t)c->n_int * c->ntab * 16);
            c->off.e2d = take(B * nsp1 * c->ntab * 8);
        } else {
            c->off.q64 = take(B * (size_t)c->n_int * c->ntab * 16);
        }
    }
    c->off.tw64_0 = take((size_t)c->n0 * 16);
    c->off.tw32_0 = take((size_t)c->n0 * 8);
    const int ax1 = c->four1d ? c->fs1 : (c->d >= 2 ? c->n1 : 1);
    c->off.tw64_1 = take((size_t)ax1 * 16);
    c->off.tw32_1 = take((size_t)ax1 * 8);
    if (c->four1d) {
        c->off.tw1d64 = take((size_t)c->n0 * 16);
        c->off.tw1d32 = take((size_t)c->n0 * 8);
        c->off.tw1d32lo = take((size_t)c->n0 * 8);
    }
    c->off.tw64_2 = take((size_t)(c->d == 3 ? c->n2 : 1) * 16);
    c->off.tw32_2 = take((size_t)(c->d == 3 ? c->n2 : 1) * 8);
    c->off.tw32lo_2 = take((size_t)(c->d == 3 ? c->n2 : 1) * 8);
    c->off.tw32lo_0 = take((size_t)c->n0 * 8);
    c->off.tw32lo_1 = take((size_t)ax1 * 8);
    c->off.iv = take((size_t)c->n_int * sizeof(int2));
    c->off.tw128 = c->d == 1 && c->n0 > 8192 && !c->four1d ? take(128 * 16) : 0;
    if (c->mixed) {
        c->off.res_sums = take(B * 16);
        c->off.res_rho = take(B * 8);
        c->off.res_flags = take(B * 4);
        c->off.res_ncorr = take(B * 4);
    }
    if (c->d == 2 && c->mixed && step2d_cluster_supported(c->n0, c->n1))
        c->off.cl_tab = take(((size_t)c->cfg.nsteps + 1) * CL_TAB * sizeof(float));
    c->off.err = take(256);
    c->off.scratch = take(256);
    c->off.end = o;
    c->ws_need = o;
}

template <class T> static T* opt(const tdse_ctx* c, size_t off) { return off ? c->P<T>(off) : nullptr; }



static void split(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

// w / z_m split into hi + lo floats (complex)
static void zinv(const tdse_ctx* c, int m, double w, float* hi, float* lo) {
    const double zx = c->zdither[2 * m], zy = c->zdither[2 * m + 1];
    const double n2 = zx * zx + zy * zy;
    split(w * zx / n2, hi[0], lo[0]);
    split(-w * zy / n2, hi[1], lo[1]);
}

// The same weights for every step m, as rows of the cluster kernel's table
// (layout in kargs.h); lags before step 0 are zero (never used: Adams steps
// start after the start-up).
static std::vector<float> cluster_weight_table(const tdse_ctx* c) {
    std::vector<float> t(((size_t)c->cfg.nsteps + 1) * CL_TAB, 0.0f);
    for (int m = 0; m <= c->cfg.nsteps; ++m) {
        float* r = t.data() + (size_t)m * CL_TAB;
        r[0] = c->zdither[2 * m];
        r[1] = c->zdither[2 * m + 1];
        float dh[2], dl[2];
        zinv(c, m, c->cfg.dt * c->mu[0], dh, dl);
        r[2] = dh[0]; r[3] = dh[1]; r[4] = dl[0]; r[5] = dl[1];
        for (int j = 1; j < c->m && j <= MAX_HIST; ++j) {
            if (m - j < 0) continue;
            float ch[2], cl[2];
            zinv(c, m - j, c->mu[j], ch, cl);
            float* w = r + 6 + 4 * (j - 1);
            w[0] = ch[0]; w[1] = ch[1]; w[2] = cl[0]; w[3] = cl[1];
        }
    }
    return t;
}

static KArgs base_args(const tdse_ctx* c) {
    KArgs a{};
    a.B = c->B;
    a.n0 = c->n0;
    a.n1 = c->n1;
    a.tn0 = c->n0;
    a.tn1 = c->d >= 2 ? c->n1 : 1;
    a.tn2 = c->d == 3 ? c->n2 : 0;
    a.shape1d = c->shape1d;
    a.uhat = c->P<void>(c->off.uhat);
    a.ring = c->P<void>(c->off.ring);
    a.ring_slots = c->RS;
    a.aux = c->P<double2>(c->off.aux);
    a.aux2 = c->P<double2>(c->off.aux2);
    a.V0 = c->P<double>(c->off.V0);
    a.V0f = c->P<float2>(c->off.V0f);
    a.vstride = c->vshared ? 0 : (size_t)c->vrows * c->NP;
    a.tfac = c->P<double>(c->off.tfac);
    a.ntf = c->ntf;
    a.n_int = c->n_int;
    a.dt = c->cfg.dt;
    a.phi = c->P<double>(c->off.phi);
    a.kin64 = opt<double2>(c, c->off.kin64);
    a.kinff = opt<float4>(c, c->off.kinff);
    a.adv64 = opt<double2>(c, c->off.adv64);
    a.advff = opt<float4>(c, c->off.advff);
    a.nh = c->nh;
    a.nl = c->nl;
    a.lb = c->lb;
    a.q64 = opt<double2>(c, c->off.q64);
    a.qff = opt<float4>(c, c->off.qff);
    a.e2d = opt<float2>(c, c->off.e2d);
    a.k1d_lo = opt<float2>(c, c->off.k1lo);
    a.k1d_hi = opt<float2>(c, c->off.k1hi);
    a.a1d = opt<float2>(c, c->off.a1d);
    a.tw64_0 = c->P<double2>(c->off.tw64_0);
    a.tw32_0 = c->P<float2>(c->off.tw32_0);
    a.tw64_1 = c->P<double2>(c->off.tw64_1);
    a.tw32_1 = c->P<float2>(c->off.tw32_1);
    a.tw32lo_0 = c->P<float2>(c->off.tw32lo_0);
    a.tw32lo_1 = c->P<float2>(c->off.tw32lo_1);
    a.tw64_2 = c->P<double2>(c->off.tw64_2);
    a.tw32_2 = c->P<float2>(c->off.tw32_2);
    a.tw32lo_2 = c->P<float2>(c->off.tw32lo_2);
    if (c->four1d) {   // 1D through the 2D passes: geometry fs0 x fs1, tables of the N-point grid
        a.n0 = c->fs0;
        a.n1 = c->fs1;
        a.tn0 = c->n0;
        a.tn1 = 1;
        a.flat1d = 1;
        a.tw1d64 = c->P<double2>(c->off.tw1d64);
        a.tw1d32 = c->P<float2>(c->off.tw1d32);
    }
    return a;
}

// per-step scalars: h, mu (and their hi/lo splits)
// The launch evaluates V at t = tf dt / 8: with a potential table, point V0 /
// V0f at that time's row.
static void set_time(const tdse_ctx* c, KArgs& a, int tf) {
    a.tf = tf;
    const size_t off = vrow(c, tf) * c->NP;
    a.V0 = c->P<double>(c->off.V0) + off;
    a.V0f = c->P<float2>(c->off.V0f) + off;
}

static void set_weights(KArgs& a, double h, const double* mu, int nmu) {
    a.h = h;
    split(h, a.h_hi, a.h_lo);
    for (int j = 0; j < nmu; ++j) {
        a.mu[j] = mu[j];
        split(mu[j], a.mu_hi[j], a.mu_lo[j]);
    }
    split(h * mu[0], a.hmu0_hi, a.hmu0_lo);
}

static int step_combo(const tdse_ctx* c) { return c->cfg.precision == TDSE_MIXED ? COMBO_F32 : COMBO_F64; }
static int f64_combo(const tdse_ctx* c) { return c->cfg.precision == TDSE_MIXED ? COMBO_F64_R32 : COMBO_F64; }

static cudaError_t run(const tdse_ctx* c, const KArgs& a, int combo, cudaStream_t s) {
    if (c->d == 3) return launch_periodic3d(a, combo, s);
    return c->d == 1 && !c->four1d ? launch_periodic1d(a, combo, s) : launch_periodic2d(a, combo, s);
}

static tdse_status build_phase_tables(tdse_ctx* c, int b, cudaStream_t s) {
    if (c->fs) return fs_build_phase_tables(c, b, s);
    const int2* iv = c->P<int2>(c->off.iv);
    const double* phi = c->P<double>(c->off.phi) + (size_t)b * c->d * c->ntf;
    const size_t nsp1 = (size_t)c->cfg.nsteps + 1;
    if (c->d == 1) {
        const size_t per = (size_t)c->n_int * (c->nh + c->nl);
        TDSE_CK(c, launch_adv1d(c->mixed ? nullptr : c->P<double2>(c->off.adv64) + b * per,
                                c->mixed ? c->P<float4>(c->off.advff) + b * per : nullptr, iv, c->n_int, phi, c->ntf,
                                c->n0, c->nh, c->nl, s));
        if (c->mixed)
            TDSE_CK(c, launch_a1d(c->P<float2>(c->off.a1d) + b * nsp1 * (c->nh + c->nl), phi, c->ntf, c->cfg.nsteps,
                                  c->n0, c->nh, c->nl, s));
    } else {
        const size_t per = (size_t)c->n_int * c->ntab;
        const int n2t = c->d == 3 ? c->n2 : 0;
        TDSE_CK(c, launch_q2d(c->mixed ? nullptr : c->P<double2>(c->off.q64) + b * per,
                              c->mixed ? c->P<float4>(c->off.qff) + b * per : nullptr, iv, c->n_int, phi, c->ntf,
                              c->n0, c->n1, n2t, c->cfg.dt, s));
        if (c->mixed)
            TDSE_CK(c, launch_e2d(c->P<float2>(c->off.e2d) + b * nsp1 * c->ntab, phi, c->ntf, c->cfg.nsteps, c->n0,
                                  c->n1, n2t, c->cfg.dt, s));
    }
    return TDSE_OK;
}

static bool instance_range(const tdse_ctx* c, int instance, int& lo, int& hi) {
    if (instance == -1) { lo = 0; hi = c->B; return true; }
    if (instance < 0 || instance >= c->B) return false;
    lo = instance;
    hi = instance + 1;
    return true;
}

// ---------------------------------------------------------------------------
extern "C" {

tdse_status tdse_adams_weights(int order, double* mu_out) {
    if (!mu_out || order < 1 || order > 12) return TDSE_EINVAL;
    return adams_weights(order, mu_out) ? TDSE_OK : TDSE_EINVAL;
}

tdse_status tdse_create(const tdse_config* cfg, tdse_ctx** out) {
    if (!cfg || !out) return TDSE_EINVAL;
    *out = nullptr;
    if (cfg->dim != 1 && cfg->dim != 2 && cfg->dim != 3) return TDSE_EINVAL;
    if (cfg->bc != TDSE_PERIODIC && cfg->bc != TDSE_FREE) return TDSE_EINVAL;
    const bool fs = cfg->bc == TDSE_FREE;
    if (!(cfg->dt > 0.0) || !std::isfinite(cfg->dt) || cfg->nsteps < 1 || cfg->batch < 1) return TDSE_EINVAL;
    if (cfg->order < 2 || cfg->order > 8 || cfg->order % 2) return TDSE_EINVAL;
    if (cfg->precision != TDSE_FP64 && cfg->precision != TDSE_MIXED) return TDSE_EINVAL;
    const int S = cfg->startup_steps < 0 ? cfg->order - 1 : cfg->startup_steps;
    if (S < cfg->order - 2) return TDSE_EINVAL;
    const int n0 = cfg->n[0], n1 = cfg->dim >= 2 ? cfg->n[1] : 1, n2 = cfg->dim == 3 ? cfg->n_z : 1;
    if (!is_pow2(n0) || (cfg->dim >= 2 && !is_pow2(n1)) || (cfg->dim == 3 && !is_pow2(n2))) return TDSE_EINVAL;
    if (cfg->dim == 3 && !fs && !periodic3d_supported(n0, n1, n2)) return TDSE_EUNSUPPORTED;
    if (cfg->layout_1d < TDSE_LAYOUT_AUTO || cfg->layout_1d > TDSE_LAYOUT_PASSES) return TDSE_EINVAL;
    const bool big1d = !fs && cfg->dim == 1 && cfg->precision == TDSE_MIXED && n0 == four_step_n();
    const bool cta1d = periodic1d_supported(n0) || big1d;   // one CTA per instance is built
    // the four-step transform through the 2D passes (larger 1D grids, or by choice), 64..2^20 points
    const bool four1d = !fs && cfg->dim == 1 && n0 >= 64 && n0 <= (1 << 20) &&
                        (cfg->layout_1d == TDSE_LAYOUT_PASSES || (cfg->layout_1d == TDSE_LAYOUT_AUTO && !cta1d));
    if (!fs && cfg->dim == 1 && !four1d && !(cta1d && cfg->layout_1d != TDSE_LAYOUT_PASSES)) return TDSE_EUNSUPPORTED;
    if (!fs && cfg->dim == 2 && !periodic2d_supported(n0, n1)) return TDSE_EUNSUPPORTED;
    if ((long long)cfg->nsteps * SUB + 1 > (1LL << 30)) return TDSE_EINVAL;
    if (cfg->potential != TDSE_V_SEPARABLE && cfg->potential != TDSE_V_TABLE &&
        cfg->potential != TDSE_V_TABLE_SHARED)
        return TDSE_EINVAL;

    tdse_ctx* c = new (std::nothrow) tdse_ctx();
    if (!c) return TDSE_ENOMEM;
    c->cfg = *cfg;
    c->cfg.startup_steps = S;
    c->d = cfg->dim;
    c->n0 = n0;
    c->n1 = n1;
    c->n2 = n2;
    c->NP = (size_t)n0 * n1 * n2;
    c->four1d = four1d;
    if (four1d) {
        int lg = 0;
        while ((1 << lg) < n0) ++lg;
        c->fs1 = 1 << ((lg + 1) / 2);
        c->fs0 = n0 / c->fs1;
    }
    c->ntab = (size_t)n0 + (cfg->dim >= 2 ? n1 : 0) + (cfg->dim == 3 ? n2 : 0);
    c->B = cfg->batch;
    c->m = cfg->order;
    c->L = cfg->order / 2;
    c->S = S;
    c->S_eff = S < cfg->nsteps ? S : cfg->nsteps;
    c->RS = cfg->order - 1 > 1 ? cfg->order - 1 : 1;
    c->ntf = cfg->nsteps * SUB + 1;
    c->rsz = cfg->precision == TDSE_MIXED ? 8 : 16;
    c->mixed = cfg->precision == TDSE_MIXED;
    adams_weights(c->m, c->mu);
    // Richardson: T[l][c] = (4^l T[l-1][c+1] - T[l-1][c]) / (4^l - 1); final T[L-1][0] = sum rich[c] T[0][c]
    {
        std::vector<std::vector<double>> T(c->L, std::vector<double>(c->L, 0.0));
        for (int q = 0; q < c->L; ++q) T[q][q] = 1.0;   // T[c] as coefficient vectors
        for (int lev = 1; lev < c->L; ++lev) {
            const double f = std::pow(4.0, lev);
            for (int q = 0; q + 1 < (int)T.size(); ++q)
                for (int r = 0; r < c->L; ++r) T[q][r] = (f * T[q + 1][r] - T[q][r]) / (f - 1.0);
            T.pop_back();
        }
        for (int r = 0; r < c->L; ++r) c->rich[r] = T[0][r];
    }
    // interval schedule (see startup_interval / main_interval)
    c->n_int_startup = c->S_eff * ((1 << c->L) - 1);
    const int n_main_rest = cfg->nsteps - c->S_eff;
    // periodic TDSE_MIXED evaluates the main-step phases from closed forms; the
    // free-space variant keeps tables for every step.
    const bool main_tables = !c->mixed || fs;
    c->n_int = c->n_int_startup + (main_tables ? n_main_rest : 0);
    c->intervals.resize(c->n_int);
    for (int s = 1; s <= c->S_eff; ++s)
        for (int ch = 0; ch < c->L; ++ch) {
            const int len = SUB >> ch;
            for (int i = 0; i < (1 << ch); ++i)
                c->intervals[startup_interval(c, s, ch, i)] =
                    make_int2(SUB * (s - 1) + i * len, SUB * (s - 1) + (i + 1) * len);
        }
    if (main_tables)
        for (int n = c->S_eff + 1; n <= cfg->nsteps; ++n)
            c->intervals[main_interval(c, n)] = make_int2(SUB * (n - 1), SUB * n);
    if (fs && c->mixed) {   // zero-length interval: the FP64 residual check re-evaluates a step with p_0 = 1
        c->intervals.push_back(make_int2(0, 0));
        c->F.zero_iv = c->n_int++;
    }
    c->nhi = cfg->nsteps / E1D_NLO + 1;
    // Ring dither: r~_n = z_n r^_n with z_n = e^{i psi_n}, psi_n = 2 pi frac(n (sqrt2 - 1)),
    // rounded to FP32 once; the history weights divide it out exactly (FP64).
    c->zdither.resize(2 * ((size_t)cfg->nsteps + 1));
    for (int n = 0; n <= cfg->nsteps; ++n) {
        const double f = (double)n * 0.41421356237309504880;
        const double psi = 6.28318530717958647692 * (f - std::floor(f));
        c->zdither[2 * n] = (float)std::cos(psi);
        c->zdither[2 * n + 1] = (float)std::sin(psi);
    }
    if (c->d == 1) {
        c->nl = n0 / 2 < 64 ? n0 / 2 : 64;
        c->lb = 0;
        while ((1 << c->lb) < c->nl) ++c->lb;
        c->nh = n0 / c->nl;
    }
    c->have_V.assign(c->B, 0);
    c->have_u0.assign(c->B, 0);
    c->vtable = cfg->potential != TDSE_V_SEPARABLE;
    c->vshared = cfg->potential == TDSE_V_TABLE_SHARED;
    c->vrows = c->vtable ? SUB * c->S_eff + 1 + (cfg->nsteps - c->S_eff) : 1;
    if (fs) {
        c->fs = true;
        const tdse_status st = fs_create(c);
        if (st != TDSE_OK) {
            delete c;
            return st;
        }
    } else {
        plan_workspace(c);
    }
    *out = c;
    return TDSE_OK;
}

size_t tdse_workspace_bytes(const tdse_ctx* c) { return c ? c->ws_need : 0; }

tdse_status tdse_bind_workspace(tdse_ctx* c, void* dev, size_t bytes, void* stream) {
    if (!c || !dev) return TDSE_EINVAL;
    if (bytes < c->ws_need) return c->fail(TDSE_ENOMEM, "workspace smaller than tdse_workspace_bytes()");
    if (reinterpret_cast<uintptr_t>(dev) & 255) return c->fail(TDSE_EINVAL, "workspace not 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    c->ws = static_cast<char*>(dev);
    TDSE_CK(c, cudaMemcpyAsync(c->P<int2>(c->off.iv), c->intervals.data(), c->intervals.size() * sizeof(int2),
                               cudaMemcpyHostToDevice, s));
    if (c->fs) {
        tdse_status st = fs_bind(c, s);
        if (st != TDSE_OK) return st;
    } else {
    TDSE_CK(c, launch_twiddles(c->P<double2>(c->off.tw64_0), c->P<float2>(c->off.tw32_0),
                               c->P<float2>(c->off.tw32lo_0), c->four1d ? c->fs0 : c->n0, s));
    if (c->four1d) {
        TDSE_CK(c, launch_twiddles(c->P<double2>(c->off.tw64_1), c->P<float2>(c->off.tw32_1),
                                   c->P<float2>(c->off.tw32lo_1), c->fs1, s));
        TDSE_CK(c, launch_twiddles(c->P<double2>(c->off.tw1d64), c->P<float2>(c->off.tw1d32),
                                   c->P<float2>(c->off.tw1d32lo), c->n0, s));
    }
    if (c->d == 3)
        TDSE_CK(c, launch_twiddles(c->P<double2>(c->off.tw64_2), c->P<float2>(c->off.tw32_2),
                                   c->P<float2>(c->off.tw32lo_2), c->n2, s));
    if (c->d >= 2)
        TDSE_CK(c, launch_twiddles(c->P<double2>(c->off.tw64_1), c->P<float2>(c->off.tw32_1),
                                   c->P<float2>(c->off.tw32lo_1), c->n1, s));
    else
        TDSE_CK(c, launch_kin1d(opt<double2>(c, c->off.kin64), opt<float4>(c, c->off.kinff), c->n0, c->L, c->cfg.dt, s));
    if (c->d == 1 && c->mixed)
        TDSE_CK(c, launch_k1d(c->P<float2>(c->off.k1lo), c->P<float2>(c->off.k1hi), c->nhi, c->n0, c->cfg.dt, s));
    if (c->off.tw128) TDSE_CK(c, launch_four_step_tables(c->P<double2>(c->off.tw128), s));
    TDSE_CK(c, cudaMemsetAsync(c->P<int>(c->off.err), 0, sizeof(int), s));
    c->cl_ok = false;
    if (c->off.cl_tab) {
        const std::vector<float> tab = cluster_weight_table(c);
        TDSE_CK(c, cudaMemcpyAsync(c->P<float>(c->off.cl_tab), tab.data(), tab.size() * sizeof(float),
                                   cudaMemcpyHostToDevice, s));
        TDSE_CK(c, cudaStreamSynchronize(s));      // the host table is freed on return
        const long long vrows_total = (long long)(c->vshared ? 1 : c->B) * c->vrows * c->n0;
        // no cluster path (no driver entry point, no resident cluster): the pass kernels run instead
        if (step2d_cluster_plan(c->cl, c->P<void>(c->off.uhat), c->P<void>(c->off.ring), c->P<void>(c->off.V0f), c->B,
                                c->RS, vrows_total) == cudaSuccess &&
            c->cl.clusters > 0)
            c->cl_ok = true;
        (void)cudaGetLastError();
    }
    }
    // defaults: A == 0 (phi == 0), f(t) == 1
    TDSE_CK(c, cudaMemsetAsync(c->P<double>(c->off.phi), 0, (size_t)c->B * c->d * c->ntf * 8, s));
    std::vector<double> ones(c->ntf, 1.0);
    for (int b = 0; b < c->B; ++b)
        TDSE_CK(c, cudaMemcpyAsync(c->P<double>(c->off.tfac) + (size_t)b * c->ntf, ones.data(), c->ntf * 8,
                                   cudaMemcpyHostToDevice, s));
    for (int b = 0; b < c->B; ++b) {
        tdse_status st = build_phase_tables(c, b, s);
        if (st != TDSE_OK) return st;
    }
    TDSE_CK(c, cudaStreamSynchronize(s));
    c->step = 0;
    c->inited = false;
    c->ip = false;
    return TDSE_OK;
}

tdse_status tdse_set_potential(tdse_ctx* c, int instance, const double* V0, const double* tf, int where,
                               void* stream) {
    if (!c || !V0) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    if (c->vtable) return c->fail(TDSE_ESTATE, "potential-table context: use tdse_set_potential_table");
    int lo, hi;
    if (!instance_range(c, instance, lo, hi)) return c->fail(TDSE_EINVAL, "instance out of range");
    if (where != TDSE_HOST && where != TDSE_DEVICE) return TDSE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = where == TDSE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int b = lo; b < hi; ++b) {
        double* dV = c->P<double>(c->off.V0) + (size_t)b * c->NP;
        if (c->four1d) {    // natural order -> the passes' transposed layout (through the intermediate buffer)
            double* tmp = c->P<double>(c->off.aux);
            TDSE_CK(c, cudaMemcpyAsync(tmp, V0, c->NP * 8, kind, s));
            TDSE_CK(c, launch_transpose_1d(dV, tmp, c->fs0, c->fs1, 1, 8, 1, s));
        } else {
            TDSE_CK(c, cudaMemcpyAsync(dV, V0, c->NP * 8, kind, s));
        }
        TDSE_CK(c, launch_split_float(c->P<float2>(c->off.V0f) + (size_t)b * c->NP, dV, c->NP, s));
        if (tf) {
            for (int i = 0; i < c->ntf; ++i)
                if (!std::isfinite(tf[i])) return c->fail(TDSE_EINVAL, "non-finite time factor");
            TDSE_CK(c, cudaMemcpyAsync(c->P<double>(c->off.tfac) + (size_t)b * c->ntf, tf, c->ntf * 8,
                                       cudaMemcpyHostToDevice, s));
        } else {
            std::vector<double> ones(c->ntf, 1.0);   // pageable: taken before the copy call returns
            TDSE_CK(c, cudaMemcpyAsync(c->P<double>(c->off.tfac) + (size_t)b * c->ntf, ones.data(), c->ntf * 8,
                                       cudaMemcpyHostToDevice, s));
        }
        c->have_V[b] = 1;
    }
    if (where == TDSE_HOST || tf) TDSE_CK(c, cudaStreamSynchronize(s));
    return TDSE_OK;
}

int tdse_potential_times(const tdse_ctx* c, double* t_out) {
    if (!c || !c->vtable) return -1;
    if (t_out) {
        const int fine = SUB * c->S_eff;
        for (int r = 0; r < c->vrows; ++r) {
            const int tf = r <= fine ? r : SUB * (c->S_eff + (r - fine));
            t_out[r] = (double)tf * c->cfg.dt / SUB;
        }
    }
    return c->vrows;
}

tdse_status tdse_set_potential_table(tdse_ctx* c, int instance, const double* V, int where, void* stream) {
    if (!c || !V) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    if (!c->vtable) return c->fail(TDSE_ESTATE, "separable-potential context: use tdse_set_potential");
    int lo, hi;
    if (!instance_range(c, instance, lo, hi)) return c->fail(TDSE_EINVAL, "instance out of range");
    if (c->vshared && instance != -1) return c->fail(TDSE_EINVAL, "shared potential table: instance must be -1");
    if (where != TDSE_HOST && where != TDSE_DEVICE) return TDSE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = where == TDSE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const size_t per = (size_t)c->vrows * c->NP;
    std::vector<double> ones(c->ntf, 1.0);
    for (int b = lo; b < hi; ++b) {
        if (!c->vshared || b == lo) {
            double* dV = c->P<double>(c->off.V0) + (size_t)b * per;
            if (c->four1d) {   // each row into the transposed layout
                double* tmp = c->P<double>(c->off.aux);
                for (int r = 0; r < c->vrows; ++r) {
                    TDSE_CK(c, cudaMemcpyAsync(tmp, V + (size_t)r * c->NP, c->NP * 8, kind, s));
                    TDSE_CK(c, launch_transpose_1d(dV + (size_t)r * c->NP, tmp, c->fs0, c->fs1, 1, 8, 1, s));
                }
            } else {
                TDSE_CK(c, cudaMemcpyAsync(dV, V, per * 8, kind, s));
            }
            TDSE_CK(c, launch_split_float(c->P<float2>(c->off.V0f) + (size_t)b * per, dV, per, s));
        }
        TDSE_CK(c, cudaMemcpyAsync(c->P<double>(c->off.tfac) + (size_t)b * c->ntf, ones.data(), c->ntf * 8,
                                   cudaMemcpyHostToDevice, s));
        c->have_V[b] = 1;
    }
    TDSE_CK(c, cudaStreamSynchronize(s));   // host sources and `ones` are released on return
    return TDSE_OK;
}

static tdse_status set_field(tdse_ctx* c, int instance, tdse_field_fn A, void* user, void* stream) {
    if (!c) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    int lo, hi;
    if (!instance_range(c, instance, lo, hi)) return c->fail(TDSE_EINVAL, "instance out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // phi(t_m), t_m = m dt/8: 8-point Gauss-Legendre on each [t_m, t_{m+1}],
    // accumulated with Neumaier's compensated summation in double (eq. phi):
    // the same bits on every host, error ~1e-16 relative to sum |parts|.
    std::vector<double> phi((size_t)c->d * c->ntf, 0.0);
    if (A) {
        std::vector<double> gx, gw;
        gauss_legendre(8, gx, gw);
        const double hs = c->cfg.dt / SUB;
        double acc[2] = {0.0, 0.0}, comp[2] = {0.0, 0.0};
        double Av[2] = {0.0, 0.0};
        for (int mm = 0; mm + 1 < c->ntf; ++mm) {
            const double t0 = (double)mm * hs, t1 = (double)(mm + 1) * hs;
            const double half = 0.5 * (t1 - t0), mid = 0.5 * (t0 + t1);
            double part[2] = {0.0, 0.0};
            for (int q = 0; q < 8; ++q) {
                A(mid + half * gx[q], Av, user);
                for (int dd = 0; dd < c->d; ++dd) part[dd] += gw[q] * Av[dd];
            }
            for (int dd = 0; dd < c->d; ++dd) {
                if (!std::isfinite(part[dd])) return c->fail(TDSE_EINVAL, "non-finite A(t)");
                const double x = part[dd] * half, t = acc[dd] + x;
                comp[dd] += std::fabs(acc[dd]) >= std::fabs(x) ? (acc[dd] - t) + x : (x - t) + acc[dd];
                acc[dd] = t;
                phi[(size_t)dd * c->ntf + mm + 1] = acc[dd] + comp[dd];
            }
        }
    }
    for (int b = lo; b < hi; ++b) {
        TDSE_CK(c, cudaMemcpyAsync(c->P<double>(c->off.phi) + (size_t)b * c->d * c->ntf, phi.data(),
                                   phi.size() * 8, cudaMemcpyHostToDevice, s));
        tdse_status st = build_phase_tables(c, b, s);
        if (st != TDSE_OK) return st;
    }
    // phi is pageable host memory: each copy has taken it before returning
    return TDSE_OK;
}

tdse_status tdse_set_vector_potential(tdse_ctx* c, int instance, tdse_field_fn A, void* user, void* stream) {
    return set_field(c, instance, A, user, stream);
}

tdse_status tdse_set_pulse(tdse_ctx* c, int instance, double A0, double omega, double Tp, const double* dir,
                           void* stream) {
    if (!c || !dir || !(Tp > 0.0) || !std::isfinite(A0) || !std::isfinite(omega)) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    int lo, hi;
    if (!instance_range(c, instance, lo, hi)) return c->fail(TDSE_EINVAL, "instance out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // phi in closed form on the device (no host pass over the fine time grid)
    const double d2[3] = {dir[0], c->d >= 2 ? dir[1] : 0.0, c->d == 3 ? dir[2] : 0.0};
    for (int b = lo; b < hi; ++b) {
        TDSE_CK(c, launch_pulse_phi(c->P<double>(c->off.phi) + (size_t)b * c->d * c->ntf, c->ntf, c->d,
                                    c->cfg.dt / SUB, A0, omega, Tp, d2, s));
        tdse_status st = build_phase_tables(c, b, s);
        if (st != TDSE_OK) return st;
    }
    return TDSE_OK;
}

tdse_status tdse_set_initial(tdse_ctx* c, int instance, const double* u0, int where, void* stream) {
    if (!c || !u0) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    int lo, hi;
    if (!instance_range(c, instance, lo, hi)) return c->fail(TDSE_EINVAL, "instance out of range");
    if (where != TDSE_HOST && where != TDSE_DEVICE) return TDSE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = where == TDSE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    for (int b = lo; b < hi; ++b) {
        if (c->fs) {
            tdse_status st = fs_set_initial(c, b, u0, kind, s);
            if (st != TDSE_OK) return st;
        } else if (c->four1d) {
            double2* tmp = c->P<double2>(c->off.aux);
            TDSE_CK(c, cudaMemcpyAsync(tmp, u0, c->NP * 16, kind, s));
            TDSE_CK(c, launch_transpose_1d(c->P<double2>(c->off.uhat) + (size_t)b * c->NP, tmp, c->fs0, c->fs1, 1, 16,
                                           1, s));
        } else {
            TDSE_CK(c, cudaMemcpyAsync(c->P<double2>(c->off.uhat) + (size_t)b * c->NP, u0, c->NP * 16, kind, s));
        }
        c->have_u0[b] = 1;
    }
    if (c->mixed && c->off.res_ncorr) {
        TDSE_CK(c, cudaMemsetAsync(c->P<int>(c->off.res_ncorr), 0, (size_t)c->B * 4, s));
        TDSE_CK(c, cudaMemsetAsync(c->P<double>(c->off.res_rho), 0, (size_t)c->B * 8, s));
    }
    if (where == TDSE_HOST) TDSE_CK(c, cudaStreamSynchronize(s));
    c->step = 0;
    c->inited = false;
    c->ip = false;
    c->res_checks = 0;
    return TDSE_OK;
}

tdse_status tdse_set_initial_batch(tdse_ctx* c, const double* u0, int where, void* stream) {
    if (!c || !u0) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    if (where != TDSE_HOST && where != TDSE_DEVICE) return TDSE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const cudaMemcpyKind kind = where == TDSE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    // the grid values of all instances are contiguous in the workspace (stride n0 n1)
    double2* dst = c->fs ? c->P<double2>(c->F.off.u) : c->P<double2>(c->off.uhat);
    if (c->four1d) {
        double2* tmp = c->P<double2>(c->off.aux);
        TDSE_CK(c, cudaMemcpyAsync(tmp, u0, (size_t)c->B * c->NP * 16, kind, s));
        TDSE_CK(c, launch_transpose_1d(dst, tmp, c->fs0, c->fs1, c->B, 16, 1, s));
    } else {
        TDSE_CK(c, cudaMemcpyAsync(dst, u0, (size_t)c->B * c->NP * 16, kind, s));
    }
    std::fill(c->have_u0.begin(), c->have_u0.end(), 1);
    if (c->mixed && c->off.res_ncorr) {
        TDSE_CK(c, cudaMemsetAsync(c->P<int>(c->off.res_ncorr), 0, (size_t)c->B * 4, s));
        TDSE_CK(c, cudaMemsetAsync(c->P<double>(c->off.res_rho), 0, (size_t)c->B * 8, s));
    }
    if (where == TDSE_HOST) TDSE_CK(c, cudaStreamSynchronize(s));
    c->step = 0;
    c->inited = false;
    c->ip = false;
    c->res_checks = 0;
    return TDSE_OK;
}

static tdse_status do_init(tdse_ctx* c, cudaStream_t s) {
    KArgs a = base_args(c);
    a.mode = MODE_INIT;
    a.out_slot = slot_of(c, 0);
    set_time(c, a, 0);
    if (c->off.tw128)
        TDSE_CK(c, launch_four_step_init(a, c->P<double2>(c->off.tw128), s));
    else
        TDSE_CK(c, run(c, a, f64_combo(c), s));
    c->inited = true;
    return TDSE_OK;
}

static tdse_status startup_step(tdse_ctx* c, int n, cudaStream_t s) {
    const size_t NPB = c->NP * c->B;
    char* chain_u = c->P<char>(c->off.chain_uhat);
    char* chain_r = c->P<char>(c->off.chain_ring);
    const double half[2] = {0.5, 0.5};
    for (int ch = 0; ch < c->L; ++ch) {
        void* cu = chain_u + (size_t)ch * NPB * 16;
        void* cr = chain_r + (size_t)ch * NPB * c->rsz;
        TDSE_CK(c, cudaMemcpyAsync(cu, c->P<void>(c->off.uhat), NPB * 16, cudaMemcpyDeviceToDevice, s));
        TDSE_CK(c, launch_copy_slot(cr, c->P<void>(c->off.ring), c->RS, slot_of(c, n - 1), c->B, c->NP, c->rsz, s));
        const int len = SUB >> ch;
        for (int i = 0; i < (1 << ch); ++i) {
            KArgs a = base_args(c);
            a.mode = MODE_STEP;
            a.uhat = cu;
            a.ring = cr;
            a.ring_slots = 1;
            a.nhist = 1;
            set_weights(a, c->cfg.dt / (double)(1 << ch), half, 2);
            a.hist_slot[0] = 0;
            a.out_slot = 0;
            a.interval[0] = startup_interval(c, n, ch, i);
            a.kin = ch;
            set_time(c, a, SUB * (n - 1) + (i + 1) * len);
            TDSE_CK(c, run(c, a, step_combo(c), s));
        }
    }
    TDSE_CK(c, launch_combine(c->P<void>(c->off.uhat), chain_u, NPB, c->L, c->rich, NPB, c->mixed, s));
    KArgs a = base_args(c);
    a.mode = MODE_REFRESH;
    a.out_slot = slot_of(c, n);
    set_time(c, a, SUB * n);
    TDSE_CK(c, run(c, a, step_combo(c), s));
    return TDSE_OK;
}

// Mixed mode: after the start-up, move the state and the ring to the
// interaction picture (v^ = u^ / E_n, r^_j = R_j / E_j).
static tdse_status enter_interaction(tdse_ctx* c, int n, cudaStream_t s) {
    int steps[8];
    float zs[16];
    for (int q = 0; q < c->RS && q < 8; ++q) {
        const int j = n - ((n - q) % c->RS + c->RS) % c->RS;
        steps[q] = j >= 0 ? j : -1;
        zs[2 * q] = j >= 0 ? c->zdither[2 * j] : 1.f;
        zs[2 * q + 1] = j >= 0 ? c->zdither[2 * j + 1] : 0.f;
    }
    KArgs a = base_args(c);
    TDSE_CK(c, launch_to_interaction(a, n, steps, zs, c->RS < 8 ? c->RS : 8, s));
    c->ip = true;
    return TDSE_OK;
}

// interaction-picture weights: c_j = mu_j / z_{nb - j} for the step nb being
// begun, d = h mu_0 / z_ne for the step ne being finished, zr = z_ne.
static void set_dither(const tdse_ctx* c, KArgs& a, int nb, int ne) {
    for (int j = 1; j < c->m; ++j) zinv(c, nb - j, c->mu[j], a.c_hi[j], a.c_lo[j]);
    zinv(c, ne, c->cfg.dt * c->mu[0], a.d_hi, a.d_lo);
    a.zr[0] = c->zdither[2 * ne];
    a.zr[1] = c->zdither[2 * ne + 1];
}

// The cluster kernel runs only when asked for: measured slower than the pass
// kernels on the 512^2 workload (1.07 against 0.52 ms per 64-instance step).
static bool use_cluster(const tdse_ctx* c) {
    return c->cl_ok && c->step_path == TDSE_PATH_CLUSTER && c->d == 2 && c->mixed;
}

static KArgs adams_args(const tdse_ctx* c, int n) {
    KArgs a = base_args(c);
    a.mode = MODE_STEP;
    a.nhist = c->m - 1;
    set_weights(a, c->cfg.dt, c->mu, c->m);
    for (int j = 1; j <= a.nhist; ++j) a.hist_slot[j - 1] = slot_of(c, n - j);
    a.out_slot = slot_of(c, n);
    if (!c->mixed)
        for (int i = 0; i < a.nhist; ++i) a.interval[i] = main_interval(c, n - i);
    a.kin = 0;
    set_time(c, a, SUB * n);
    a.ip = c->mixed ? 1 : 0;
    a.e_step = n;
    if (c->mixed) set_dither(c, a, n, n);
    return a;
}

// One pass kernel of the 2D or 3D step chain.
static cudaError_t step_part(const tdse_ctx* c, const KArgs& a, int combo, int part, cudaStream_t s) {
    return c->d == 3 ? launch_periodic3d_part(a, combo, part, s) : launch_periodic2d_part(a, combo, part, s);
}

// The launch arguments of instances [lo, hi) of a batch: every per-instance
// array advanced to instance lo (the kernels index instance b of a launch
// from these bases).
static KArgs group_args(const tdse_ctx* c, KArgs a, int lo, int hi) {
    const size_t l = (size_t)lo, NP = c->NP;
    a.B = hi - lo;
    a.uhat = static_cast<char*>(a.uhat) + l * NP * 16;
    a.ring = static_cast<char*>(a.ring) + l * a.ring_slots * NP * c->rsz;
    a.aux += l * NP;
    a.aux2 += l * NP;
    a.V0 += l * a.vstride;
    a.V0f += l * a.vstride;
    a.tfac += l * a.ntf;
    a.phi += l * (size_t)c->d * a.ntf;
    const size_t nsp1 = (size_t)c->cfg.nsteps + 1;
    if (a.q64) a.q64 += l * (size_t)c->n_int * c->ntab;
    if (a.qff) a.qff += l * (size_t)c->n_int * c->ntab;
    if (a.e2d) a.e2d += l * nsp1 * c->ntab;
    if (a.adv64) a.adv64 += l * (size_t)c->n_int * (c->nh + c->nl);
    if (a.advff) a.advff += l * (size_t)c->n_int * (c->nh + c->nl);
    if (a.a1d) a.a1d += l * nsp1 * (c->nh + c->nl);
    return a;
}

static tdse_status adams_chain_2d(tdse_ctx* c, int n0, int k, int lo, int hi, cudaStream_t s);

// k consecutive Adams steps n0+1 .. n0+k.  2D runs them as col_begin,
// (row_mid, col_fused) x (k-1), row_mid, col_end; with step groups, one such
// chain per group of instances on parallel streams.
static tdse_status adams_steps(tdse_ctx* c, int n0, int k, cudaStream_t s) {
    const int combo = step_combo(c);
    if (use_cluster(c) && c->ip) {
        const KArgs a = adams_args(c, n0 + 1);
        ClArgs ca{};
        ca.n_first = n0 + 1;
        ca.k = k;
        ca.S_eff = c->S_eff;
        ca.vrows = c->vrows;
        ca.vtable = c->vtable ? 1 : 0;
        ca.vshared = c->vshared ? 1 : 0;
        ca.tab = c->P<float>(c->off.cl_tab);
        ca.err = c->P<int>(c->off.err);
        TDSE_CK(c, launch_step2d_cluster(a, ca, c->cl, s));
        return TDSE_OK;
    }
    if ((c->d == 1 && !c->four1d) || k == 1) {
        for (int n = n0 + 1; n <= n0 + k; ++n) TDSE_CK(c, run(c, adams_args(c, n), combo, s));
        return TDSE_OK;
    }
    const int G = c->step_groups < c->B ? c->step_groups : c->B;
    if (G <= 1) return adams_chain_2d(c, n0, k, 0, c->B, s);
    if ((int)c->group_streams.size() < G) {
        if (!c->group_fork) TDSE_CK(c, cudaEventCreateWithFlags(&c->group_fork, cudaEventDisableTiming));
        while ((int)c->group_streams.size() < G) {
            cudaStream_t gs = nullptr;
            cudaEvent_t ge = nullptr;
            TDSE_CK(c, cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
            c->group_streams.push_back(gs);
            TDSE_CK(c, cudaEventCreateWithFlags(&ge, cudaEventDisableTiming));
            c->group_join.push_back(ge);
        }
    }
    // The groups' launches are issued step by step, alternating between the
    // streams: enqueued one whole chain after another, a long run would fill
    // the launch queue with one group's kernels and the groups would not overlap.
    TDSE_CK(c, cudaEventRecord(c->group_fork, s));
    std::vector<int> lo(G), hi(G);
    for (int g = 0; g < G; ++g) {
        lo[g] = (int)((long long)c->B * g / G);
        hi[g] = (int)((long long)c->B * (g + 1) / G);
        TDSE_CK(c, cudaStreamWaitEvent(c->group_streams[g], c->group_fork, 0));
    }
    for (int g = 0; g < G; ++g)
        TDSE_CK(c, step_part(c, group_args(c, adams_args(c, n0 + 1), lo[g], hi[g]), combo, PART_COL_BEGIN,
                                          c->group_streams[g]));
    for (int n = n0 + 1; n < n0 + k; ++n) {
        const KArgs r = adams_args(c, n);
        KArgs f = adams_args(c, n + 1);     // as in adams_chain_2d
        f.out_slot = slot_of(c, n);
        f.e_step = n;
        f.e_next = n + 1;
        if (c->mixed) set_dither(c, f, n + 1, n);
        for (int g = 0; g < G; ++g) {
            TDSE_CK(c, step_part(c, group_args(c, r, lo[g], hi[g]), combo, PART_ROW_MID, c->group_streams[g]));
            TDSE_CK(c, step_part(c, group_args(c, f, lo[g], hi[g]), combo, PART_COL_FUSED,
                                              c->group_streams[g]));
        }
    }
    const KArgs last = adams_args(c, n0 + k);
    for (int g = 0; g < G; ++g) {
        const KArgs lg = group_args(c, last, lo[g], hi[g]);
        TDSE_CK(c, step_part(c, lg, combo, PART_ROW_MID, c->group_streams[g]));
        TDSE_CK(c, step_part(c, lg, combo, PART_COL_END, c->group_streams[g]));
        TDSE_CK(c, cudaEventRecord(c->group_join[g], c->group_streams[g]));
        TDSE_CK(c, cudaStreamWaitEvent(s, c->group_join[g], 0));
    }
    return TDSE_OK;
}

// The 2D pass chain of k Adams steps for instances [lo, hi).
static tdse_status adams_chain_2d(tdse_ctx* c, int n0, int k, int lo, int hi, cudaStream_t s) {
    const int combo = step_combo(c);
    auto A = [&](int n) { return group_args(c, adams_args(c, n), lo, hi); };
    TDSE_CK(c, step_part(c, A(n0 + 1), combo, PART_COL_BEGIN, s));
    for (int n = n0 + 1; n < n0 + k; ++n) {
        TDSE_CK(c, step_part(c, A(n), combo, PART_ROW_MID, s));
        KArgs f = A(n + 1);                 // history slots, intervals and E of the next step ...
        f.out_slot = slot_of(c, n);         // ... ring slot and E of the step being finished
        f.e_step = n;
        f.e_next = n + 1;
        if (c->mixed) set_dither(c, f, n + 1, n);
        TDSE_CK(c, step_part(c, f, combo, PART_COL_FUSED, s));
    }
    const KArgs last = A(n0 + k);
    TDSE_CK(c, step_part(c, last, combo, PART_ROW_MID, s));
    TDSE_CK(c, step_part(c, last, combo, PART_COL_END, s));
    return TDSE_OK;
}

// FP64 residual of the implicit equation for the step just completed, and the
// FP64 redo of that step where it exceeds the tolerance (resid.cu).
static tdse_status residual_check(tdse_ctx* c, cudaStream_t s) {
    ResArgs r{};
    r.a = base_args(c);
    set_time(c, r.a, SUB * c->step);
    r.n = c->step;
    r.slot = slot_of(c, c->step);
    r.z[0] = c->zdither[2 * c->step];
    r.z[1] = c->zdither[2 * c->step + 1];
    r.hmu0 = c->cfg.dt * c->mu[0];
    r.tol = c->res_tol;
    r.sums = c->P<double>(c->off.res_sums);
    r.flags = c->P<int>(c->off.res_flags);
    r.rho = c->P<double>(c->off.res_rho);
    r.ncorr = c->P<int>(c->off.res_ncorr);
    TDSE_CK(c, launch_residual_check(r, true, s));
    ++c->res_checks;
    return TDSE_OK;
}

tdse_status tdse_step(tdse_ctx* c, int nsteps, void* stream) {
    if (!c) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    if (nsteps < 0) return c->fail(TDSE_EINVAL, "negative step count");
    if (c->step + nsteps > c->cfg.nsteps) return c->fail(TDSE_EINVAL, "beyond the nsteps the tables cover");
    for (int b = 0; b < c->B; ++b)
        if (!c->have_V[b] || !c->have_u0[b]) return c->fail(TDSE_ESTATE, "instance lacks V or u0");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (nsteps == 0) return TDSE_OK;
    if (c->fs) return fs_steps(c, nsteps, s);
    if (!c->inited) {
        tdse_status st = do_init(c, s);
        if (st != TDSE_OK) return st;
    }
    int k = 0;
    while (k < nsteps) {
        const int n = c->step + 1;
        if (n <= c->S) {
            tdse_status st = startup_step(c, n, s);
            if (st != TDSE_OK) return st;
            c->step = n;
            ++k;
            continue;
        }
        if (c->mixed && !c->ip) {
            tdse_status st = enter_interaction(c, c->step, s);
            if (st != TDSE_OK) return st;
        }
        int run_len = nsteps - k;
        if (c->mixed && c->res_every > 0) {   // stop at the next step to check
            const int to_check = c->res_every - c->step % c->res_every;
            if (to_check < run_len) run_len = to_check;
        }
        tdse_status st = adams_steps(c, c->step, run_len, s);
        if (st != TDSE_OK) return st;
        c->step += run_len;
        k += run_len;
        if (c->mixed && c->res_every > 0 && c->step % c->res_every == 0) {
            st = residual_check(c, s);
            if (st != TDSE_OK) return st;
        }
    }
    return TDSE_OK;
}

tdse_status tdse_solve_to(tdse_ctx* c, double T, void* stream) {
    if (!c || !std::isfinite(T) || T < 0) return TDSE_EINVAL;
    const long long target = llround(T / c->cfg.dt);
    if (target < c->step) return c->fail(TDSE_EINVAL, "T is before the current time");
    if (target > c->cfg.nsteps) return c->fail(TDSE_EINVAL, "T beyond the nsteps the tables cover");
    return tdse_step(c, (int)(target - c->step), stream);
}

tdse_status tdse_read_u(tdse_ctx* c, int instance, double* u_out, int where, void* stream) {
    if (!c || !u_out) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    int lo, hi;
    if (!instance_range(c, instance, lo, hi)) return c->fail(TDSE_EINVAL, "instance out of range");
    if (where != TDSE_HOST && where != TDSE_DEVICE) return TDSE_EINVAL;
    for (int b = lo; b < hi; ++b)
        if (!c->have_u0[b]) return c->fail(TDSE_ESTATE, "instance has no initial state");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nb = (size_t)(hi - lo);
    if (c->fs) {
        tdse_status st = fs_read_u(c, lo, hi, u_out, where == TDSE_HOST ? cudaMemcpyDeviceToHost
                                                                      : cudaMemcpyDeviceToDevice, s);
        if (st != TDSE_OK) return st;
        if (where == TDSE_HOST) TDSE_CK(c, cudaStreamSynchronize(s));
        return TDSE_OK;
    }
    const double2* src;
    if (!c->inited) {
        src = c->P<double2>(c->off.uhat) + (size_t)lo * c->NP;    // u0 still parked in physical form
    } else {
        KArgs a = base_args(c);
        a.mode = MODE_READ;
        a.B = (int)nb;
        a.uhat = c->P<char>(c->off.uhat) + (size_t)lo * c->NP * 16;
        a.phi = c->P<double>(c->off.phi) + (size_t)lo * c->d * c->ntf;
        a.ip = c->ip ? 1 : 0;
        a.e_step = c->step;
        if (c->off.tw128)
            TDSE_CK(c, launch_four_step_read(a, c->P<double2>(c->off.tw128), s));
        else
            TDSE_CK(c, run(c, a, f64_combo(c), s));
        src = a.aux2;
    }
    if (c->four1d) {   // the passes' transposed layout -> natural order
        double2* nat = c->P<double2>(c->off.aux);
        TDSE_CK(c, launch_transpose_1d(nat, src, c->fs0, c->fs1, (int)nb, 16, 0, s));
        src = nat;
    }
    const cudaMemcpyKind kind = where == TDSE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    TDSE_CK(c, cudaMemcpyAsync(u_out, src, nb * c->NP * 16, kind, s));
    if (where == TDSE_HOST) TDSE_CK(c, cudaStreamSynchronize(s));
    return TDSE_OK;
}

tdse_status tdse_check_finite(tdse_ctx* c, void* stream) {
    if (!c) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!c->fs && c->off.err) {
        int ew = 0;
        TDSE_CK(c, cudaMemcpyAsync(&ew, c->P<int>(c->off.err), sizeof(int), cudaMemcpyDeviceToHost, s));
        TDSE_CK(c, cudaStreamSynchronize(s));
        if (ew) return c->fail(TDSE_ETIMEOUT, "a bounded wait in a step kernel gave up: results are invalid");
    }
    int* cnt = c->P<int>(c->off.scratch);
    TDSE_CK(c, cudaMemsetAsync(cnt, 0, sizeof(int), s));
    const size_t nmodes = c->fs ? c->F.NM : c->NP;
    // the free-space mode state is FP64 in both precisions
    TDSE_CK(c, launch_count_nonfinite(c->P<void>(c->off.uhat), nmodes * c->B * 2, c->mixed && c->inited && !c->fs,
                                      cnt, s));
    int h = 0;
    TDSE_CK(c, cudaMemcpyAsync(&h, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    TDSE_CK(c, cudaStreamSynchronize(s));
    if (h) return c->fail(TDSE_ENONFINITE, "non-finite values in the mode state");
    return TDSE_OK;
}

tdse_status tdse_read_modes(tdse_ctx* c, int instance, double* u_out, int where, void* stream) {
    if (!c || !u_out) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    if (c->mixed && !c->fs) return c->fail(TDSE_EUNSUPPORTED, "periodic mode state is FP64 only in TDSE_FP64");
    if (!c->inited) return c->fail(TDSE_ESTATE, "no step taken yet");
    int lo, hi;
    if (!instance_range(c, instance, lo, hi)) return c->fail(TDSE_EINVAL, "instance out of range");
    if (where != TDSE_HOST && where != TDSE_DEVICE) return TDSE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t nm = c->fs ? c->F.NM : c->NP;
    const cudaMemcpyKind kind = where == TDSE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    TDSE_CK(c, cudaMemcpyAsync(u_out, c->P<double2>(c->off.uhat) + (size_t)lo * nm, (size_t)(hi - lo) * nm * 16,
                               kind, s));
    if (where == TDSE_HOST) TDSE_CK(c, cudaStreamSynchronize(s));
    return TDSE_OK;
}

tdse_status tdse_set_residual_check(tdse_ctx* c, int every, double tol) {
    if (!c) return TDSE_EINVAL;
    if (every < 0 || !(tol >= 0.0)) return c->fail(TDSE_EINVAL, "every >= 0 and tol >= 0 required");
    if (every > 0 && !c->mixed) return c->fail(TDSE_EUNSUPPORTED, "residual check: TDSE_MIXED only");
    if (every > 0 && !c->fs && !residual_supported(c->d, c->n0, c->n1))
        return c->fail(TDSE_EUNSUPPORTED, "residual check: n up to 8192 (1D) or 1024 per dimension (2D)");
    c->res_every = every;
    c->res_tol = tol;
    return TDSE_OK;
}

tdse_status tdse_residual_report(tdse_ctx* c, double* rho, int* corrections, int* checks, void* stream) {
    if (!c) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    if (checks) *checks = c->res_checks;
    if (!c->mixed || !c->off.res_rho) return TDSE_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (rho) TDSE_CK(c, cudaMemcpyAsync(rho, c->P<double>(c->off.res_rho), (size_t)c->B * 8, cudaMemcpyDeviceToHost, s));
    if (corrections)
        TDSE_CK(c, cudaMemcpyAsync(corrections, c->P<int>(c->off.res_ncorr), (size_t)c->B * 4, cudaMemcpyDeviceToHost,
                                   s));
    TDSE_CK(c, cudaStreamSynchronize(s));
    if (rho && c->res_checks > 0)
        for (int b = 0; b < c->B; ++b)
            if (!std::isfinite(rho[b])) return c->fail(TDSE_ENONFINITE, "non-finite residual");
    return TDSE_OK;
}

// ---- checkpoint: header, then the whole workspace
namespace {
constexpr char kCkptMagic[8] = {'T', 'D', 'S', 'E', 'C', 'K', 'P', '2'};
struct CkptHeader {
    char magic[8];
    int dim, bc, n0, n1, n2, batch, nsteps, order, startup, precision, nu0, nu1, alpert_p, gauss_q, n_r;
    double dt, H;
    unsigned long long ws_bytes;
    int step, inited, ip, res_every, res_checks, nu2;
    double res_tol;
};
void fill_header(const tdse_ctx* c, CkptHeader& h) {
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kCkptMagic, 8);
    const tdse_config& g = c->cfg;
    h.dim = g.dim; h.bc = g.bc; h.n0 = g.n[0]; h.n1 = g.dim >= 2 ? g.n[1] : 1; h.n2 = g.dim == 3 ? g.n_z : 1;
    h.batch = g.batch;
    h.nsteps = g.nsteps; h.order = g.order; h.startup = c->S; h.precision = g.precision;
    if (g.bc == TDSE_FREE) {
        h.nu0 = g.nu[0]; h.nu1 = g.dim >= 2 ? g.nu[1] : 0; h.nu2 = g.dim == 3 ? g.nu_z : 0; h.alpert_p = g.alpert_p; h.gauss_q = g.gauss_q;
        h.n_r = g.n_r; h.H = g.H;
    }
    h.dt = g.dt;
    h.ws_bytes = c->ws_need;
    h.step = c->step; h.inited = c->inited; h.ip = c->ip;
    h.res_every = c->res_every; h.res_checks = c->res_checks; h.res_tol = c->res_tol;
}
}  // namespace

tdse_status tdse_save(tdse_ctx* c, void* blob, size_t* size, void* stream) {
    if (!c || !size) return TDSE_EINVAL;
    const size_t need = sizeof(CkptHeader) + 2 * (size_t)c->B + c->ws_need;
    if (!blob) {
        *size = need;
        return TDSE_OK;
    }
    if (*size < need) return c->fail(TDSE_EINVAL, "checkpoint buffer smaller than the size tdse_save reports");
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CkptHeader h;
    fill_header(c, h);
    char* out = static_cast<char*>(blob);
    std::memcpy(out, &h, sizeof(h));
    for (int b = 0; b < c->B; ++b) {
        out[sizeof(h) + 2 * b] = c->have_V[b];
        out[sizeof(h) + 2 * b + 1] = c->have_u0[b];
    }
    TDSE_CK(c, cudaMemcpyAsync(out + sizeof(h) + 2 * (size_t)c->B, c->ws, c->ws_need, cudaMemcpyDeviceToHost, s));
    TDSE_CK(c, cudaStreamSynchronize(s));
    *size = need;
    return TDSE_OK;
}

tdse_status tdse_load(tdse_ctx* c, const void* blob, size_t size, void* stream) {
    if (!c || !blob) return TDSE_EINVAL;
    if (!c->ws) return c->fail(TDSE_ESTATE, "workspace not bound");
    const size_t need = sizeof(CkptHeader) + 2 * (size_t)c->B + c->ws_need;
    if (size < need) return c->fail(TDSE_EINVAL, "checkpoint too short");
    CkptHeader h, mine;
    std::memcpy(&h, blob, sizeof(h));
    fill_header(c, mine);
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0) return c->fail(TDSE_EINVAL, "not a checkpoint of this library");
    const bool same = h.dim == mine.dim && h.bc == mine.bc && h.n0 == mine.n0 && h.n1 == mine.n1 && h.n2 == mine.n2 &&
                      h.batch == mine.batch && h.nsteps == mine.nsteps && h.order == mine.order &&
                      h.startup == mine.startup && h.precision == mine.precision && h.nu0 == mine.nu0 &&
                      h.nu1 == mine.nu1 && h.alpert_p == mine.alpert_p && h.gauss_q == mine.gauss_q &&
                      h.n_r == mine.n_r && h.dt == mine.dt && h.H == mine.H && h.ws_bytes == mine.ws_bytes;
    if (!same) return c->fail(TDSE_EINVAL, "checkpoint of a different configuration");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const char* in = static_cast<const char*>(blob);
    TDSE_CK(c, cudaMemcpyAsync(c->ws, in + sizeof(h) + 2 * (size_t)c->B, c->ws_need, cudaMemcpyHostToDevice, s));
    TDSE_CK(c, cudaStreamSynchronize(s));
    for (int b = 0; b < c->B; ++b) {
        c->have_V[b] = in[sizeof(h) + 2 * b];
        c->have_u0[b] = in[sizeof(h) + 2 * b + 1];
    }
    c->step = h.step;
    c->inited = h.inited != 0;
    c->ip = h.ip != 0;
    c->res_every = h.res_every;
    c->res_checks = h.res_checks;
    c->res_tol = h.res_tol;
    return TDSE_OK;
}

tdse_status tdse_set_step_path(tdse_ctx* c, int path) {
    if (!c) return TDSE_EINVAL;
    if (path != TDSE_PATH_AUTO && path != TDSE_PATH_PASSES && path != TDSE_PATH_CLUSTER)
        return c->fail(TDSE_EINVAL, "unknown step path");
    if (path == TDSE_PATH_CLUSTER && !(c->cl_ok && c->d == 2 && c->mixed && !c->fs))
        return c->fail(TDSE_EUNSUPPORTED, "cluster step path: 2D periodic TDSE_MIXED 512 x 512 on a device that runs "
                                          "16-CTA clusters, after tdse_bind_workspace");
    c->step_path = path;
    return TDSE_OK;
}

tdse_status tdse_set_step_groups(tdse_ctx* c, int groups) {
    if (!c) return TDSE_EINVAL;
    if (groups < 1 || groups > 64) return c->fail(TDSE_EINVAL, "step groups: 1..64");
    c->step_groups = groups;
    return TDSE_OK;
}

int tdse_step_path(const tdse_ctx* c) {
    if (!c) return -1;
    return (!c->fs && use_cluster(c)) ? TDSE_PATH_CLUSTER : TDSE_PATH_PASSES;
}

tdse_status tdse_describe_steps(const tdse_ctx* c, char* buf, size_t len) {
    if (!c || !buf || len == 0) return TDSE_EINVAL;
    int n;
    if (!c->fs && use_cluster(c))
        n = std::snprintf(buf, len,
                          "{\"path\": \"cluster\", \"clusters\": %d, \"ctas_per_cluster\": %d, \"threads\": %d, "
                          "\"smem_bytes\": %d}",
                          c->cl.clusters, CL_Q, step2d_cluster_threads(), step2d_cluster_smem());
    else if (!c->fs && c->d == 1 && !c->four1d)   // one CTA per instance
        n = std::snprintf(buf, len, "{\"path\": \"cta\", \"shape\": %d, \"threads\": %d}", c->shape1d,
                          c->mixed ? periodic1d_f32_threads(c->n0, c->shape1d) : 0);
    else if (c->four1d)
        n = std::snprintf(buf, len, "{\"path\": \"passes\", \"groups\": %d, \"four_step\": [%d, %d]}",
                          c->step_groups < c->B ? c->step_groups : c->B, c->fs0, c->fs1);
    else
        n = std::snprintf(buf, len, "{\"path\": \"passes\", \"groups\": %d}",
                          c->d >= 2 && !c->fs ? (c->step_groups < c->B ? c->step_groups : c->B) : 1);
    return (n < 0 || (size_t)n >= len) ? TDSE_EINVAL : TDSE_OK;
}

int tdse_step_index(const tdse_ctx* c) { return c ? c->step : -1; }
double tdse_time(const tdse_ctx* c) { return c ? c->step * c->cfg.dt : 0.0; }

const char* tdse_last_error(const tdse_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

void tdse_destroy(tdse_ctx* c) { delete c; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Uneven batches: one persistent launch per Adams step for all members.
struct tdse_batch {
    std::vector<tdse_ctx*> m;
    std::vector<int> var;           // launch variant per member
    std::vector<int> per;           // instances per work item per member (<= MULTI_CTA / T)
    int grid = 0;                   // persistent CTAs
    int sms = 0;
    bool tuned = false;
    size_t smem = 0;
    std::vector<MultiItem> items;
    MultiArgs1D args{};             // reused launch argument block (22 KB)
    // Adams phase: 0 = one fused persistent launch per step for all members;
    // 1 = each member's own single-size kernel on its own stream (forked from
    // and joined to the caller's stream; parallel branches of the graph)
    int mode = 0;
    float fused_ms = 0, stream_ms = 0;   // tuner's per-step times of the two modes
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    struct Graph {
        int from, n;
        bool inited;
        cudaGraphExec_t exec;
        std::vector<int> step;
        std::vector<char> inited_after, ip_after;
    };
    std::vector<Graph> graphs;
    std::string err;
    tdse_status fail(tdse_status s, const std::string& msg) {
        err = msg;
        return s;
    }
};

static int default_threads_1d(int n) { return n / 8 < 32 ? 32 : (n / 8 > MULTI_CTA ? MULTI_CTA : n / 8); }

static void drop_graphs(tdse_batch* b) {
    for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

// Work items (cost-descending so that the CTA-strided assignment starts with
// the largest) and the launch's shared memory.
static tdse_status build_items(tdse_batch* b) {
    b->items.clear();
    b->smem = 0;
    for (size_t g = 0; g < b->m.size(); ++g) {
        const tdse_ctx* c = b->m[g];
        const int var = b->var[g];
        const int per = b->per[g];
        if (var < 0) continue;              // four-step layout: its own pass chain beside the launch
        for (int b0 = 0; b0 < c->B; b0 += per) {
            MultiItem it{};
            it.g = (unsigned char)g;
            it.var = (unsigned char)var;
            it.count = (unsigned short)std::min(per, c->B - b0);
            it.b0 = b0;
            b->items.push_back(it);
            b->smem = std::max(b->smem, multi_item_smem(var, it.count));
        }
    }
    if (b->items.size() > (size_t)MULTI_MAX_ITEMS) return b->fail(TDSE_EINVAL, "more than 1536 work items");
    auto cost = [&](const MultiItem& it) {
        const double n = multi_variant_n(it.var);
        return n * std::log2(n) * it.count;
    };
    std::stable_sort(b->items.begin(), b->items.end(),
                     [&](const MultiItem& x, const MultiItem& y) { return cost(x) > cost(y); });
    b->args.nitems = (int)b->items.size();
    b->args.next = b->m[0]->P<int>(b->m[0]->off.scratch) + 1;   // word 0 is tdse_check_finite's counter
    std::copy(b->items.begin(), b->items.end(), b->args.items);
    return TDSE_OK;
}

static int default_grid(tdse_batch* b) {
    const int occ = std::max(1, multi_occupancy(b->smem));
    return std::max(1, std::min((int)b->items.size(), b->sms * occ));
}

static tdse_status batch_prepare(tdse_batch* b) {
    cudaError_t e = multi_prepare(b->smem);
    for (tdse_ctx* c : b->m) {
        if (c->four1d) continue;            // the 2D pass kernels set their attributes at first launch
        if (e == cudaSuccess) e = periodic1d_prepare(c->n0, COMBO_F32);
        if (e == cudaSuccess && !c->off.tw128) e = periodic1d_prepare(c->n0, COMBO_F64_R32);
    }
    if (e != cudaSuccess) return b->fail(TDSE_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    return TDSE_OK;
}

static tdse_status member_status(tdse_batch* b, tdse_ctx* c, tdse_status st) {
    if (st != TDSE_OK) return b->fail(st, "member: " + c->err);
    return TDSE_OK;
}

// Launches of Adams step n of the run n0+1 .. n0+k of a member in the
// four-step layout: the step's part of the 2D pass chain (adams_chain_2d).
static cudaError_t four1d_chain_step(const tdse_ctx* c, int n0, int k, int n, cudaStream_t s) {
    const int combo = step_combo(c);
    auto A = [&](int m) { return group_args(c, adams_args(c, m), 0, c->B); };
    cudaError_t e = cudaSuccess;
    if (n == n0 + 1) e = step_part(c, A(n), combo, PART_COL_BEGIN, s);
    if (e == cudaSuccess) e = step_part(c, A(n), combo, PART_ROW_MID, s);
    if (e != cudaSuccess) return e;
    if (n < n0 + k) {
        KArgs f = A(n + 1);                 // as in adams_chain_2d
        f.out_slot = slot_of(c, n);
        f.e_step = n;
        f.e_next = n + 1;
        if (c->mixed) set_dither(c, f, n + 1, n);
        return step_part(c, f, combo, PART_COL_FUSED, s);
    }
    return step_part(c, A(n), combo, PART_COL_END, s);
}

// Adams steps n0+1 .. n0+k: each step one persistent launch for the members
// of one CTA per instance; members in the four-step layout run their pass
// chains on their own streams beside it (forked from and joined to s).
static tdse_status batch_adams(tdse_batch* b, int n0, int k, int grid, cudaStream_t s) {
    bool side = false;
    for (tdse_ctx* c : b->m) side = side || c->four1d;
    cudaError_t e = side ? cudaEventRecord(b->fork, s) : cudaSuccess;
    for (size_t g = 0; g < b->m.size() && e == cudaSuccess; ++g)
        if (b->m[g]->four1d) e = cudaStreamWaitEvent(b->streams[g], b->fork, 0);
    for (int n = n0 + 1; n <= n0 + k && e == cudaSuccess; ++n) {
        for (size_t g = 0; g < b->m.size() && e == cudaSuccess; ++g) {
            if (b->m[g]->four1d) e = four1d_chain_step(b->m[g], n0, k, n, b->streams[g]);
            else b->args.args[g] = adams_args(b->m[g], n);
        }
        if (e == cudaSuccess) e = launch_periodic1d_multi(b->args, grid, b->smem, s);
    }
    for (size_t g = 0; g < b->m.size() && side; ++g) {   // always join, so that a capture can end
        if (!b->m[g]->four1d) continue;
        cudaError_t j = cudaEventRecord(b->join[g], b->streams[g]);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(s, b->join[g], 0);
        if (e == cudaSuccess) e = j;
    }
    if (e != cudaSuccess) return b->fail(TDSE_ECUDA, std::string("fused step: ") + cudaGetErrorString(e));
    for (tdse_ctx* c : b->m) c->step = n0 + k;
    return TDSE_OK;
}

// Adams steps n0+1 .. n0+k of every member, each member on its own stream.
static tdse_status batch_adams_streams(tdse_batch* b, int n0, int k, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(b->fork, s);
    for (size_t g = 0; g < b->m.size() && e == cudaSuccess; ++g) e = cudaStreamWaitEvent(b->streams[g], b->fork, 0);
    for (int n = n0 + 1; n <= n0 + k && e == cudaSuccess; ++n)
        for (size_t g = 0; g < b->m.size() && e == cudaSuccess; ++g)
            e = b->m[g]->four1d ? four1d_chain_step(b->m[g], n0, k, n, b->streams[g])
                                : run(b->m[g], adams_args(b->m[g], n), step_combo(b->m[g]), b->streams[g]);
    for (size_t g = 0; g < b->m.size(); ++g) {   // always join, so that a capture can end
        cudaError_t j = cudaEventRecord(b->join[g], b->streams[g]);
        if (j == cudaSuccess) j = cudaStreamWaitEvent(s, b->join[g], 0);
        if (e == cudaSuccess) e = j;
    }
    if (e != cudaSuccess) return b->fail(TDSE_ECUDA, std::string("member streams: ") + cudaGetErrorString(e));
    for (tdse_ctx* c : b->m) c->step = n0 + k;
    return TDSE_OK;
}

// The launch sequence of nsteps steps (no capture logic).
static tdse_status batch_run(tdse_batch* b, int nsteps, cudaStream_t s) {
    for (tdse_ctx* c : b->m)
        if (!c->inited) {
            tdse_status st = member_status(b, c, do_init(c, s));
            if (st != TDSE_OK) return st;
        }
    int k = 0;
    while (k < nsteps) {
        const int n = b->m[0]->step + 1;
        if (n <= b->m[0]->S) {
            for (tdse_ctx* c : b->m) {
                tdse_status st = member_status(b, c, startup_step(c, n, s));
                if (st != TDSE_OK) return st;
                c->step = n;
            }
            ++k;
            continue;
        }
        for (tdse_ctx* c : b->m)
            if (!c->ip) {
                tdse_status st = member_status(b, c, enter_interaction(c, c->step, s));
                if (st != TDSE_OK) return st;
            }
        if (b->mode == 1) {
            tdse_status st = batch_adams_streams(b, n - 1, nsteps - k, s);
            if (st != TDSE_OK) return st;
            k = nsteps;
            continue;
        }
        tdse_status st = batch_adams(b, n - 1, nsteps - k, b->grid, s);
        if (st != TDSE_OK) return st;
        k = nsteps;
    }
    return TDSE_OK;
}

static tdse_status batch_check(tdse_batch* b, int nsteps) {
    const tdse_ctx* c0 = b->m[0];
    for (tdse_ctx* c : b->m) {
        if (!c->ws) return b->fail(TDSE_ESTATE, "member workspace not bound");
        for (int i = 0; i < c->B; ++i)
            if (!c->have_V[i] || !c->have_u0[i]) return b->fail(TDSE_ESTATE, "member instance lacks V or u0");
        if (c->step != c0->step || c->inited != c0->inited || c->ip != c0->ip)
            return b->fail(TDSE_ESTATE, "members are not at the same step");
        if (c->step + nsteps > c->cfg.nsteps) return b->fail(TDSE_EINVAL, "beyond the nsteps the tables cover");
    }
    return TDSE_OK;
}

extern "C" {

tdse_status tdse_set_shape_1d(tdse_ctx* c, int shape) {
    if (!c) return TDSE_EINVAL;
    if (shape != 0 && shape != 1) return c->fail(TDSE_EINVAL, "shape must be 0 or 1");
    if (c->fs || c->d != 1 || !c->mixed || c->four1d || periodic1d_f32_threads(c->n0, shape) == 0)
        return c->fail(TDSE_EUNSUPPORTED, "launch shapes: 1D periodic TDSE_MIXED, shape 1 for n >= 512");
    c->shape1d = shape;
    return TDSE_OK;
}

int tdse_shape_1d(const tdse_ctx* c) { return c ? c->shape1d : -1; }

tdse_status tdse_batch_create(tdse_ctx* const* members, int count, tdse_batch** out) {
    if (!members || !out || count < 1) return TDSE_EINVAL;
    *out = nullptr;
    if (count > MULTI_MAX_GROUPS) return TDSE_EINVAL;
    const tdse_ctx* c0 = members[0];
    if (!c0) return TDSE_EINVAL;
    for (int g = 0; g < count; ++g) {
        const tdse_ctx* c = members[g];
        if (!c || !c->ws) return TDSE_EINVAL;
        for (int h = 0; h < g; ++h)
            if (members[h] == c) return TDSE_EINVAL;
        if (c->fs || c->d != 1 || !c->mixed) return TDSE_EUNSUPPORTED;
        if (c->cfg.dt != c0->cfg.dt || c->cfg.nsteps != c0->cfg.nsteps || c->cfg.order != c0->cfg.order ||
            c->S != c0->S)
            return TDSE_EINVAL;
        if (!c->four1d && multi_variant(c->n0, default_threads_1d(c->n0)) < 0) return TDSE_EUNSUPPORTED;
    }
    tdse_batch* b = new (std::nothrow) tdse_batch();
    if (!b) return TDSE_ENOMEM;
    b->m.assign(members, members + count);
    for (tdse_ctx* c : b->m) {
        b->var.push_back(c->four1d ? -1 : multi_variant(c->n0, default_threads_1d(c->n0)));
        b->per.push_back(c->four1d ? 0 : MULTI_CTA / default_threads_1d(c->n0));
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        b->sms = 1;
    if (build_items(b) != TDSE_OK) {
        delete b;
        return TDSE_EINVAL;
    }
    if (batch_prepare(b) != TDSE_OK) {
        delete b;
        return TDSE_ECUDA;
    }
    b->grid = default_grid(b);
    b->streams.assign(b->m.size(), nullptr);
    b->join.assign(b->m.size(), nullptr);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (size_t g = 0; g < b->m.size() && ok; ++g)
        ok = cudaStreamCreateWithFlags(&b->streams[g], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[g], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        tdse_batch_destroy(b);
        return TDSE_ECUDA;
    }
    *out = b;
    return TDSE_OK;
}

tdse_status tdse_batch_step(tdse_batch* b, int nsteps, void* stream) {
    if (!b) return TDSE_EINVAL;
    if (nsteps < 0) return b->fail(TDSE_EINVAL, "negative step count");
    tdse_status st = batch_check(b, nsteps);
    if (st != TDSE_OK || nsteps == 0) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (s == nullptr || s == cudaStreamLegacy) return batch_run(b, nsteps, s);   // not capturable
    const int from = b->m[0]->step;
    const bool inited = b->m[0]->inited;
    for (auto& g : b->graphs)
        if (g.from == from && g.n == nsteps && g.inited == inited) {
            cudaError_t e = cudaGraphLaunch(g.exec, s);
            if (e != cudaSuccess) return b->fail(TDSE_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
            for (size_t i = 0; i < b->m.size(); ++i) {
                b->m[i]->step = g.step[i];
                b->m[i]->inited = g.inited_after[i];
                b->m[i]->ip = g.ip_after[i];
            }
            return TDSE_OK;
        }
    st = batch_prepare(b);
    if (st != TDSE_OK) return st;
    std::vector<int> step0;
    std::vector<char> init0, ip0;
    for (tdse_ctx* c : b->m) {
        step0.push_back(c->step);
        init0.push_back(c->inited);
        ip0.push_back(c->ip);
    }
    auto restore = [&]() {
        for (size_t i = 0; i < b->m.size(); ++i) {
            b->m[i]->step = step0[i];
            b->m[i]->inited = init0[i];
            b->m[i]->ip = ip0[i];
        }
    };
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return b->fail(TDSE_ECUDA, std::string("begin capture: ") + cudaGetErrorString(e));
    st = batch_run(b, nsteps, s);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (st != TDSE_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        restore();
        return st != TDSE_OK ? st : b->fail(TDSE_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
    }
    tdse_batch::Graph g{from, nsteps, inited, nullptr, {}, {}, {}};
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        restore();
        return b->fail(TDSE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    for (tdse_ctx* c : b->m) {
        g.step.push_back(c->step);
        g.inited_after.push_back(c->inited);
        g.ip_after.push_back(c->ip);
    }
    b->graphs.push_back(g);
    e = cudaGraphLaunch(g.exec, s);
    if (e != cudaSuccess) return b->fail(TDSE_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return TDSE_OK;
}

tdse_status tdse_batch_tune(tdse_batch* b, int trial_steps, void* stream) {
    if (!b || trial_steps < 1) return TDSE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    tdse_status st = batch_check(b, 0);
    if (st != TDSE_OK) return st;
    drop_graphs(b);
    // reach the Adams phase (start of every member, then the change of frame)
    const int S = b->m[0]->S;
    if (b->m[0]->step < S || !b->m[0]->inited) {
        st = batch_run(b, S - b->m[0]->step, s);
        if (st != TDSE_OK) return st;
    }
    for (tdse_ctx* c : b->m)
        if (!c->ip) {
            st = member_status(b, c, enter_interaction(c, c->step, s));
            if (st != TDSE_OK) return st;
        }
    if (b->m[0]->step >= b->m[0]->cfg.nsteps) return b->fail(TDSE_EINVAL, "no step left to time");
    const int n = b->m[0]->step + 1;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return b->fail(TDSE_ECUDA, "event create");
    // time `trial_steps` launches of step n (state is overwritten repeatedly)
    auto timed = [&](float& ms) -> tdse_status {
        tdse_status r = build_items(b);
        if (r != TDSE_OK) return r;
        r = batch_prepare(b);
        if (r != TDSE_OK) return r;
        r = batch_adams(b, n - 1, 1, b->grid, s);
        if (r != TDSE_OK) return r;
        cudaEventRecord(e0, s);
        for (int i = 0; i < trial_steps; ++i) {
            r = batch_adams(b, n - 1, 1, b->grid, s);
            if (r != TDSE_OK) return r;
        }
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return b->fail(TDSE_ECUDA, "event sync");
        cudaEventElapsedTime(&ms, e0, e1);
        for (tdse_ctx* c : b->m) c->step = n - 1;
        return TDSE_OK;
    };
    float best = 0;
    b->grid = 0;
    st = build_items(b);
    if (st == TDSE_OK) {
        b->grid = default_grid(b);
        st = timed(best);
    }
    // launch shape per member: threads per instance (the FFT's points per
    // thread) among the variants built for its n, the default N / 8 first
    for (size_t g = 0; g < b->m.size() && st == TDSE_OK; ++g) {
        for (int v = 0; v < MULTI_NVAR && st == TDSE_OK && b->var[g] >= 0; ++v) {
            if (multi_variant_n(v) != b->m[g]->n0 || v == b->var[g]) continue;
            const int keep_v = b->var[g], keep_p = b->per[g], keep_grid = b->grid;
            b->var[g] = v;
            b->per[g] = MULTI_CTA / multi_variant_t(v);
            st = build_items(b);
            if (st != TDSE_OK) break;
            b->grid = default_grid(b);
            float ms = 0;
            st = timed(ms);
            if (st != TDSE_OK) break;
            if (ms < best) {
                best = ms;
            } else {
                b->var[g] = keep_v;
                b->per[g] = keep_p;
                b->grid = keep_grid;
            }
        }
    }
    // instances per work item, member by member (fewer: more, smaller items)
    for (size_t g = 0; g < b->m.size() && st == TDSE_OK; ++g) {
        if (b->var[g] < 0) continue;
        const int full = MULTI_CTA / multi_variant_t(b->var[g]);
        for (int per : {full / 2, full / 4}) {
            if (per < 1 || per == b->per[g]) continue;
            const int keep = b->per[g], keep_grid = b->grid;
            b->per[g] = per;
            st = build_items(b);
            if (st != TDSE_OK) break;
            b->grid = default_grid(b);
            float ms = 0;
            st = timed(ms);
            if (st != TDSE_OK) break;
            if (ms < best) {
                best = ms;
            } else {
                b->per[g] = keep;
                b->grid = keep_grid;
            }
        }
    }
    // CTA count: multiples of the SM count up to one CTA per item
    if (st == TDSE_OK) st = build_items(b);
    if (st == TDSE_OK) {
        const int occ = std::max(1, multi_occupancy(b->smem));
        const int keep = b->grid;
        int best_grid = keep;
        for (int k = 1; k <= occ * 2 && st == TDSE_OK; ++k) {
            const int grid = std::min((int)b->items.size(), b->sms * k);
            if (grid == keep) continue;
            b->grid = grid;
            float ms = 0;
            st = timed(ms);
            if (st == TDSE_OK && ms < best) {
                best = ms;
                best_grid = grid;
            }
            if (grid == (int)b->items.size()) break;
        }
        b->grid = best_grid;
    }
    // the members' own kernels on parallel streams against the best fused launch
    b->mode = 0;
    if (st == TDSE_OK && b->m.size() >= 1) {
        auto timed_streams = [&](float& ms) -> tdse_status {
            tdse_status r = batch_adams_streams(b, n - 1, 1, s);
            for (tdse_ctx* c : b->m) c->step = n - 1;
            if (r != TDSE_OK) return r;
            cudaEventRecord(e0, s);
            for (int i = 0; i < trial_steps && r == TDSE_OK; ++i) {
                r = batch_adams_streams(b, n - 1, 1, s);
                for (tdse_ctx* c : b->m) c->step = n - 1;
            }
            if (r != TDSE_OK) return r;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return b->fail(TDSE_ECUDA, "event sync");
            cudaEventElapsedTime(&ms, e0, e1);
            return TDSE_OK;
        };
        float ms = 0;
        st = timed_streams(ms);
        // the same choice of launch shape for each member's own kernel
        for (size_t g = 0; g < b->m.size() && st == TDSE_OK; ++g) {
            tdse_ctx* c = b->m[g];
            if (c->four1d || periodic1d_f32_threads(c->n0, 1 - c->shape1d) == 0) continue;
            c->shape1d = 1 - c->shape1d;
            float ms2 = 0;
            st = timed_streams(ms2);
            if (st == TDSE_OK && ms2 < ms) ms = ms2;
            else c->shape1d = 1 - c->shape1d;
        }
        b->stream_ms = ms / trial_steps;
        b->fused_ms = best / trial_steps;
        if (st == TDSE_OK && ms < best) b->mode = 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TDSE_OK) return st;
    for (tdse_ctx* c : b->m) {
        std::fill(c->have_u0.begin(), c->have_u0.end(), 0);   // state undefined until tdse_set_initial
        c->step = 0;
        c->inited = false;
        c->ip = false;
    }
    b->tuned = true;
    return TDSE_OK;
}

tdse_status tdse_batch_describe(const tdse_batch* b, char* buf, size_t len) {
    if (!b || !buf || len == 0) return TDSE_EINVAL;
    std::string js = "{\"grid\": " + std::to_string(b->grid) + ", \"sms\": " + std::to_string(b->sms) +
                     ", \"items\": " + std::to_string(b->items.size()) + ", \"smem\": " + std::to_string(b->smem) +
                     ", \"graphs\": " + std::to_string(b->graphs.size()) + ", \"tuned\": " +
                     (b->tuned ? "true" : "false") + ", \"mode\": \"" + (b->mode ? "streams" : "fused") +
                     "\", \"fused_ms\": " + std::to_string(b->fused_ms) + ", \"streams_ms\": " +
                     std::to_string(b->stream_ms) + ", \"members\": [";
    for (size_t g = 0; g < b->m.size(); ++g) {
        const int t = multi_variant_t(b->var[g]);
        js += std::string(g ? ", " : "") + "{\"n\": " + std::to_string(b->m[g]->n0) + ", \"batch\": " +
              std::to_string(b->m[g]->B) + ", \"threads\": " + std::to_string(t) + ", \"per_item\": " +
              std::to_string(b->per[g]) + ", \"stream_threads\": " +
              std::to_string(b->m[g]->four1d ? 0 : periodic1d_f32_threads(b->m[g]->n0, b->m[g]->shape1d)) +
              ", \"layout\": \"" + (b->m[g]->four1d ? "passes" : "cta") + "\"}";
    }
    js += "]}";
    if (js.size() + 1 > len) return TDSE_EINVAL;
    std::memcpy(buf, js.c_str(), js.size() + 1);
    return TDSE_OK;
}

tdse_status tdse_batch_set_mode(tdse_batch* b, int mode) {
    if (!b || (mode != TDSE_BATCH_FUSED && mode != TDSE_BATCH_STREAMS)) return TDSE_EINVAL;
    if (mode != b->mode) drop_graphs(b);
    b->mode = mode;
    return TDSE_OK;
}

const char* tdse_batch_last_error(const tdse_batch* b) { return b ? b->err.c_str() : "null batch"; }

void tdse_batch_destroy(tdse_batch* b) {
    if (!b) return;
    drop_graphs(b);
    for (cudaStream_t st : b->streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

}  // extern "C"
