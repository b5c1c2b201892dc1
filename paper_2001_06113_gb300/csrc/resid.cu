// FP64 residual check of the mixed-precision implicit step (periodic).
//
// For the step n just completed, with the state u^_n and R_n = (Vu)^_n of its
// ring slot taken back to the lab frame in FP64 (u^ = E_n v^,
// R = E_n r~ / z_n), the step solved
//     u^_n = W - i mu_0 h DFT(V u),  u = IDFT(W) / (1 + i mu_0 h V),  W = u^_n + i mu_0 h R_n
// in FP32 transforms.  In FP64:
//     R64 = DFT(V IDFT(W) / (1 + i mu_0 h V)) / NP,
//     rho = mu_0 h ||R64 - R_n||_2 / ||u^_n||_2        (per instance),
// the relative residual of the implicit equation.  Where rho exceeds the
// tolerance (or is not finite) the step is redone in FP64:
//     u^_n <- W - i mu_0 h R64,   R_n <- R64,
// stored back in the interaction picture (state double-float, ring FP32 with
// its dither).  Transforms: one CTA per instance in 1D; column / row / column
// passes in 2D, all complex FP64 in shared memory.
#include "step_common.cuh"

namespace tdse {

struct ResArgs {
    KArgs a;           // base arguments: state, ring, aux (W, then R64), aux2 (u^), V0, tfac, phi, tables
    int n;             // step checked
    int slot;          // its ring slot
    float z[2];        // ring dither z_n
    double hmu0;       // mu_0 h
    double tol;
    double* sums;      // [B][2]: ||R64 - R_n||^2, ||u^_n||^2
    int* flags;        // [B]
    double* rho;       // [B]
    int* ncorr;        // [B]
};

namespace {

constexpr int RT = 256;   // threads per CTA
constexpr int RL = 8;     // lines per CTA in the 2D passes

__device__ __forceinline__ double2 lab_E(const KArgs& a, int b, int n, size_t k) {
    const int k0 = a.n1 > 1 ? (int)(k / a.n1) : (int)k;
    const int k1 = a.n1 > 1 ? (int)(k % a.n1) : 0;
    return e_exact(a, b, n, kmode(k0, a.n0), a.n1 > 1 ? kmode(k1, a.n1) : 0.0, a.n1 > 1 ? 2 : 1);
}

// R_n in the lab frame: E_n r~ / z_n
__device__ __forceinline__ double2 lab_R(const ResArgs& r, int b, size_t k, double2 E) {
    const size_t NP = (size_t)r.a.n0 * r.a.n1;
    const float2 rv = reinterpret_cast<const float2*>(r.a.ring)[((size_t)b * r.a.ring_slots + r.slot) * NP + k];
    const double zx = r.z[0], zy = r.z[1], zz = zx * zx + zy * zy;
    const double2 q = make_double2((rv.x * zx + rv.y * zy) / zz, (rv.y * zx - rv.x * zy) / zz);
    return cmul(E, q);
}

__device__ __forceinline__ void block_add(double v, double* dst) {
    __shared__ double red[RT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(dst, s);
    }
    __syncthreads();
}

// aux = W, aux2 = u^ (lab frame), sums[b][1] += ||u^||^2
__global__ void k_res_prep(const ResArgs r) {
    const KArgs& a = r.a;
    const int b = blockIdx.y;
    const size_t NP = (size_t)a.n0 * a.n1;
    const float4* st = reinterpret_cast<const float4*>(a.uhat) + (size_t)b * NP;
    double acc = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < NP; k += (size_t)gridDim.x * blockDim.x) {
        const double2 E = lab_E(a, b, r.n, k);
        const double2 uh = cmul(E, st_to_d(st[k]));
        const double2 R = lab_R(r, b, k, E);
        a.aux[(size_t)b * NP + k] = make_double2(uh.x - r.hmu0 * R.y, uh.y + r.hmu0 * R.x);   // u^ + i mu0 h R
        a.aux2[(size_t)b * NP + k] = uh;
        acc += uh.x * uh.x + uh.y * uh.y;
    }
    block_add(acc, &r.sums[2 * b + 1]);
}

__device__ __forceinline__ double2 solve_times_V(double2 y, double V, double hmu0) {
    const double c = hmu0 * V, den = 1.0 + c * c;
    const double2 u = make_double2((y.x + c * y.y) / den, (y.y - c * y.x) / den);
    return make_double2(u.x * V, u.y * V);
}

// 1D: aux <- DFT(V IDFT(aux) / (1 + i mu0 h V)), one CTA per instance (unscaled)
template <int N>
__global__ void __launch_bounds__(RT) k_res_1d(const ResArgs r) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double2* buf = reinterpret_cast<double2*>(sm_raw);
    const KArgs& a = r.a;
    const int b = blockIdx.x;
    double2* X = a.aux + (size_t)b * N;
    for (int k = threadIdx.x; k < N; k += RT) buf[k] = X[k];
    __syncthreads();
    CtaFft<double2, N, 1, 1, RT, true>::run(buf, a.tw64_0, nullptr);
    const double vf = a.tfac[(size_t)b * a.ntf + 8 * r.n];
    for (int j = threadIdx.x; j < N; j += RT) buf[j] = solve_times_V(buf[j], vf * a.V0[(size_t)b * a.vstride + j], r.hmu0);
    __syncthreads();
    CtaFft<double2, N, 1, 1, RT, false>::run(buf, a.tw64_0, nullptr);
    for (int k = threadIdx.x; k < N; k += RT) X[k] = buf[k];
}

// 2D column pass (axis 0) in place on aux, RL columns per CTA.
template <int N, bool INV>
__global__ void __launch_bounds__(RT) k_res_cols(const ResArgs r) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double2* buf = reinterpret_cast<double2*>(sm_raw);
    const KArgs& a = r.a;
    const int b = blockIdx.y, c0 = blockIdx.x * RL, n1 = a.n1;
    double2* X = a.aux + (size_t)b * N * n1;
    for (int it = threadIdx.x; it < N * RL; it += RT) {
        const int j = it / RL, c = it % RL;
        buf[j * RL + c] = X[(size_t)j * n1 + c0 + c];
    }
    __syncthreads();
    CtaFft<double2, N, RL, RL, RT, INV>::run(buf, a.tw64_0, nullptr);
    for (int it = threadIdx.x; it < N * RL; it += RT) {
        const int j = it / RL, c = it % RL;
        X[(size_t)j * n1 + c0 + c] = buf[j * RL + c];
    }
}

// 2D row pass (axis 1): inverse, implicit solve and V, forward, in place.
template <int N>
__global__ void __launch_bounds__(RT) k_res_rows(const ResArgs r) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double2* buf = reinterpret_cast<double2*>(sm_raw);
    constexpr int LS = RL + 1;
    const KArgs& a = r.a;
    const int b = blockIdx.y, r0 = blockIdx.x * RL;
    double2* X = a.aux + (size_t)b * a.n0 * N;
    for (int it = threadIdx.x; it < N * RL; it += RT) {
        const int c = it / N, j = it % N;
        buf[j * LS + c] = X[(size_t)(r0 + c) * N + j];
    }
    __syncthreads();
    CtaFft<double2, N, RL, LS, RT, true>::run(buf, a.tw64_1, nullptr);
    const double vf = a.tfac[(size_t)b * a.ntf + 8 * r.n];
    for (int it = threadIdx.x; it < N * RL; it += RT) {
        const int c = it / N, j = it % N;
        buf[j * LS + c] = solve_times_V(buf[j * LS + c], vf * a.V0[(size_t)b * a.vstride + (size_t)(r0 + c) * N + j],
                                        r.hmu0);
    }
    __syncthreads();
    CtaFft<double2, N, RL, LS, RT, false>::run(buf, a.tw64_1, nullptr);
    for (int it = threadIdx.x; it < N * RL; it += RT) {
        const int c = it / N, j = it % N;
        X[(size_t)(r0 + c) * N + j] = buf[j * LS + c];
    }
}

// aux <- R64 = aux / NP; sums[b][0] += ||R64 - R_n||^2
__global__ void k_res_compare(const ResArgs r) {
    const KArgs& a = r.a;
    const int b = blockIdx.y;
    const size_t NP = (size_t)a.n0 * a.n1;
    const double s = 1.0 / (double)NP;
    double acc = 0;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < NP; k += (size_t)gridDim.x * blockDim.x) {
        const double2 R64 = cscale(a.aux[(size_t)b * NP + k], s);
        a.aux[(size_t)b * NP + k] = R64;
        const double2 R = lab_R(r, b, k, lab_E(a, b, r.n, k));
        const double dx = R64.x - R.x, dy = R64.y - R.y;
        acc += dx * dx + dy * dy;
    }
    block_add(acc, &r.sums[2 * b]);
}

__global__ void k_res_decide(const ResArgs r) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= r.a.B) return;
    const double rho = r.hmu0 * sqrt(r.sums[2 * b] / r.sums[2 * b + 1]);
    r.rho[b] = rho;
    const int bad = !(rho <= r.tol);
    r.flags[b] = bad;
    if (bad) r.ncorr[b] += 1;
}

// flagged instances: u^ <- u^ + i mu0 h (R_n - R64), R_n <- R64, stored in the interaction picture
__global__ void k_res_correct(const ResArgs r) {
    const KArgs& a = r.a;
    const int b = blockIdx.y;
    if (!r.flags[b]) return;
    const size_t NP = (size_t)a.n0 * a.n1;
    float4* st = reinterpret_cast<float4*>(a.uhat) + (size_t)b * NP;
    float2* ring = reinterpret_cast<float2*>(a.ring) + ((size_t)b * a.ring_slots + r.slot) * NP;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < NP; k += (size_t)gridDim.x * blockDim.x) {
        const double2 E = lab_E(a, b, r.n, k);
        const double2 R = lab_R(r, b, k, E);
        const double2 R64 = a.aux[(size_t)b * NP + k];
        const double2 uh = a.aux2[(size_t)b * NP + k];
        const double2 d = make_double2(R.x - R64.x, R.y - R64.y);
        const double2 un = make_double2(uh.x - r.hmu0 * d.y, uh.y + r.hmu0 * d.x);
        const double2 Ec = make_double2(E.x, -E.y);
        st[k] = d_to_st<float4>(cmul(Ec, un));
        const double2 q = cmul(Ec, R64);
        ring[k] = cvt<float2>(cmul(make_double2(r.z[0], r.z[1]), q));
    }
}

unsigned grid_of(size_t n) {
    const size_t g = (n + RT - 1) / RT;
    return (unsigned)(g > 1024 ? 1024 : (g ? g : 1));
}

template <class K>
cudaError_t set_smem(K kern, size_t smem) {
    return smem > 48 * 1024 ? cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                            : cudaSuccess;
}

template <int N>
cudaError_t op_1d(const ResArgs& r, cudaStream_t s) {
    const size_t smem = (size_t)N * sizeof(double2);
    cudaError_t e = set_smem(k_res_1d<N>, smem);
    if (e != cudaSuccess) return e;
    k_res_1d<N><<<r.a.B, RT, smem, s>>>(r);
    return cudaGetLastError();
}

template <int N, bool INV>
cudaError_t cols(const ResArgs& r, cudaStream_t s) {
    const size_t smem = (size_t)N * RL * sizeof(double2);
    cudaError_t e = set_smem(k_res_cols<N, INV>, smem);
    if (e != cudaSuccess) return e;
    k_res_cols<N, INV><<<dim3(r.a.n1 / RL, r.a.B), RT, smem, s>>>(r);
    return cudaGetLastError();
}

template <int N>
cudaError_t rows(const ResArgs& r, cudaStream_t s) {
    const size_t smem = (size_t)N * (RL + 1) * sizeof(double2);
    cudaError_t e = set_smem(k_res_rows<N>, smem);
    if (e != cudaSuccess) return e;
    k_res_rows<N><<<dim3(r.a.n0 / RL, r.a.B), RT, smem, s>>>(r);
    return cudaGetLastError();
}

#define RES_SWITCH(n, CALL)                          \
    switch (n) {                                     \
        case 8: return CALL(8);                      \
        case 16: return CALL(16);                    \
        case 32: return CALL(32);                    \
        case 64: return CALL(64);                    \
        case 128: return CALL(128);                  \
        case 256: return CALL(256);                  \
        case 512: return CALL(512);                  \
        case 1024: return CALL(1024);                \
        default: break;                              \
    }

cudaError_t dispatch_1d(const ResArgs& r, cudaStream_t s) {
#define C1(N) op_1d<N>(r, s)
    RES_SWITCH(r.a.n0, C1)
    if (r.a.n0 == 2048) return op_1d<2048>(r, s);
    if (r.a.n0 == 4096) return op_1d<4096>(r, s);
    if (r.a.n0 == 8192) return op_1d<8192>(r, s);
    return cudaErrorInvalidValue;
#undef C1
}
cudaError_t dispatch_cols(const ResArgs& r, bool inv, cudaStream_t s) {
#define CI(N) cols<N, true>(r, s)
#define CF(N) cols<N, false>(r, s)
    if (inv) { RES_SWITCH(r.a.n0, CI) } else { RES_SWITCH(r.a.n0, CF) }
    return cudaErrorInvalidValue;
#undef CI
#undef CF
}
cudaError_t dispatch_rows(const ResArgs& r, cudaStream_t s) {
#define CR(N) rows<N>(r, s)
    RES_SWITCH(r.a.n1, CR)
    return cudaErrorInvalidValue;
#undef CR
}

}  // namespace

bool residual_supported(int dim, int n0, int n1) {
    if (dim == 3) return false;
    if (dim == 1) return n0 >= 8 && n0 <= 8192;
    return n0 >= 8 && n0 <= 1024 && n1 >= 8 && n1 <= 1024;
}

cudaError_t launch_residual_check(const ResArgs& r, bool correct, cudaStream_t s) {
    const size_t NP = (size_t)r.a.n0 * r.a.n1;
    cudaError_t e = cudaMemsetAsync(r.sums, 0, sizeof(double) * 2 * r.a.B, s);
    if (e != cudaSuccess) return e;
    const dim3 eg(grid_of(NP), r.a.B);
    k_res_prep<<<eg, RT, 0, s>>>(r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (r.a.n1 == 1) {
        e = dispatch_1d(r, s);
    } else {
        e = dispatch_cols(r, true, s);
        if (e == cudaSuccess) e = dispatch_rows(r, s);
        if (e == cudaSuccess) e = dispatch_cols(r, false, s);
    }
    if (e != cudaSuccess) return e;
    k_res_compare<<<eg, RT, 0, s>>>(r);
    k_res_decide<<<(r.a.B + 127) / 128, 128, 0, s>>>(r);
    if (correct) k_res_correct<<<eg, RT, 0, s>>>(r);
    return cudaGetLastError();
}

}  // namespace tdse
