// Uneven 1D batches: one persistent launch runs the mixed-precision step of
// many contexts (instances of different n), see kargs.h.
#include "step1d.cuh"

namespace tdse {

namespace {

struct Variant {
    int n, t;
};
// Variants 0..11: the default threads per instance (N / 8, 32..512); 12..14:
// half of it (twice the points per thread), a launch shape the batch tuner
// may pick per member.
constexpr Variant kVariants[MULTI_NVAR] = {{256, 32},  {512, 64},  {1024, 128}, {2048, 256}, {4096, 512},
                                           {8192, 512}, {16384, 512}, {128, 32}, {64, 32},    {32, 32},
                                           {16, 32},   {8, 32},    {2048, 128}, {4096, 256}, {8192, 256}};

// `count` instances b0.. of one context, each by a group of T threads with
// its own N-element slice of shared memory.  Each variant is a separate
// (not inlined) function: the kernel stays a small dispatcher.
template <int N, int T>
__device__ __noinline__ void run_group(const KArgs& a, int b0, int count, float2* smem) {
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
            case 2: run_group<1024, 128>(a, it.b0, it.count, smem); break;
            case 3: run_group<2048, 256>(a, it.b0, it.count, smem); break;
            case 4: run_group<4096, 512>(a, it.b0, it.count, smem); break;
            case 5: run_group<8192, 512>(a, it.b0, it.count, smem); break;
            case 6: run_group<16384, 512>(a, it.b0, it.count, smem); break;
            case 7: run_group<128, 32>(a, it.b0, it.count, smem); break;
            case 8: run_group<64, 32>(a, it.b0, it.count, smem); break;
            case 9: run_group<32, 32>(a, it.b0, it.count, smem); break;
            case 10: run_group<16, 32>(a, it.b0, it.count, smem); break;
            case 11: run_group<8, 32>(a, it.b0, it.count, smem); break;
            case 12: run_group<2048, 128>(a, it.b0, it.count, smem); break;
            case 13: run_group<4096, 256>(a, it.b0, it.count, smem); break;
            case 14: run_group<8192, 256>(a, it.b0, it.count, smem); break;
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

}  // namespace tdse
