// percolation.cu -- site percolation on the supported lattices (the paper's
// Supplemental Material: largest-cluster statistics and the Binder ratio of
// the chimera lattice).  One CTA per mask: a lock-free union-find in shared
// memory (roots hook to the smaller index with atomicCAS, finds halve paths),
// then a count per root and a block maximum.
#include "icmpt.h"

#include <string>

#include "icm_internal.h"

namespace icm {
void set_ctx_error(icm_ctx *ctx, const std::string &msg);
icm_status ctx_device_alloc(icm_ctx *ctx, void **p, size_t bytes);
void ctx_device_free(icm_ctx *ctx, void *p, size_t bytes);
cudaStream_t ctx_stream(const icm_ctx *ctx);
}  // namespace icm

namespace {

__device__ __forceinline__ int find_root(volatile int *parent, int x)
{
    int p = parent[x];
    while (p != x) {
        const int gp = parent[p];
        if (gp != p) parent[x] = gp;   // path halving: only ever points to an ancestor
        x = p;
        p = gp;
    }
    return x;
}

__device__ __forceinline__ void unite(int *parent, int a, int b)
{
    volatile int *vp = parent;
    for (;;) {
        a = find_root(vp, a);
        b = find_root(vp, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(&parent[b], b, a);   // hook the larger root under the smaller
        if (old == b) return;
        b = old;
    }
}

// occupancy of position p of mask m: given masks (site order) or Philox draws
__device__ __forceinline__ bool occupied(const uint8_t *masks, const uint16_t *pos2site, int N, long long m, int p,
                                         uint32_t thr, uint32_t k0, uint32_t k1)
{
    const int site = pos2site[p];
    if (masks) return masks[m * N + site] != 0;
    // Philox4x32-10, ctr {site, mask, 0, 5 << 24}, word 0 < floor(p 2^32)
    uint32_t c0 = (uint32_t)site, c1 = (uint32_t)m, c2 = 0u, c3 = 5u << 24;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint64_t p0 = (uint64_t)c0 * 0xD2511F53ull, p1 = (uint64_t)c2 * 0xCD9E8D57ull;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0 < thr;
}

template <int Z>
__global__ void __launch_bounds__(256) largest_cluster_kernel(const uint8_t *__restrict__ masks, int n_masks, int N,
                                                              const uint16_t *__restrict__ nbr,
                                                              const uint16_t *__restrict__ pos2site, uint32_t thr,
                                                              uint32_t k0, uint32_t k1, int32_t *__restrict__ smax)
{
    extern __shared__ int sh[];
    int *parent = sh;                  // [N], -1 = empty
    int *count = sh + N;               // [N]
    __shared__ int best;
    for (long long m = blockIdx.x; m < n_masks; m += gridDim.x) {
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            parent[p] = occupied(masks, pos2site, N, m, p, thr, k0, k1) ? p : -1;
            count[p] = 0;
        }
        if (threadIdx.x == 0) best = 0;
        __syncthreads();
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            if (parent[p] < 0) continue;
#pragma unroll
            for (int d = 0; d < Z; ++d) {
                const int q = nbr[p * Z + d];
                if (q > p && ((volatile int *)parent)[q] >= 0) unite(parent, p, q);
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < N; p += blockDim.x)
            if (parent[p] >= 0) atomicAdd(&count[find_root(parent, p)], 1);
        __syncthreads();
        int mx = 0;
        for (int p = threadIdx.x; p < N; p += blockDim.x) mx = max(mx, count[p]);
        for (int o = 16; o >= 1; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&best, mx);
        __syncthreads();
        if (threadIdx.x == 0) smax[m] = best;
        __syncthreads();
    }
}

icm_status percolation(icm_ctx *ctx, int32_t lattice, int32_t L, int32_t n_masks, const uint8_t *masks,
                       double p_occ, uint64_t seed, int32_t *smax, uint32_t flags)
{
    if (!ctx) return ICM_ERR_ARG;
    if (!smax || n_masks < 0) {
        icm::set_ctx_error(ctx, "icm_percolation: bad arguments");
        return ICM_ERR_ARG;
    }
    if (n_masks == 0) return ICM_OK;
    icm::HostTables tab;
    if (!icm::host_tables(lattice, L, tab)) {
        icm::set_ctx_error(ctx, "icm_percolation: unsupported lattice");
        return ICM_ERR_ARG;
    }
    const int N = tab.N, Z = tab.Z;
    const size_t smem = (size_t)N * 8;
    if (smem > 200 * 1024) {
        icm::set_ctx_error(ctx, "icm_percolation: lattice too large for one CTA");
        return ICM_ERR_UNSUPPORTED;
    }
    cudaStream_t st = icm::ctx_stream(ctx);
    const bool dev = (flags & ICM_DEVICE_PTR) != 0;
    uint16_t *d_nbr = nullptr, *d_p2s = nullptr;
    uint8_t *d_masks = nullptr;
    int32_t *d_out = nullptr;
    const size_t b_nbr = tab.nbr.size() * 2, b_p2s = tab.pos2site.size() * 2;
    const size_t b_masks = (size_t)n_masks * N, b_out = (size_t)n_masks * 4;
    icm_status ast = icm::ctx_device_alloc(ctx, (void **)&d_nbr, b_nbr);
    if (!ast) ast = icm::ctx_device_alloc(ctx, (void **)&d_p2s, b_p2s);
    if (!ast && masks && !dev) ast = icm::ctx_device_alloc(ctx, (void **)&d_masks, b_masks);
    if (!ast && !dev) ast = icm::ctx_device_alloc(ctx, (void **)&d_out, b_out);
    auto release = [&]() {
        icm::ctx_device_free(ctx, d_nbr, b_nbr);
        icm::ctx_device_free(ctx, d_p2s, b_p2s);
        icm::ctx_device_free(ctx, d_masks, b_masks);
        icm::ctx_device_free(ctx, d_out, b_out);
    };
    if (ast) {
        release();
        return ast;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_nbr, tab.nbr.data(), tab.nbr.size() * 2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_p2s, tab.pos2site.data(), tab.pos2site.size() * 2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d_masks) e = cudaMemcpyAsync(d_masks, masks, (size_t)n_masks * N, cudaMemcpyHostToDevice, st);
    const uint8_t *mk = masks ? (dev ? masks : d_masks) : nullptr;
    int32_t *out = dev ? smax : d_out;
    double tv = p_occ <= 0.0 ? 0.0 : (p_occ >= 1.0 ? 4294967295.0 : p_occ * 4294967296.0);
    const uint32_t thr = (uint32_t)tv;
    const int grid = n_masks < 152 * 8 ? n_masks : 152 * 8;
    if (e == cudaSuccess) {
        auto kern = Z == 4 ? largest_cluster_kernel<4> : Z == 6 ? largest_cluster_kernel<6> : largest_cluster_kernel<8>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            kern<<<grid, 256, smem, st>>>(mk, n_masks, N, d_nbr, d_p2s, thr, (uint32_t)seed, (uint32_t)(seed >> 32), out);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(smax, d_out, (size_t)n_masks * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    else cudaStreamSynchronize(st);            // nothing may still use the blocks freed below
    release();
    if (e != cudaSuccess) {
        icm::set_ctx_error(ctx, std::string("icm_percolation: ") + cudaGetErrorString(e));
        return ICM_ERR_CUDA;
    }
    return ICM_OK;
}

}  // namespace

extern "C" icm_status icm_percolation(icm_ctx *ctx, int32_t lattice, int32_t L, int32_t n_masks,
                                      const uint8_t *masks, int32_t *smax, uint32_t flags)
{
    if (!masks) {
        if (ctx) icm::set_ctx_error(ctx, "icm_percolation: masks are required");
        return ICM_ERR_ARG;
    }
    return percolation(ctx, lattice, L, n_masks, masks, 0.0, 0, smax, flags);
}

extern "C" icm_status icm_percolation_random(icm_ctx *ctx, int32_t lattice, int32_t L, double p, uint64_t seed,
                                             int32_t n_masks, int32_t *smax, uint32_t flags)
{
    if (!(p >= 0.0 && p <= 1.0)) {
        if (ctx) icm::set_ctx_error(ctx, "icm_percolation_random: p must lie in [0, 1]");
        return ICM_ERR_ARG;
    }
    return percolation(ctx, lattice, L, n_masks, nullptr, p, seed, smax, flags);
}
