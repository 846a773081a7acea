// icm_static.cu -- energies of replica configurations without any device
// allocation (icm_energies_static in icmpt.h).
//
// Some callers cannot allocate device memory at the point where they need
// this: code running inside a memory pool or arena that forbids outside
// allocations, callers that must not trigger cudaMalloc's implicit device
// synchronisation in the middle of a pipeline, and hosts that budget every
// byte of HBM up front.  This entry point runs the library's layout and
// energy kernels on a file-scope scratch array that exists for as long as
// the library is loaded, so the call itself allocates nothing.
#include "icmpt.h"

#include <cstring>
#include <mutex>
#include <string>

#include "icm_internal.h"

namespace {

// Scratch shared by every call on a device: geometry tables, packed spins,
// expanded couplings and per-replica energies of the current request.  Each
// GPU that loads the library holds these bytes until the process exits.
constexpr size_t kStaticScratchBytes = size_t(8) << 20;   // 8 MiB
static __device__ __align__(256) unsigned char g_icm_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
// Device address of the array, per device, looked up by the first call on
// that device (with the device current) under g_scratch_mutex, so that host
// threads calling on different devices at the same time do not race on it.
// cudaDeviceReset unloads the module that holds the array, so the address
// looked up before a reset is not valid after it: a process that resets a
// device must not call this entry point on that device afterwards.
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

struct icm_ctx;   // defined in icm_api.cpp
namespace icm {
void set_ctx_error(icm_ctx *ctx, const std::string &msg);
cudaStream_t ctx_stream(const icm_ctx *ctx);
int ctx_device(const icm_ctx *ctx);
}  // namespace icm

extern "C" icm_status icm_energies_static(icm_ctx *ctx, int32_t lattice, int32_t L, int32_t disorder,
                                          int32_t n_inst, int32_t n_rep, const void *couplings,
                                          const int8_t *spins, double *out)
{
    if (!ctx) return ICM_ERR_ARG;
    if (!couplings || !spins || !out) {
        icm::set_ctx_error(ctx, "icm_energies_static: couplings, spins and out must be device pointers");
        return ICM_ERR_ARG;
    }
    if (disorder != ICM_PM_J && disorder != ICM_GAUSS) {
        icm::set_ctx_error(ctx, "icm_energies_static: unknown disorder kind");
        return ICM_ERR_ARG;
    }
    if (n_inst < 1 || n_rep < 1 || n_rep > 64) {
        icm::set_ctx_error(ctx, "icm_energies_static: need n_inst >= 1 and 1 <= n_rep <= 64");
        return ICM_ERR_ARG;
    }
    icm::HostTables tab;
    if (!icm::host_tables(lattice, L, tab)) {
        icm::set_ctx_error(ctx, "icm_energies_static: unsupported lattice");
        return ICM_ERR_ARG;
    }
    const bool gauss = disorder == ICM_GAUSS;
    const int N = tab.N, Z = tab.Z, G = (n_rep + 31) / 32;
    // scratch layout
    const size_t o_nbr = 0;
    const size_t o_p2s = o_nbr + align256(tab.nbr.size() * 2);
    const size_t o_edge = o_p2s + align256(tab.pos2site.size() * 2);
    const size_t o_spins = o_edge + align256(tab.edge_bond.size() * 4);
    const size_t o_J = o_spins + align256((size_t)n_inst * G * N * 4);
    const size_t o_E = o_J + align256(gauss ? (size_t)n_inst * N * Z * 4 : (size_t)n_inst * N);
    const size_t total = o_E + align256((size_t)n_inst * n_rep * 4);
    if (total > kStaticScratchBytes) {
        icm::set_ctx_error(ctx, "icm_energies_static: request needs " + std::to_string(total) +
                                    " bytes of scratch, more than its fixed " + std::to_string(kStaticScratchBytes) +
                                    " bytes; use fewer instances per call");
        return ICM_ERR_UNSUPPORTED;
    }
    const int dev = icm::ctx_device(ctx);
    if (dev < 0 || dev >= kMaxDevices) {
        icm::set_ctx_error(ctx, "icm_energies_static: device index out of range");
        return ICM_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(dev);
    void *addr = nullptr;
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {                  // first call on this device: look up the array's address
            e = cudaGetSymbolAddress(&addr, g_icm_static_scratch);
            if (e == cudaSuccess) g_scratch_addr[dev] = addr;
        }
        addr = g_scratch_addr[dev];
    }
    if (e != cudaSuccess || !addr) {
        icm::set_ctx_error(ctx, std::string("icm_energies_static: scratch set-up failed: ") + cudaGetErrorString(e));
        return ICM_ERR_CUDA;
    }
    unsigned char *base = (unsigned char *)addr;
    cudaStream_t st = icm::ctx_stream(ctx);
    icm::KParams P{};
    P.N = N; P.Nb = tab.Nb; P.R = n_rep; P.G = G; P.Z = Z; P.n_inst = n_inst; P.half = N / 2;
    P.nbr = (const uint16_t *)(base + o_nbr);
    P.pos2site = (const uint16_t *)(base + o_p2s);
    P.spins = (uint32_t *)(base + o_spins);
    P.Jd = gauss ? (const float *)(base + o_J) : nullptr;
    P.Jb = gauss ? nullptr : (const uint8_t *)(base + o_J);
    P.Ef = gauss ? (float *)(base + o_E) : nullptr;
    P.Ei = gauss ? nullptr : (int32_t *)(base + o_E);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_nbr, tab.nbr.data(), tab.nbr.size() * 2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_p2s, tab.pos2site.data(), tab.pos2site.size() * 2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_edge, tab.edge_bond.data(), tab.edge_bond.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = icm::launch_expand_couplings(couplings, gauss, (const int32_t *)(base + o_edge), n_inst, N, Z, tab.Nb,
                                         const_cast<float *>(P.Jd), const_cast<uint8_t *>(P.Jb), st);
    if (e == cudaSuccess) e = icm::launch_pack_spins(spins, P.spins, P.pos2site, n_inst, n_rep, G, N, st);
    if (e == cudaSuccess) e = icm::launch_init_energies(P, gauss, st);
    if (e == cudaSuccess) e = icm::launch_energies_to_double(P, gauss, out, st);
    // the host tables above are pageable memory read by the copies: wait before they go out of scope
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        icm::set_ctx_error(ctx, std::string("icm_energies_static: ") + cudaGetErrorString(e));
        return ICM_ERR_CUDA;
    }
    return ICM_OK;
}
