// icm_api.cpp -- host half of the C ABI declared in include/icmpt.h.
//
// Builds the lattice (bond order as documented in the header), the
// colour-major site positions and neighbour tables, the integer acceptance
// tables of the +-J path, allocates the batch's device state and launches
// the kernels of pt_icm.cu on the context's stream.
#include "icmpt.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "icm_internal.h"

struct icm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int max_smem_optin = 0;
    std::string err = "no error";
    std::set<icm_batch *> batches;   // live batches, freed with the context
    size_t budget = 0;               // device bytes the batches may hold (0 = no limit)
    size_t in_use = 0;               // device bytes they hold now
    bool hooked = false;             // allocations go through `alloc`
    icm_allocator alloc{};
};

namespace {

struct Geometry {
    int N = 0, Nb = 0, Z = 0;
    std::vector<int> bi, bj;        // bond endpoints, bond order
    std::vector<uint8_t> color;     // [N]
};

int lattice_size(int lattice, int L, int *N, int *Nb)
{
    if (L < 1) return -1;
    switch (lattice) {
    case ICM_SQUARE2D: *N = L * L; *Nb = 2 * L * L; return 0;
    case ICM_CUBIC3D: *N = L * L * L; *Nb = 3 * L * L * L; return 0;
    case ICM_CHIMERA: *N = 8 * L * L; *Nb = 16 * L * L + 8 * L * (L - 1); return 0;
    case ICM_HYPERCUBIC4D:
        if (L > 64) return -1;               // L^4 sites must stay an int
        *N = L * L * L * L;
        *Nb = 4 * L * L * L * L;
        return 0;
    default: return -1;
    }
}

// Bond list in the order documented for each lattice kind in icmpt.h.
bool build_geometry(int lattice, int L, Geometry &g)
{
    if (lattice_size(lattice, L, &g.N, &g.Nb)) return false;
    g.bi.resize(g.Nb);
    g.bj.resize(g.Nb);
    g.color.resize(g.N);
    if (lattice == ICM_SQUARE2D) {
        g.Z = 4;
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                const int i = x + L * y;
                g.color[i] = (uint8_t)((x + y) & 1);
                g.bi[2 * i] = i;
                g.bj[2 * i] = ((x + 1) % L) + L * y;
                g.bi[2 * i + 1] = i;
                g.bj[2 * i + 1] = x + L * ((y + 1) % L);
            }
    } else if (lattice == ICM_CUBIC3D) {
        g.Z = 6;
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    const int i = x + L * (y + L * z);
                    g.color[i] = (uint8_t)((x + y + z) & 1);
                    const int nx = ((x + 1) % L) + L * (y + L * z);
                    const int ny = x + L * (((y + 1) % L) + L * z);
                    const int nz = x + L * (y + L * ((z + 1) % L));
                    g.bi[3 * i] = i; g.bj[3 * i] = nx;
                    g.bi[3 * i + 1] = i; g.bj[3 * i + 1] = ny;
                    g.bi[3 * i + 2] = i; g.bj[3 * i + 2] = nz;
                }
    } else if (lattice == ICM_HYPERCUBIC4D) {
        g.Z = 8;
        for (int w = 0; w < L; ++w)
            for (int z = 0; z < L; ++z)
                for (int y = 0; y < L; ++y)
                    for (int x = 0; x < L; ++x) {
                        const int i = x + L * (y + L * (z + L * w));
                        g.color[i] = (uint8_t)((x + y + z + w) & 1);
                        g.bi[4 * i] = i; g.bj[4 * i] = ((x + 1) % L) + L * (y + L * (z + L * w));
                        g.bi[4 * i + 1] = i; g.bj[4 * i + 1] = x + L * (((y + 1) % L) + L * (z + L * w));
                        g.bi[4 * i + 2] = i; g.bj[4 * i + 2] = x + L * (y + L * (((z + 1) % L) + L * w));
                        g.bi[4 * i + 3] = i; g.bj[4 * i + 3] = x + L * (y + L * (z + L * ((w + 1) % L)));
                    }
    } else {
        g.Z = 6;
        const int M = L;
        auto site = [M](int r, int c, int h, int k) { return 8 * (r * M + c) + 4 * h + k; };
        for (int r = 0; r < M; ++r)
            for (int c = 0; c < M; ++c)
                for (int h = 0; h < 2; ++h)
                    for (int k = 0; k < 4; ++k) g.color[site(r, c, h, k)] = (uint8_t)((r + c + h) & 1);
        int b = 0;
        for (int cell = 0; cell < M * M; ++cell)
            for (int k0 = 0; k0 < 4; ++k0)
                for (int k1 = 0; k1 < 4; ++k1, ++b) {
                    g.bi[b] = 8 * cell + k0;
                    g.bj[b] = 8 * cell + 4 + k1;
                }
        for (int r = 0; r + 1 < M; ++r)
            for (int c = 0; c < M; ++c)
                for (int k = 0; k < 4; ++k, ++b) {
                    g.bi[b] = site(r, c, 0, k);
                    g.bj[b] = site(r + 1, c, 0, k);
                }
        for (int r = 0; r < M; ++r)
            for (int c = 0; c + 1 < M; ++c)
                for (int k = 0; k < 4; ++k, ++b) {
                    g.bi[b] = site(r, c, 1, k);
                    g.bj[b] = site(r, c + 1, 1, k);
                }
        if (b != g.Nb) return false;
    }
    return true;
}

// Philox4x32-10 on the host (Salmon, Moraes, Dror, Shaw, SC'11: multipliers
// 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85), for
// disorder drawn from the seed when a caller passes no couplings.
void host_philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed, uint32_t o[4])
{
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        const uint64_t m0 = (uint64_t)c0 * 0xD2511F53ull;
        const uint64_t m1 = (uint64_t)c2 * 0xCD9E8D57ull;
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(m0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)m1;
        c3 = (uint32_t)m0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
}

// Couplings [n][Nb] of instances ids[0..n) drawn from the seed (Philox domain
// 3, counters by instance id and bond index only):
//   +-J      bond b: the top bit of word b & 3 of ctr {b >> 2, 0, 0, 3<<24 | id}
//            (0 -> +1, 1 -> -1), the paper's bimodal distribution;
//   Gaussian bond b: words o0, o1 of ctr {b, 1, 0, 3<<24 | id}, u1 = (o0 + 1) 2^-32,
//            u2 = o1 2^-32, J = sqrt(-2 ln u1) cos(2 pi u2) (Box-Muller, in
//            double, rounded to fp32), the paper's N(0, 1).
void generate_couplings(bool gauss, int n, int Nb, const uint32_t *ids, uint64_t seed,
                        std::vector<unsigned char> &out)
{
    out.assign((size_t)n * Nb * (gauss ? 4 : 1), 0);
    for (int a = 0; a < n; ++a) {
        const uint32_t c3 = (3u << 24) | ids[a];
        if (gauss) {
            float *J = (float *)out.data() + (size_t)a * Nb;
            for (int b = 0; b < Nb; ++b) {
                uint32_t o[4];
                host_philox((uint32_t)b, 1u, 0u, c3, seed, o);
                const double u1 = ((double)o[0] + 1.0) * (1.0 / 4294967296.0);
                const double u2 = (double)o[1] * (1.0 / 4294967296.0);
                const double r = std::sqrt(-2.0 * std::log(u1));
                const double w = std::cos(6.283185307179586 * u2);
                J[b] = (float)(r * w);
            }
        } else {
            int8_t *J = (int8_t *)out.data() + (size_t)a * Nb;
            for (int b = 0; b < Nb; ++b) {
                uint32_t o[4];
                host_philox((uint32_t)b >> 2, 0u, 0u, c3, seed, o);
                J[b] = (o[b & 3] >> 31) ? (int8_t)-1 : (int8_t)1;
            }
        }
    }
}

// floor(exp(a) * 2^32), saturated at 2^32 - 1 (a <= 0).
uint32_t acceptance_threshold(double a)
{
    const double v = std::floor(std::exp(a) * 4294967296.0);
    if (v >= 4294967295.0) return 4294967295u;
    if (v <= 0.0) return 0u;
    return (uint32_t)v;
}

// Temperature-dependent tables of a ladder T[0..n_T-1] (ascending):
//  thr_metro[r][m] = floor(exp((-2m) beta_k) 2^32) for the +-J Metropolis
//    test at replica position r = 2k + c and m = s_i h_i = 1..Z, and 2^31 at
//    m = 0 (the zero-energy proposal of a diluted instance; the other
//    instances accept every m <= 0 before the table); stride thr_stride(Z);
//  b2l[r] = -2 beta_k log2(e) for the Gaussian test;
//  dbeta_l2e[k] = (beta_k - beta_{k+1}) log2(e) for PT decisions (the Gaussian
//    test; the +-J count of thresholds above a draw starts from it);
//  thr_swap (per pair k, d = 1..len_k) = floor(exp((-2d)(beta_k - beta_{k+1})) 2^32)
//    for +-J PT decisions, cut where it reaches 0.  The kernels count the
//    leading thresholds above a draw (stepping from the closed form), which
//    needs each pair's run to be non-increasing in d (exp is monotone);
//    swap_monotone records that it is.
struct TempTables {
    std::vector<double> beta;
    std::vector<uint32_t> thr_metro;
    std::vector<float> b2l, dbeta_l2e;
    std::vector<uint32_t> thr_swap;
    std::vector<int32_t> swap_off, swap_len;
    bool swap_monotone = true;
};

void temperature_tables(const double *T, int n_T, int Nb, int Z, TempTables &t)
{
    const int R = 2 * n_T, TS = icm::thr_stride(Z);
    t.beta.assign(n_T, 0.0);
    for (int k = 0; k < n_T; ++k) t.beta[k] = 1.0 / T[k];
    t.thr_metro.assign((size_t)R * TS, 0u);
    t.b2l.assign(R, 0.f);
    for (int r = 0; r < R; ++r) {
        const double bk = t.beta[r / 2];
        t.thr_metro[(size_t)r * TS] = 0x80000000u;
        for (int m = 1; m <= Z; ++m) t.thr_metro[(size_t)r * TS + m] = acceptance_threshold((double)(-2 * m) * bk);
        t.b2l[r] = (float)(-2.0 * bk * 1.4426950408889634);
    }
    t.dbeta_l2e.assign(n_T > 1 ? n_T - 1 : 0, 0.f);
    for (int k = 0; k + 1 < n_T; ++k) t.dbeta_l2e[k] = (float)((t.beta[k] - t.beta[k + 1]) * 1.4426950408889634);
    t.thr_swap.clear();
    t.swap_off.assign(n_T > 1 ? n_T - 1 : 0, 0);
    t.swap_len.assign(n_T > 1 ? n_T - 1 : 0, 0);
    for (int k = 0; k + 1 < n_T; ++k) {
        const double db = t.beta[k] - t.beta[k + 1];
        t.swap_off[k] = (int32_t)t.thr_swap.size();
        int len = 0;
        for (int d = 1; d <= Nb; ++d) {
            const uint32_t v = acceptance_threshold((double)(-2 * d) * db);
            if (v == 0u) break;
            if (len > 0 && v > t.thr_swap.back()) t.swap_monotone = false;
            t.thr_swap.push_back(v);
            ++len;
        }
        t.swap_len[k] = len;
    }
    if (t.thr_swap.empty()) t.thr_swap.push_back(0u);
}

struct DevBuf {
    void *p = nullptr;
};

}  // namespace

struct icm_batch {
    icm_ctx *ctx = nullptr;
    int lattice = 0, L = 0, disorder = 0, n_inst = 0, nT = 0;
    bool gauss = false;
    double T_icm = 0.0;
    uint64_t seed = 0;
    Geometry geo;
    std::vector<double> T;
    icm_schedule sched{};
    icm::KParams kp{};
    int threads = 0, grid = 0, ctas_per_sm = 0, n_icm = 0;
    size_t thr_swap_cap = 0;      // entries allocated for the +-J swap thresholds
    int64_t launches = 0;
    std::vector<std::pair<void *, size_t>> allocs;   // device blocks and their sizes
    std::vector<uint16_t> h_pos2site;  // [N] site of each colour-major position
    // staging buffers for loads and reads
    void *raw_coup = nullptr;     // [n_inst][Nb] int8 or float
    int8_t *raw_spins = nullptr;  // [n_inst][R][N]
    double *raw_E = nullptr;      // [n_inst][R]
    int32_t *edge_bond = nullptr; // [N][Z]
    // dilution: bonds present per instance (host copy of nb_inst), and the
    // degree of the undiluted lattice when uniform (0: chimera)
    std::vector<int32_t> h_nb;
    int uniform_z = 0;
    // invalid couplings per instance (not finite; +-J outside -1, 0, +1)
    int32_t *d_bad = nullptr;         // [n_inst]
    std::vector<int32_t> h_bad;
    // cluster layout: one instance per thread-block cluster of cluster_k CTAs
    int cluster_k = 0;
    int cl_growth = -1;               // cluster growth: -1 = by the library (scans), 0 = scans, 1 = union-find
    uint16_t *d_cl_order = nullptr;   // [N] growth order of the cluster layout's own sites (KParams::cl_order)
    icm::ClusterLayout cl{};
    int n_clusters = 0;
    // wide (global-resident) layout: per-CTA scratch, grown on demand (in allocs)
    uint32_t *scratch = nullptr;      // [scratch_ctas][wide_scratch_words(N)]
    int scratch_ctas = 0;
    // per-slot control (serving), allocated on first use
    uint8_t *d_active = nullptr;      // [n_inst]
    long long *d_tmeas = nullptr;     // [n_inst]
    std::vector<uint8_t> h_active;
    std::vector<long long> h_tmeas;
    int groups = 0;                   // live groups whose graphs launch this batch's kernels
};

extern "C" {
static icm_status apply_threads(icm_batch *b, int threads);   // defined with the ABI functions
static icm_status apply_cluster(icm_batch *b, int K, int threads);
}

namespace {

icm_status fail(icm_ctx *ctx, icm_status code, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

icm_status cuda_fail(icm_ctx *ctx, cudaError_t e, const char *what)
{
    return fail(ctx, ICM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define ICM_CUDA(ctx, call)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Device memory of a context: through its allocator hooks or cudaMalloc,
// counted against its budget.
icm_status ctx_alloc(icm_ctx *ctx, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return fail(ctx, ICM_ERR_BUDGET, "device memory budget exceeded (" + std::to_string(ctx->in_use + bytes) +
                                             " > " + std::to_string(ctx->budget) + " bytes)");
    if (ctx->hooked) {
        *p = ctx->alloc.alloc(bytes, ctx->device, (void *)ctx->stream, ctx->alloc.user);
        if (!*p) return fail(ctx, ICM_ERR_OOM, "allocator hook returned NULL");
    } else {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            *p = nullptr;
            return fail(ctx, ICM_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    ctx->in_use += bytes;
    return ICM_OK;
}

void ctx_free(icm_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (ctx->hooked) ctx->alloc.free(p, bytes, ctx->device, (void *)ctx->stream, ctx->alloc.user);
    else cudaFree(p);
    ctx->in_use -= bytes;
}

template <typename T>
icm_status dalloc(icm_batch *b, T **p, size_t count)
{
    void *q = nullptr;
    const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
    icm_status st = ctx_alloc(b->ctx, &q, bytes);
    if (st) return st;
    b->allocs.push_back({q, bytes});
    *p = (T *)q;
    return ICM_OK;
}

icm_status copy_in(icm_ctx *ctx, void *dst, const void *src, size_t bytes, uint32_t flags)
{
    const cudaMemcpyKind kind = (flags & ICM_DEVICE_PTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ICM_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, kind, ctx->stream));
    return ICM_OK;
}

icm_status copy_out(icm_ctx *ctx, void *dst, const void *src, size_t bytes, uint32_t flags)
{
    const cudaMemcpyKind kind = (flags & ICM_DEVICE_PTR) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    ICM_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, kind, ctx->stream));
    return ICM_OK;
}

// One launch of n_sweeps simulation steps of the batch, in its layout.
cudaError_t launch_batch(const icm_batch *b, const icm::KParams &P, uint32_t n_sweeps, cudaStream_t st)
{
    if (b->cluster_k) return icm::launch_cluster(P, b->cl, b->gauss, b->threads, b->n_clusters, n_sweeps, st);
    return icm::launch_fused(P, b->gauss, b->threads, b->grid, n_sweeps, st);
}

// Per-instance dilution tables of slots [first, first + count) from the bond
// couplings in raw_coup, then the batch flags: the batch is diluted while any
// instance has an absent bond (the kernels then read per-instance neighbour
// tables and degrees).  Waits for the stream (the counts come back to the host).
icm_status refresh_dilution(icm_batch *b, int first, int count)
{
    icm_ctx *ctx = b->ctx;
    icm::KParams &P = b->kp;
    const size_t esz = b->gauss ? 4 : 1;
    int32_t *nb = const_cast<int32_t *>(P.nb_inst) + first;
    int32_t *bad = b->d_bad + first;
    ICM_CUDA(ctx, cudaMemsetAsync(nb, 0, (size_t)count * sizeof(int32_t), ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(bad, 0, (size_t)count * sizeof(int32_t), ctx->stream));
    ICM_CUDA(ctx, icm::launch_expand_dilution((const unsigned char *)b->raw_coup + (size_t)first * P.Nb * esz, b->gauss,
                                              b->edge_bond, P.nbr, count, P.N, P.Z, P.Nb,
                                              const_cast<uint16_t *>(P.nbr_inst) + (size_t)first * P.N * P.Z,
                                              const_cast<uint8_t *>(P.zdeg_inst) + (size_t)first * P.N, nb, bad,
                                              ctx->stream));
    b->h_nb.resize(b->n_inst, P.Nb);
    b->h_bad.resize(b->n_inst, 0);
    ICM_CUDA(ctx, cudaMemcpyAsync(b->h_nb.data() + first, nb, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    ICM_CUDA(ctx, cudaMemcpyAsync(b->h_bad.data() + first, bad, (size_t)count * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, ctx->stream));
    ICM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    bool diluted = false;
    for (int32_t v : b->h_nb) diluted |= v < P.Nb;
    const bool was_diluted = P.diluted != 0;
    P.diluted = diluted ? 1 : 0;
    P.const_z = diluted ? 0 : b->uniform_z;
    if (b->cluster_k && diluted != was_diluted) {
        // the cluster layout switches to its kernels with per-instance tables
        // (or back): the clusters that fit are counted again
        icm_status st = apply_cluster(b, b->cluster_k, b->threads);
        if (st) return st;
    }
    long long n_bad = 0;
    for (int i = first; i < first + count; ++i) n_bad += b->h_bad[i];
    if (n_bad)
        return fail(ctx, ICM_ERR_ARG, std::to_string(n_bad) + " invalid couplings (not finite, or +-J outside -1, 0, +1)");
    return ICM_OK;
}

icm_status upload_state(icm_batch *b, const void *couplings, const int8_t *spins, uint32_t flags)
{
    icm_ctx *ctx = b->ctx;
    icm::KParams &P = b->kp;
    if (couplings) {
        const size_t bytes = (size_t)b->n_inst * P.Nb * (b->gauss ? 4 : 1);
        icm_status st = copy_in(ctx, b->raw_coup, couplings, bytes, flags);
        if (st) return st;
        ICM_CUDA(ctx, icm::launch_expand_couplings(b->raw_coup, b->gauss, b->edge_bond, b->n_inst, P.N, P.Z, P.Nb,
                                                   const_cast<float *>(P.Jd), const_cast<uint8_t *>(P.Jb),
                                                   ctx->stream));
        if ((st = refresh_dilution(b, 0, b->n_inst))) return st;
    }
    if (spins) {
        const size_t bytes = (size_t)b->n_inst * P.R * P.N;
        icm_status st = copy_in(ctx, b->raw_spins, spins, bytes, flags);
        if (st) return st;
        ICM_CUDA(ctx, icm::launch_pack_spins(b->raw_spins, P.spins, P.pos2site, b->n_inst, P.R, P.G, P.N,
                                             ctx->stream));
    }
    ICM_CUDA(ctx, icm::launch_init_energies(P, b->gauss, ctx->stream));
    return ICM_OK;
}

icm_status clear_observables(icm_batch *b)
{
    icm_ctx *ctx = b->ctx;
    icm::KParams &P = b->kp;
    const size_t nk = (size_t)b->n_inst * P.nT;
    ICM_CUDA(ctx, cudaMemsetAsync(P.accE, 0, nk * sizeof(double), ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(P.acc64, 0, 4 * nk * sizeof(long long), ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(P.hist, 0, nk * (P.N + 1) * sizeof(unsigned long long), ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(P.n_meas, 0, (size_t)b->n_inst * sizeof(long long), ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(P.icm_stats, 0, 2 * (size_t)b->n_inst * sizeof(unsigned long long), ctx->stream));
    return ICM_OK;
}

void destroy_batch(icm_batch *b)
{
    if (!b) return;
    if (b->ctx) {
        cudaStreamSynchronize(b->ctx->stream);
        b->ctx->batches.erase(b);
    }
    for (auto &a : b->allocs) ctx_free(b->ctx, a.first, a.second);
    delete b;
}

}  // namespace

namespace icm {

void set_ctx_error(icm_ctx *ctx, const std::string &msg)
{
    if (ctx) ctx->err = msg;
}
cudaStream_t ctx_stream(const icm_ctx *ctx) { return ctx->stream; }
int ctx_device(const icm_ctx *ctx) { return ctx->device; }
// device memory of the context (its allocator and budget) for the other
// translation units; the status is ICM_OK, ICM_ERR_BUDGET or ICM_ERR_OOM
icm_status ctx_device_alloc(icm_ctx *ctx, void **p, size_t bytes) { return ctx_alloc(ctx, p, bytes); }
void ctx_device_free(icm_ctx *ctx, void *p, size_t bytes) { ctx_free(ctx, p, bytes); }

}  // namespace icm

namespace icm {

// Position tables of one lattice for the layout kernels (colour-major site
// positions, neighbour positions padded with the site itself, bond index per
// directed edge or -1).  Returns false for a lattice this library does not
// support.
bool host_tables(int lattice, int L, HostTables &t)
{
    Geometry g;
    if ((lattice != ICM_CHIMERA && (L < 2 || (L & 1))) || (lattice == ICM_CHIMERA && L < 1)) return false;
    if (!build_geometry(lattice, L, g) || g.N > 65535) return false;
    const int N = g.N, Z = g.Z;
    t.N = N;
    t.Nb = g.Nb;
    t.Z = Z;
    std::vector<int> pos(N);
    t.pos2site.assign(N, 0);
    int next[2] = {0, N / 2};
    for (int i = 0; i < N; ++i) {
        if (next[g.color[i]] >= (g.color[i] ? N : N / 2)) return false;
        pos[i] = next[g.color[i]]++;
        t.pos2site[pos[i]] = (uint16_t)i;
    }
    std::vector<std::vector<std::pair<int, int>>> inc(N);
    for (int e = 0; e < g.Nb; ++e) {
        inc[g.bi[e]].push_back({g.bj[e], e});
        inc[g.bj[e]].push_back({g.bi[e], e});
    }
    t.nbr.assign((size_t)N * Z, 0);
    t.edge_bond.assign((size_t)N * Z, -1);
    for (int i = 0; i < N; ++i) {
        const int deg = (int)inc[i].size(), p = pos[i];
        if (deg > Z) return false;
        for (int d = 0; d < Z; ++d) {
            t.nbr[(size_t)p * Z + d] = (uint16_t)(d < deg ? pos[inc[i][d].first] : p);
            t.edge_bond[(size_t)p * Z + d] = d < deg ? inc[i][d].second : -1;
        }
    }
    return true;
}

}  // namespace icm

extern "C" {

icm_status icm_ctx_create(icm_ctx **out, int32_t device, void *cuda_stream)
{
    return icm_ctx_create_ex(out, device, cuda_stream, 0, nullptr);
}

icm_status icm_ctx_create_ex(icm_ctx **out, int32_t device, void *cuda_stream, size_t hbm_budget,
                             const icm_allocator *alloc)
{
    if (!out) return ICM_ERR_ARG;
    if (alloc && (!alloc->alloc || !alloc->free)) return ICM_ERR_ARG;
    *out = nullptr;
    icm_ctx *ctx = new (std::nothrow) icm_ctx();
    if (!ctx) return ICM_ERR_OOM;
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) {
        delete ctx;
        return ICM_ERR_CUDA;
    }
    ctx->budget = hbm_budget;
    if (alloc) {
        ctx->hooked = true;
        ctx->alloc = *alloc;
    }
    *out = ctx;
    return ICM_OK;
}

icm_status icm_ctx_memory(const icm_ctx *ctx, size_t *in_use, size_t *budget)
{
    if (!ctx) return ICM_ERR_ARG;
    if (in_use) *in_use = ctx->in_use;
    if (budget) *budget = ctx->budget;
    return ICM_OK;
}

icm_status icm_ctx_destroy(icm_ctx *ctx)
{
    if (!ctx) return ICM_ERR_ARG;
    while (!ctx->batches.empty()) destroy_batch(*ctx->batches.begin());
    delete ctx;
    return ICM_OK;
}

const char *icm_last_error(const icm_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

icm_status icm_sync(icm_ctx *ctx)
{
    if (!ctx) return ICM_ERR_ARG;
    ICM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return ICM_OK;
}

icm_status icm_query(icm_ctx *ctx)
{
    if (!ctx) return ICM_ERR_ARG;
    const cudaError_t e = cudaStreamQuery(ctx->stream);
    if (e == cudaSuccess) return ICM_OK;
    if (e == cudaErrorNotReady) {
        (void)cudaGetLastError();
        return ICM_PENDING;
    }
    return cuda_fail(ctx, e, "stream query");
}

icm_status icm_lattice_size(int32_t lattice, int32_t L, int32_t *n_sites, int32_t *n_bonds)
{
    int N, Nb;
    if (!n_sites || !n_bonds || lattice_size(lattice, L, &N, &Nb)) return ICM_ERR_ARG;
    *n_sites = N;
    *n_bonds = Nb;
    return ICM_OK;
}

icm_status icm_batch_create(icm_ctx *ctx, int32_t lattice, int32_t L, int32_t disorder, int32_t n_inst,
                            const void *couplings, const int8_t *spins, const uint32_t *instance_ids,
                            const double *T, int32_t n_T, double T_icm, uint64_t seed, uint32_t flags,
                            icm_batch **out)
{
    if (!ctx) return ICM_ERR_ARG;
    if (!out) return fail(ctx, ICM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (lattice < 0 || lattice > 3) return fail(ctx, ICM_ERR_ARG, "unknown lattice kind");
    if (disorder != ICM_PM_J && disorder != ICM_GAUSS) return fail(ctx, ICM_ERR_ARG, "unknown disorder kind");
    if (lattice != ICM_CHIMERA && (L < 2 || (L & 1))) return fail(ctx, ICM_ERR_ARG, "lattices need an even L >= 2");
    if (lattice == ICM_CHIMERA && L < 1) return fail(ctx, ICM_ERR_ARG, "chimera needs M >= 1");
    if (n_inst < 1) return fail(ctx, ICM_ERR_ARG, "n_inst must be >= 1");
    if (!T || n_T < 1 || n_T > 32) return fail(ctx, ICM_ERR_ARG, "need 1 <= n_T <= 32 temperatures");
    for (int k = 0; k < n_T; ++k) {
        if (!(T[k] > 0.0) || !std::isfinite(T[k])) return fail(ctx, ICM_ERR_ARG, "temperatures must be finite and > 0");
        if (k && !(T[k] > T[k - 1])) return fail(ctx, ICM_ERR_ARG, "temperatures must be strictly ascending");
    }
    icm_batch *b = new (std::nothrow) icm_batch();
    if (!b) return fail(ctx, ICM_ERR_OOM, "host allocation failed");
    b->ctx = ctx;
    b->lattice = lattice;
    b->L = L;
    b->disorder = disorder;
    b->gauss = (disorder == ICM_GAUSS);
    b->n_inst = n_inst;
    b->nT = n_T;
    b->T_icm = T_icm;
    b->seed = seed;
    b->T.assign(T, T + n_T);
    b->sched = icm_schedule{1, 1, 1, 1, 0, 0, 0};
    if (!build_geometry(lattice, L, b->geo)) {
        destroy_batch(b);
        return fail(ctx, ICM_ERR_ARG, "geometry construction failed");
    }
    Geometry &g = b->geo;
    const int N = g.N, Z = g.Z, R = 2 * n_T, G = (R + 31) / 32;
    if (N > 65535) {
        destroy_batch(b);
        return fail(ctx, ICM_ERR_UNSUPPORTED, "more than 65535 sites");
    }
    // colour-major positions, ascending site index inside a colour
    std::vector<int> pos(N);
    std::vector<uint16_t> pos2site(N);
    int cnt[2] = {0, 0};
    for (int i = 0; i < N; ++i) cnt[g.color[i]]++;
    if (cnt[0] != N / 2 || cnt[1] != N / 2) {
        destroy_batch(b);
        return fail(ctx, ICM_ERR_ARG, "colour classes are not balanced");
    }
    int next[2] = {0, N / 2};
    for (int i = 0; i < N; ++i) {
        pos[i] = next[g.color[i]]++;
        pos2site[pos[i]] = (uint16_t)i;
    }
    // incident bonds of every site in bond order, padded to Z with (self, -1)
    std::vector<std::vector<std::pair<int, int>>> inc(N);
    for (int e = 0; e < g.Nb; ++e) {
        if (g.color[g.bi[e]] == g.color[g.bj[e]]) {
            destroy_batch(b);
            return fail(ctx, ICM_ERR_ARG, "bond inside a colour class");
        }
        inc[g.bi[e]].push_back({g.bj[e], e});
        inc[g.bj[e]].push_back({g.bi[e], e});
    }
    std::vector<uint16_t> nbr((size_t)N * Z);
    std::vector<int32_t> edge_bond((size_t)N * Z);
    std::vector<uint8_t> zdeg(N);
    bool uniform = true;
    for (int i = 0; i < N; ++i) {
        const int deg = (int)inc[i].size();
        if (deg < 4 || deg > Z) {
            destroy_batch(b);
            return fail(ctx, ICM_ERR_UNSUPPORTED, "site degree outside 4..8");
        }
        if (deg != Z) uniform = false;
        const int p = pos[i];
        zdeg[p] = (uint8_t)deg;
        for (int d = 0; d < Z; ++d) {
            if (d < deg) {
                nbr[(size_t)p * Z + d] = (uint16_t)pos[inc[i][d].first];
                edge_bond[(size_t)p * Z + d] = inc[i][d].second;
            } else {
                nbr[(size_t)p * Z + d] = (uint16_t)p;
                edge_bond[(size_t)p * Z + d] = -1;
            }
        }
    }
    // launch shape: the shared-memory layout when several instances fit one
    // SM; the global-resident layout with wider CTAs when the instance does not
    // fit one CTA's shared memory, or fits only one or two CTAs per SM and has
    // more sites per colour than a shared-memory CTA has threads (there the
    // L1-cached wide CTA keeps more warps busy per SM)
    int n_icm = 0;
    while (n_icm < n_T && T[n_icm] <= T_icm) ++n_icm;
    int threads = icm::fused_threads(N);
    if (n_inst < ctx->num_sms) {
        // few instances: each CTA alone on its SM is latency-bound, so a tiny
        // instance gets a warp group per 16-bit pass (the passes run at once)
        const int gthr = (N / 2 + 31) / 32 * 32, npass = (R + 15) / 16;
        const int t = gthr * npass < icm::kMaxThreads ? gthr * npass : icm::kMaxThreads / gthr * gthr;
        if (t > threads) threads = t;
    }
    {
        const icm::SmemLayout sm0 = icm::smem_layout(N, Z, R, G, n_T, n_icm, threads / 32, b->gauss, false);
        bool wide = sm0.total > ctx->max_smem_optin;
        int c0 = 0;
        if (!wide && N / 2 > icm::kMaxThreads &&
            icm::fused_occupancy(b->gauss, Z, false, threads, sm0.total, &c0) == cudaSuccess && c0 <= 2)
            wide = true;
        (void)cudaGetLastError();
        if (wide) threads = icm::fused_threads_wide(N);
    }
    b->n_icm = n_icm;
    const int half = N / 2;

    // temperature tables
    TempTables tt;
    temperature_tables(T, n_T, g.Nb, Z, tt);
    if (!tt.swap_monotone) {
        destroy_batch(b);
        return fail(ctx, ICM_ERR_STATE, "swap thresholds not monotone in the energy difference");
    }
    std::vector<double> &beta = tt.beta;
    std::vector<uint32_t> &thr_metro = tt.thr_metro;
    std::vector<float> &b2l = tt.b2l, &dbeta_l2e = tt.dbeta_l2e;
    std::vector<uint32_t> &thr_swap = tt.thr_swap;
    std::vector<int32_t> &swap_off = tt.swap_off, &swap_len = tt.swap_len;
    b->thr_swap_cap = thr_swap.size();

    icm::KParams &P = b->kp;
    P.N = N; P.Nb = g.Nb; P.nT = n_T; P.R = R; P.G = G; P.Z = Z; P.n_inst = n_inst; P.n_icm = n_icm;
    P.half = half; P.NW = (N + 31) / 32; P.const_z = uniform ? Z : 0;
    b->uniform_z = P.const_z;
    P.seed_lo = (uint32_t)(seed & 0xffffffffu);
    P.seed_hi = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {                 // Philox round keys (Weyl sequence of the seed)
        P.key[2 * i] = P.seed_lo + (uint32_t)i * 0x9E3779B9u;
        P.key[2 * i + 1] = P.seed_hi + (uint32_t)i * 0xBB67AE85u;
    }
    {
        icm_status st0 = apply_threads(b, threads);
        if (st0) {
            destroy_batch(b);
            return st0;
        }
    }

    icm_status st = ICM_OK;
    uint16_t *d_nbr, *d_pos2site;
    uint8_t *d_zdeg, *d_Jb;
    float *d_Jd, *d_Ef, *d_b2l, *d_treb, *d_trea;
    int32_t *d_Ei, *d_off, *d_len, *d_trn, *d_trf, *d_trs, *d_trc;
    uint32_t *d_spins, *d_t, *d_id, *d_thr, *d_thrs;
    double *d_beta, *d_accE;
    float *d_dbl;
    long long *d_acc64, *d_nmeas;
    unsigned long long *d_hist, *d_icmst;
    uint8_t *d_trsw;
    uint16_t *d_nbr_inst;
    uint8_t *d_zdeg_inst;
    int32_t *d_nb_inst;
    const size_t nk = (size_t)n_inst * n_T;
    if ((st = dalloc(b, &d_nbr, (size_t)N * Z)) || (st = dalloc(b, &d_pos2site, N)) || (st = dalloc(b, &d_zdeg, N)) ||
        (st = dalloc(b, &b->edge_bond, (size_t)N * Z)) ||
        (st = dalloc(b, &d_Jb, b->gauss ? 1 : (size_t)n_inst * N)) ||
        (st = dalloc(b, &d_Jd, b->gauss ? (size_t)n_inst * N * Z : 1)) ||
        (st = dalloc(b, &d_spins, (size_t)n_inst * G * N)) || (st = dalloc(b, &d_Ef, (size_t)n_inst * R)) ||
        (st = dalloc(b, &d_Ei, (size_t)n_inst * R)) || (st = dalloc(b, &d_t, n_inst)) ||
        (st = dalloc(b, &d_id, n_inst)) || (st = dalloc(b, &d_thr, (size_t)R * icm::thr_stride(Z))) ||
        (st = dalloc(b, &d_b2l, R)) || (st = dalloc(b, &d_nbr_inst, (size_t)n_inst * N * Z)) ||
        (st = dalloc(b, &d_zdeg_inst, (size_t)n_inst * N)) || (st = dalloc(b, &d_nb_inst, n_inst)) ||
        (st = dalloc(b, &b->d_bad, n_inst)) ||
        (st = dalloc(b, &d_beta, n_T)) || (st = dalloc(b, &d_dbl, n_T - 1)) || (st = dalloc(b, &d_thrs, thr_swap.size())) ||
        (st = dalloc(b, &d_off, n_T - 1)) || (st = dalloc(b, &d_len, n_T - 1)) || (st = dalloc(b, &d_accE, nk)) ||
        (st = dalloc(b, &d_acc64, 4 * nk)) || (st = dalloc(b, &d_hist, nk * (N + 1))) ||
        (st = dalloc(b, &d_nmeas, n_inst)) || (st = dalloc(b, &d_icmst, 2 * (size_t)n_inst)) || (st = dalloc(b, &d_trn, nk)) || (st = dalloc(b, &d_trf, nk)) ||
        (st = dalloc(b, &d_trs, nk)) || (st = dalloc(b, &d_trc, nk)) || (st = dalloc(b, &d_treb, nk)) ||
        (st = dalloc(b, &d_trea, nk)) || (st = dalloc(b, &d_trsw, (size_t)n_inst * 2 * (n_T - 1))) ||
        (st = dalloc(b, (uint8_t **)&b->raw_coup, (size_t)n_inst * g.Nb * (b->gauss ? 4 : 1))) ||
        (st = dalloc(b, &b->raw_spins, (size_t)n_inst * R * N)) || (st = dalloc(b, &b->raw_E, (size_t)n_inst * R))) {
        destroy_batch(b);
        return st;
    }
    P.nbr = d_nbr; P.pos2site = d_pos2site; P.zdeg = d_zdeg; P.Jb = d_Jb; P.Jd = d_Jd; P.spins = d_spins;
    P.Ef = d_Ef; P.Ei = d_Ei; P.tsweep = d_t; P.inst_id = d_id; P.thr_metro = d_thr; P.b2l = d_b2l;
    P.beta = d_beta; P.dbeta_l2e = d_dbl; P.thr_swap = d_thrs; P.swap_off = d_off; P.swap_len = d_len; P.accE = d_accE;
    P.acc64 = d_acc64; P.hist = d_hist; P.n_meas = d_nmeas; P.icm_stats = d_icmst; P.tr_n_pre = d_trn; P.tr_flip2a = d_trf;
    P.tr_seed = d_trs; P.tr_csize = d_trc; P.tr_eb = d_treb; P.tr_ea = d_trea; P.tr_swap = d_trsw;
    P.nbr_inst = d_nbr_inst; P.zdeg_inst = d_zdeg_inst; P.nb_inst = d_nb_inst;
    b->h_nb.assign(n_inst, g.Nb);
    b->h_bad.assign(n_inst, 0);

    std::vector<uint32_t> ids(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        ids[i] = instance_ids ? instance_ids[i] : (uint32_t)i;
        if (ids[i] >= (1u << 24)) {
            destroy_batch(b);
            return fail(ctx, ICM_ERR_ARG, "instance ids must be < 2^24");
        }
    }
    cudaStream_t s = ctx->stream;
#define UP(dst, vec) cudaMemcpyAsync(dst, (vec).data(), (vec).size() * sizeof((vec)[0]), cudaMemcpyHostToDevice, s)
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = UP(d_nbr, nbr);
    if (e == cudaSuccess) e = UP(d_pos2site, pos2site);
    b->h_pos2site = pos2site;
    if (e == cudaSuccess) e = UP(d_zdeg, zdeg);
    if (e == cudaSuccess) e = UP(b->edge_bond, edge_bond);
    if (e == cudaSuccess) e = UP(d_id, ids);
    if (e == cudaSuccess) e = UP(d_thr, thr_metro);
    if (e == cudaSuccess) e = UP(d_b2l, b2l);
    if (e == cudaSuccess) e = UP(d_beta, beta);
    if (e == cudaSuccess) e = UP(d_dbl, dbeta_l2e);
    if (e == cudaSuccess) e = UP(d_thrs, thr_swap);
    if (e == cudaSuccess) e = UP(d_off, swap_off);
    if (e == cudaSuccess) e = UP(d_len, swap_len);
#undef UP
    if (e == cudaSuccess) e = cudaMemsetAsync(d_spins, 0, (size_t)n_inst * G * N * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_t, 0, (size_t)n_inst * 4, s);
    if (e != cudaSuccess) {
        destroy_batch(b);
        return cuda_fail(ctx, e, "batch upload");
    }
    std::vector<unsigned char> drawn;
    if (!couplings) generate_couplings(b->gauss, n_inst, g.Nb, ids.data(), seed, drawn);
    if ((st = clear_observables(b)) ||
        (st = couplings ? upload_state(b, couplings, spins, flags)
                        : upload_state(b, drawn.data(), nullptr, flags & ~ICM_DEVICE_PTR)) ||
        (!couplings && spins && (st = upload_state(b, nullptr, spins, flags)))) {
        destroy_batch(b);
        return st;
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        destroy_batch(b);
        return cuda_fail(ctx, e, "batch creation");
    }
    ctx->batches.insert(b);
    *out = b;
    return ICM_OK;
}

icm_status icm_batch_destroy(icm_batch *b)
{
    if (!b) return ICM_ERR_ARG;
    if (b->groups > 0)   // their captured launches still point at this batch's memory
        return fail(b->ctx, ICM_ERR_STATE, "the batch belongs to a group: destroy the group first");
    destroy_batch(b);
    return ICM_OK;
}

icm_status icm_batch_load(icm_batch *b, const void *couplings, const int8_t *spins, uint32_t t0, uint32_t flags)
{
    if (!b) return ICM_ERR_ARG;
    icm_status st;
    if ((st = upload_state(b, couplings, spins, flags))) return st;
    std::vector<uint32_t> t(b->n_inst, t0);
    ICM_CUDA(b->ctx, cudaMemcpyAsync(b->kp.tsweep, t.data(), t.size() * 4, cudaMemcpyHostToDevice, b->ctx->stream));
    if ((st = clear_observables(b))) return st;
    // the host vector above must outlive the copy
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_set_schedule(icm_batch *b, const icm_schedule *s)
{
    if (!b || !s) return ICM_ERR_ARG;
    if (s->icm_every < 0 || s->swap_every < 0) return fail(b->ctx, ICM_ERR_ARG, "negative schedule period");
    if (s->trace && !b->kp.tr_cmask) {       // the cluster words of the trace, allocated on first use
        uint32_t *cm = nullptr;
        icm_status st = dalloc(b, &cm, (size_t)b->n_inst * 2 * b->kp.N);
        if (st) return st;
        ICM_CUDA(b->ctx, cudaMemsetAsync(cm, 0, (size_t)b->n_inst * 2 * b->kp.N * 4, b->ctx->stream));
        b->kp.tr_cmask = cm;
    }
    b->sched = *s;
    return ICM_OK;
}

icm_status icm_get_schedule(const icm_batch *b, icm_schedule *s)
{
    if (!b || !s) return ICM_ERR_ARG;
    *s = b->sched;
    return ICM_OK;
}

icm_status icm_run_sweeps(icm_batch *b, uint32_t n_sweeps)
{
    if (!b) return ICM_ERR_ARG;
    for (int i = 0; i < b->n_inst; ++i)
        if (b->h_bad[i] && (b->h_active.empty() || b->h_active[i]))
            return fail(b->ctx, ICM_ERR_STATE, "instance " + std::to_string(i) + " holds invalid couplings");
    if (n_sweeps == 0) return ICM_OK;
    icm::KParams &P = b->kp;
    P.icm_every = b->sched.icm_every;
    P.swap_every = b->sched.swap_every;
    P.enable_2a = b->sched.enable_2a;
    P.enable_metropolis = b->sched.enable_metropolis;
    P.trace = b->sched.trace;
    P.t_meas = b->sched.t_meas;
    P.active = b->d_active;
    P.t_meas_inst = b->d_tmeas;
    ICM_CUDA(b->ctx, launch_batch(b, P, n_sweeps, b->ctx->stream));
    b->launches += 1;
    return ICM_OK;
}

icm_status icm_read_bond_counts(const icm_batch *b, int32_t *out)
{
    if (!b || !out) return ICM_ERR_ARG;
    for (int i = 0; i < b->n_inst; ++i) out[i] = b->h_nb[i];
    return ICM_OK;
}

icm_status icm_read_couplings(icm_batch *b, void *out, uint32_t flags)
{
    if (!b || !out) return ICM_ERR_ARG;
    const size_t bytes = (size_t)b->n_inst * b->kp.Nb * (b->gauss ? 4 : 1);
    icm_status st = copy_out(b->ctx, out, b->raw_coup, bytes, flags);
    if (st) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_read_spins(icm_batch *b, int8_t *out, uint32_t flags)
{
    if (!b || !out) return ICM_ERR_ARG;
    icm::KParams &P = b->kp;
    ICM_CUDA(b->ctx, icm::launch_unpack_spins(P.spins, b->raw_spins, P.pos2site, b->n_inst, P.R, P.G, P.N,
                                              b->ctx->stream));
    icm_status st = copy_out(b->ctx, out, b->raw_spins, (size_t)b->n_inst * P.R * P.N, flags);
    if (st) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_read_energies(icm_batch *b, double *out, uint32_t flags)
{
    if (!b || !out) return ICM_ERR_ARG;
    icm::KParams &P = b->kp;
    ICM_CUDA(b->ctx, icm::launch_energies_to_double(P, b->gauss, b->raw_E, b->ctx->stream));
    icm_status st = copy_out(b->ctx, out, b->raw_E, (size_t)b->n_inst * P.R * sizeof(double), flags);
    if (st) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_read_sweeps(icm_batch *b, uint32_t *out, uint32_t flags)
{
    if (!b || !out) return ICM_ERR_ARG;
    icm_status st = copy_out(b->ctx, out, b->kp.tsweep, (size_t)b->n_inst * 4, flags);
    if (st) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_read_observables(icm_batch *b, double *accE, int64_t *acc_n, int64_t *acc_q2, int64_t *acc_pmin,
                                int64_t *acc_d, int64_t *hist, int64_t *n_meas, uint32_t flags)
{
    if (!b) return ICM_ERR_ARG;
    icm::KParams &P = b->kp;
    const size_t nk = (size_t)b->n_inst * P.nT;
    icm_status st = ICM_OK;
    int64_t *outs[4] = {acc_n, acc_q2, acc_pmin, acc_d};
    if (accE && (st = copy_out(b->ctx, accE, P.accE, nk * 8, flags))) return st;
    for (int a = 0; a < 4; ++a)
        if (outs[a] && (st = copy_out(b->ctx, outs[a], P.acc64 + a * nk, nk * 8, flags))) return st;
    if (hist && (st = copy_out(b->ctx, hist, P.hist, nk * (P.N + 1) * 8, flags))) return st;
    if (n_meas && (st = copy_out(b->ctx, n_meas, P.n_meas, (size_t)b->n_inst * 8, flags))) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_read_overlaps(icm_batch *b, double *q_mean, double *q2_mean, double *ql_mean, int64_t *q_hist)
{
    if (!b) return ICM_ERR_ARG;
    icm::KParams &P = b->kp;
    const size_t nk = (size_t)b->n_inst * P.nT;
    std::vector<int64_t> acc(4 * nk), nm(b->n_inst);
    icm_status st = icm_read_observables(b, nullptr, acc.data(), acc.data() + nk, nullptr, acc.data() + 3 * nk,
                                         q_hist, nm.data(), 0u);
    if (st) return st;
    const double N = (double)P.N, nan = std::nan("");
    for (int i = 0; i < b->n_inst; ++i)
        for (int k = 0; k < P.nT; ++k) {
            const size_t o = (size_t)i * P.nT + k;
            const double m = (double)nm[i], nb = (double)b->h_nb[i];
            if (q_mean) q_mean[o] = m > 0 ? 1.0 - 2.0 * (double)acc[o] / (N * m) : nan;
            if (q2_mean) q2_mean[o] = m > 0 ? (double)acc[nk + o] / (N * N * m) : nan;
            if (ql_mean) ql_mean[o] = m > 0 && nb > 0 ? 1.0 - 2.0 * (double)acc[3 * nk + o] / (nb * m) : nan;
        }
    return ICM_OK;
}

icm_status icm_read_icm_stats(icm_batch *b, uint64_t *out, uint32_t flags)
{
    if (!b || !out) return ICM_ERR_ARG;
    icm_status st = copy_out(b->ctx, out, b->kp.icm_stats, (size_t)b->n_inst * 16, flags);
    if (st) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_clear_observables(icm_batch *b)
{
    if (!b) return ICM_ERR_ARG;
    return clear_observables(b);
}

icm_status icm_read_trace(icm_batch *b, int32_t *n_pre, int32_t *flip2a, int32_t *seed_site, int32_t *csize,
                          double *esum_before, double *esum_after, uint8_t *swap_acc, uint32_t flags)
{
    if (!b) return ICM_ERR_ARG;
    if (flags & ICM_DEVICE_PTR) return fail(b->ctx, ICM_ERR_ARG, "icm_read_trace takes host buffers");
    icm::KParams &P = b->kp;
    const size_t nk = (size_t)b->n_inst * P.nT;
    std::vector<float> eb(nk), ea(nk);
    icm_status st = ICM_OK;
    if (n_pre && (st = copy_out(b->ctx, n_pre, P.tr_n_pre, nk * 4, 0))) return st;
    if (flip2a && (st = copy_out(b->ctx, flip2a, P.tr_flip2a, nk * 4, 0))) return st;
    if (seed_site && (st = copy_out(b->ctx, seed_site, P.tr_seed, nk * 4, 0))) return st;
    if (csize && (st = copy_out(b->ctx, csize, P.tr_csize, nk * 4, 0))) return st;
    if ((st = copy_out(b->ctx, eb.data(), P.tr_eb, nk * 4, 0))) return st;
    if ((st = copy_out(b->ctx, ea.data(), P.tr_ea, nk * 4, 0))) return st;
    if (swap_acc && (st = copy_out(b->ctx, swap_acc, P.tr_swap, (size_t)b->n_inst * 2 * (P.nT - 1), 0))) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    for (size_t i = 0; i < nk; ++i) {
        if (esum_before) esum_before[i] = eb[i];
        if (esum_after) esum_after[i] = ea[i];
    }
    return ICM_OK;
}

icm_status icm_read_cluster_masks(icm_batch *b, uint8_t *out)
{
    if (!b || !out) return ICM_ERR_ARG;
    icm::KParams &P = b->kp;
    if (!P.tr_cmask) return fail(b->ctx, ICM_ERR_STATE, "no trace recorded (set the schedule's trace flag)");
    const size_t N = (size_t)P.N;
    std::vector<uint32_t> w((size_t)b->n_inst * 2 * N);
    icm_status st = copy_out(b->ctx, w.data(), P.tr_cmask, w.size() * 4, 0u);
    if (st) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    for (int i = 0; i < b->n_inst; ++i)
        for (int k = 0; k < P.nT; ++k) {
            uint8_t *o = out + ((size_t)i * P.nT + k) * N;
            const int word = k >> 4, bit = 2 * (k & 15);
            for (size_t p = 0; p < N; ++p)
                o[b->h_pos2site[p]] = (uint8_t)((w[((size_t)i * N + p) * 2 + word] >> bit) & 1u);
        }
    return ICM_OK;
}

// ---------------------------------------------------------------- per-slot control

static icm_status ensure_slot_arrays(icm_batch *b)
{
    if (b->d_active) return ICM_OK;
    icm_status st;
    if ((st = dalloc(b, &b->d_active, b->n_inst)) || (st = dalloc(b, &b->d_tmeas, b->n_inst))) return st;
    b->h_active.assign(b->n_inst, 1);
    b->h_tmeas.assign(b->n_inst, b->sched.t_meas);
    ICM_CUDA(b->ctx, cudaMemcpyAsync(b->d_active, b->h_active.data(), b->n_inst, cudaMemcpyHostToDevice,
                                     b->ctx->stream));
    ICM_CUDA(b->ctx, cudaMemcpyAsync(b->d_tmeas, b->h_tmeas.data(), b->n_inst * sizeof(long long),
                                     cudaMemcpyHostToDevice, b->ctx->stream));
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

static icm_status clear_slot_observables(icm_batch *b, int slot)
{
    icm_ctx *ctx = b->ctx;
    icm::KParams &P = b->kp;
    const size_t nT = P.nT, nk = (size_t)b->n_inst * nT;
    ICM_CUDA(ctx, cudaMemsetAsync(P.accE + slot * nT, 0, nT * sizeof(double), ctx->stream));
    for (int a = 0; a < 4; ++a)
        ICM_CUDA(ctx, cudaMemsetAsync(P.acc64 + a * nk + slot * nT, 0, nT * sizeof(long long), ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(P.hist + slot * nT * (P.N + 1), 0, nT * (P.N + 1) * sizeof(unsigned long long),
                                  ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(P.n_meas + slot, 0, sizeof(long long), ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(P.icm_stats + 2 * (size_t)slot, 0, 2 * sizeof(unsigned long long), ctx->stream));
    return ICM_OK;
}

static icm_status set_slot_flags(icm_batch *b, int slot)
{
    ICM_CUDA(b->ctx, cudaMemcpyAsync(b->d_active + slot, &b->h_active[slot], 1, cudaMemcpyHostToDevice,
                                     b->ctx->stream));
    ICM_CUDA(b->ctx, cudaMemcpyAsync(b->d_tmeas + slot, &b->h_tmeas[slot], sizeof(long long),
                                     cudaMemcpyHostToDevice, b->ctx->stream));
    return ICM_OK;
}

icm_status icm_batch_set_slot(icm_batch *b, int32_t slot, const void *couplings, const int8_t *spins,
                              uint32_t instance_id, uint32_t flags)
{
    if (!b) return ICM_ERR_ARG;
    if (slot < 0 || slot >= b->n_inst) return fail(b->ctx, ICM_ERR_ARG, "slot out of range");
    if (instance_id >= (1u << 24)) return fail(b->ctx, ICM_ERR_ARG, "instance ids must be < 2^24");
    icm_status st;
    if ((st = ensure_slot_arrays(b))) return st;
    icm_ctx *ctx = b->ctx;
    icm::KParams &P = b->kp;
    const size_t esz = b->gauss ? 4 : 1;
    unsigned char *raw_c = (unsigned char *)b->raw_coup + (size_t)slot * P.Nb * esz;
    std::vector<unsigned char> drawn;
    if (!couplings) generate_couplings(b->gauss, 1, P.Nb, &instance_id, b->seed, drawn);
    if ((st = couplings ? copy_in(ctx, raw_c, couplings, (size_t)P.Nb * esz, flags)
                        : copy_in(ctx, raw_c, drawn.data(), (size_t)P.Nb * esz, flags & ~ICM_DEVICE_PTR)))
        return st;
    float *Jd = b->gauss ? const_cast<float *>(P.Jd) + (size_t)slot * P.N * P.Z : nullptr;
    uint8_t *Jb = b->gauss ? nullptr : const_cast<uint8_t *>(P.Jb) + (size_t)slot * P.N;
    ICM_CUDA(ctx, icm::launch_expand_couplings(raw_c, b->gauss, b->edge_bond, 1, P.N, P.Z, P.Nb, Jd, Jb, ctx->stream));
    if ((st = refresh_dilution(b, slot, 1))) {
        if (!b->h_bad[slot]) return st;
        // invalid couplings: the slot is freed so that the other slots keep running
        b->h_active[slot] = 0;
        if (set_slot_flags(b, slot) == ICM_OK) cudaStreamSynchronize(ctx->stream);
        return st;
    }
    uint32_t *sp = P.spins + (size_t)slot * P.G * P.N;
    if (spins) {
        int8_t *raw_s = b->raw_spins + (size_t)slot * P.R * P.N;
        if ((st = copy_in(ctx, raw_s, spins, (size_t)P.R * P.N, flags))) return st;
        ICM_CUDA(ctx, icm::launch_pack_spins(raw_s, sp, P.pos2site, 1, P.R, P.G, P.N, ctx->stream));
    } else {
        ICM_CUDA(ctx, cudaMemsetAsync(sp, 0, (size_t)P.G * P.N * 4, ctx->stream));
    }
    icm::KParams Q = P;                        // the same kernels on this one slot
    Q.n_inst = 1;
    Q.spins = sp;
    Q.Jd = Jd;
    Q.Jb = Jb;
    Q.Ef = P.Ef + (size_t)slot * P.R;
    Q.Ei = P.Ei + (size_t)slot * P.R;
    Q.nbr_inst = P.nbr_inst + (size_t)slot * P.N * P.Z;
    Q.zdeg_inst = P.zdeg_inst + (size_t)slot * P.N;
    Q.nb_inst = P.nb_inst + slot;
    ICM_CUDA(ctx, icm::launch_init_energies(Q, b->gauss, ctx->stream));
    ICM_CUDA(ctx, cudaMemsetAsync(P.tsweep + slot, 0, 4, ctx->stream));
    ICM_CUDA(ctx, cudaMemcpyAsync(const_cast<uint32_t *>(P.inst_id) + slot, &instance_id, 4, cudaMemcpyHostToDevice,
                                  ctx->stream));
    if ((st = clear_slot_observables(b, slot))) return st;
    b->h_active[slot] = 1;
    b->h_tmeas[slot] = 0;
    if ((st = set_slot_flags(b, slot))) return st;
    ICM_CUDA(ctx, cudaStreamSynchronize(ctx->stream));   // host values above are read by the copies
    return ICM_OK;
}

icm_status icm_batch_set_active(icm_batch *b, int32_t slot, int32_t active)
{
    if (!b) return ICM_ERR_ARG;
    if (slot < -1 || slot >= b->n_inst) return fail(b->ctx, ICM_ERR_ARG, "slot out of range");
    icm_status st;
    if ((st = ensure_slot_arrays(b))) return st;
    if (slot == -1) {                                     // every slot
        std::fill(b->h_active.begin(), b->h_active.end(), (uint8_t)(active ? 1 : 0));
        ICM_CUDA(b->ctx, cudaMemcpyAsync(b->d_active, b->h_active.data(), b->n_inst, cudaMemcpyHostToDevice,
                                         b->ctx->stream));
        ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
        return ICM_OK;
    }
    b->h_active[slot] = active ? 1 : 0;
    if ((st = set_slot_flags(b, slot))) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_batch_start_window(icm_batch *b, int32_t slot, int64_t t_start)
{
    if (!b) return ICM_ERR_ARG;
    if (slot < 0 || slot >= b->n_inst) return fail(b->ctx, ICM_ERR_ARG, "slot out of range");
    icm_status st;
    if ((st = ensure_slot_arrays(b))) return st;
    if ((st = clear_slot_observables(b, slot))) return st;
    b->h_tmeas[slot] = t_start;
    if ((st = set_slot_flags(b, slot))) return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    return ICM_OK;
}

icm_status icm_therm_update(icm_therm_state *st, const icm_therm_criterion *c, double e, double q_l,
                            double T_min, double bonds_per_site, int32_t *thermalized)
{
    if (!st || !c || !thermalized || !(T_min > 0.0)) return ICM_ERR_ARG;
    for (int i = 2; i > 0; --i) {
        st->e[i] = st->e[i - 1];
        st->ql[i] = st->ql[i - 1];
    }
    st->e[0] = e;
    st->ql[0] = q_l;
    st->delta = -(bonds_per_site / T_min) * (1.0 - q_l) - e;   // Eq. 1 minus <H>/N (Eq. 2, one instance)
    st->blocks += 1;
    const bool agree = st->blocks >= 2 && std::fabs(st->e[0] - st->e[1]) <= c->eps_e &&
                       std::fabs(st->ql[0] - st->ql[1]) <= c->eps_ql;
    st->stable = agree ? st->stable + 1 : 0;
    *thermalized = st->stable >= c->need ? 1 : 0;
    return ICM_OK;
}

icm_status icm_batch_delta(icm_batch *b, int32_t k, double *delta_mean, double *delta_se, int32_t *n_used)
{
    if (!b || !delta_mean) return ICM_ERR_ARG;
    icm::KParams &P = b->kp;
    if (k < 0 || k >= P.nT) return fail(b->ctx, ICM_ERR_ARG, "temperature index out of range");
    const size_t nk = (size_t)b->n_inst * P.nT;
    std::vector<double> accE(nk);
    std::vector<long long> accd(nk), nm(b->n_inst);
    icm_status st;
    if ((st = copy_out(b->ctx, accE.data(), P.accE, nk * 8, 0)) ||
        (st = copy_out(b->ctx, accd.data(), P.acc64 + 3 * nk, nk * 8, 0)) ||
        (st = copy_out(b->ctx, nm.data(), P.n_meas, (size_t)b->n_inst * 8, 0)))
        return st;
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    const double N = P.N, T = b->T[k];
    double s1 = 0, s2 = 0;
    int n = 0;
    for (int i = 0; i < b->n_inst; ++i) {
        if (nm[i] <= 0 || (!b->h_active.empty() && !b->h_active[i])) continue;
        const double Nb = b->h_nb[i] > 0 ? (double)b->h_nb[i] : 1.0;   // bonds present
        const double m = (double)nm[i];
        const double e = accE[(size_t)i * P.nT + k] / (2.0 * N * m);
        const double ql = 1.0 - 2.0 * (double)accd[(size_t)i * P.nT + k] / (Nb * m);
        const double d = -(Nb / N) * (1.0 - ql) / T - e;
        s1 += d;
        s2 += d * d;
        ++n;
    }
    if (n == 0) return fail(b->ctx, ICM_ERR_STATE, "no measured instance");
    *delta_mean = s1 / n;
    if (delta_se) *delta_se = n > 1 ? std::sqrt(std::fmax(s2 / n - (s1 / n) * (s1 / n), 0.0) / (n - 1)) : 0.0;
    if (n_used) *n_used = n;
    return ICM_OK;
}

// ---------------------------------------------------------------- launch shape, groups, autotuning

// Widths up to 128 threads use the shared-memory layout; wider CTAs (up to
// 1024 threads) use the global-resident layout, which is also the only one
// for instances that do not fit one CTA's shared memory.
static icm_status apply_threads(icm_batch *b, int threads)
{
    icm::KParams &P = b->kp;
    if (threads < 32 || threads > icm::kMaxThreadsWide || threads % 32)
        return fail(b->ctx, ICM_ERR_ARG, "threads per CTA must be a multiple of 32 in 32..1024");
    const int half = P.N / 2;
    if (((half + threads - 1) / threads) * P.Z >= 256 || (P.N + threads - 1) / threads >= 256)
        return fail(b->ctx, ICM_ERR_UNSUPPORTED, "too many sites per thread for the observable counters");
    const bool wide = threads > icm::kMaxThreads;
    const icm::SmemLayout sm = icm::smem_layout(P.N, P.Z, P.R, P.G, P.nT, b->n_icm, threads / 32, b->gauss, wide);
    if (sm.total > b->ctx->max_smem_optin)
        return fail(b->ctx, ICM_ERR_UNSUPPORTED, "instance needs " + std::to_string(sm.total) +
                                                     " bytes of shared memory at this width; widths above 128 "
                                                     "threads keep it in global memory");
    int ctas = 0;
    cudaError_t e = icm::fused_occupancy(b->gauss, P.Z, wide, threads, sm.total, &ctas);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "occupancy");
    if (ctas < 1) return fail(b->ctx, ICM_ERR_UNSUPPORTED, "kernel does not fit");
    const int slots = b->ctx->num_sms * ctas;
    const int grid = b->n_inst < slots ? b->n_inst : slots;
    const int words = icm::wide_scratch_words(P.N);
    if (wide && b->scratch_ctas < grid) {
        // a larger scratch; the old one stays allocated until the batch is
        // destroyed, since a captured group graph may still launch with it
        uint32_t *q = nullptr;
        icm_status ast = dalloc(b, &q, (size_t)grid * words);
        if (ast) return ast;
        b->scratch = q;
        b->scratch_ctas = grid;
    }
    b->cluster_k = 0;
    b->n_clusters = 0;
    P.sm = sm;
    P.wide = wide ? 1 : 0;
    P.scratch = wide ? b->scratch : nullptr;
    P.scratch_words = wide ? words : 0;
    P.small_counts = (((half + threads - 1) / threads) * P.Z < 16 && (P.N + threads - 1) / threads < 16) ? 1 : 0;
    b->threads = threads;
    b->ctas_per_sm = ctas;
    b->grid = grid;
    return ICM_OK;
}

// One instance per thread-block cluster of K CTAs (K = 2, 4, 8) of `threads`
// threads each; see cluster_icm.cu.  K = 0 returns to one CTA per instance.
static icm_status apply_cluster(icm_batch *b, int K, int threads)
{
    icm::KParams &P = b->kp;
    if (K == 0) return apply_threads(b, threads);
    if (K != 2 && K != 4 && K != 8) return fail(b->ctx, ICM_ERR_ARG, "cluster size must be 2, 4 or 8");
    if (threads < 32 || threads > icm::kMaxThreadsWide || threads % 32)
        return fail(b->ctx, ICM_ERR_ARG, "threads per CTA must be a multiple of 32 in 32..1024");
    if (P.Z != 4 && P.Z != 6 && P.Z != 8) return fail(b->ctx, ICM_ERR_UNSUPPORTED, "the cluster layout takes degrees 4, 6 and 8");
    const int half = P.N / 2;
    if (half % K || (half / K) % 32)
        return fail(b->ctx, ICM_ERR_UNSUPPORTED, "sites per colour must split into K blocks of a multiple of 32");
    const int hs = half / K;
    if (((hs + threads - 1) / threads) * P.Z >= 256 || (2 * hs + threads - 1) / threads >= 256)
        return fail(b->ctx, ICM_ERR_UNSUPPORTED, "too many sites per thread for the observable counters");
    // union-find growth (on request) takes one pair's labels in the place of
    // the overlap masks, so one pair per group costs no shared memory; a
    // group takes the most pairs (up to kMaxUfGroup) that keep as many
    // clusters resident
    const int ufg1 = b->cl_growth == 1 ? 1 : 0;
    // 2D lattices whose CTAs hold whole pairs of rows, four sites per thread:
    // each thread grows a 2 x 2 block of sites, around the block
    // (a (x0, y0), b (x0 + 1, y0), d (x0 + 1, y0 + 1), c (x0, y0 + 1)),
    // threads along the rows; local index of (x, y) in a CTA's rows: colour
    // c = (x + y) & 1, c hs + y L / 2 + x / 2 (rows per CTA even, so the
    // colour of a local row is that of the lattice row)
    const int Lx = b->L, nls = 2 * hs;
    const bool order = b->lattice == ICM_SQUARE2D && hs % (Lx / 2) == 0 && (hs / (Lx / 2)) % 2 == 0 &&
                       nls == 4 * threads;
    std::vector<uint16_t> ord;
    if (order) {
        ord.assign(nls, 0);
        std::vector<uint8_t> seen(nls, 0);
        const int dy[4] = {0, 0, 1, 1}, dx[4] = {0, 1, 1, 0};
        for (int t = 0; t < threads; ++t)
            for (int j = 0; j < 4; ++j) {
                const int y = 2 * (t / (Lx / 2)) + dy[j], x = 2 * (t % (Lx / 2)) + dx[j];
                const int li = ((x + y) & 1) * hs + y * (Lx / 2) + x / 2;
                if (li >= nls || seen[li]) return fail(b->ctx, ICM_ERR_STATE, "growth order is not a permutation");
                seen[li] = 1;
                ord[(size_t)4 * t + j] = (uint16_t)li;
            }
        if (!b->d_cl_order) {
            icm_status st = dalloc(b, &b->d_cl_order, (size_t)P.N);
            if (st) return st;
        }
        ICM_CUDA(b->ctx, cudaMemcpyAsync(b->d_cl_order, ord.data(), ord.size() * 2, cudaMemcpyHostToDevice,
                                         b->ctx->stream));
        ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));   // the host table is read by the copy
    }
    icm::ClusterLayout L = icm::cluster_layout(P.N, P.Z, P.R, P.G, P.nT, K, threads / 32, b->gauss, ufg1, order);
    if (L.total > b->ctx->max_smem_optin) return fail(b->ctx, ICM_ERR_UNSUPPORTED, "cluster slice exceeds shared memory");
    int clusters = 0;
    cudaError_t e = icm::cluster_occupancy(b->gauss, P.Z, P.diluted != 0, K, threads, L.total, &clusters);
    if (e != cudaSuccess) return cuda_fail(b->ctx, e, "cluster occupancy");
    if (clusters < 1) return fail(b->ctx, ICM_ERR_UNSUPPORTED, "cluster does not fit");
    for (int g = 2; ufg1 && g <= icm::kMaxUfGroup && g <= (P.n_icm > 1 ? P.n_icm : 1); ++g) {
        const icm::ClusterLayout Lg = icm::cluster_layout(P.N, P.Z, P.R, P.G, P.nT, K, threads / 32, b->gauss, g,
                                                          order);
        int cg = 0;
        if (Lg.total > b->ctx->max_smem_optin ||
            icm::cluster_occupancy(b->gauss, P.Z, P.diluted != 0, K, threads, Lg.total, &cg) != cudaSuccess ||
            cg < clusters)
            break;
        L = Lg;
    }
    b->cluster_k = K;
    b->cl = L;
    P.cl_order = order ? b->d_cl_order : nullptr;
    b->threads = threads;
    b->n_clusters = b->n_inst < clusters ? b->n_inst : clusters;
    b->grid = b->n_clusters * K;
    // CTAs per SM when the most clusters are resident
    b->ctas_per_sm = (clusters * K + b->ctx->num_sms - 1) / b->ctx->num_sms;
    P.small_counts = 0;
    return ICM_OK;
}

icm_status icm_batch_set_cluster(icm_batch *b, int32_t K, int32_t threads)
{
    if (!b) return ICM_ERR_ARG;
    return apply_cluster(b, K, threads);
}

icm_status icm_batch_cluster(const icm_batch *b, int32_t *K)
{
    if (!b || !K) return ICM_ERR_ARG;
    *K = b->cluster_k;
    return ICM_OK;
}

icm_status icm_batch_set_cluster_growth(icm_batch *b, int32_t mode)
{
    if (!b) return ICM_ERR_ARG;
    if (mode < -1 || mode > 1) return fail(b->ctx, ICM_ERR_ARG, "cluster growth must be -1, 0 or 1");
    const int was = b->cl_growth;
    b->cl_growth = mode;
    if (!b->cluster_k) return ICM_OK;
    const icm_status st = apply_cluster(b, b->cluster_k, b->threads);
    if (st) {
        b->cl_growth = was;
        apply_cluster(b, b->cluster_k, b->threads);
    }
    return st;
}

icm_status icm_batch_cluster_growth(const icm_batch *b, int32_t *pairs_per_group)
{
    if (!b || !pairs_per_group) return ICM_ERR_ARG;
    *pairs_per_group = b->cluster_k ? b->cl.ufg : 0;
    return ICM_OK;
}

icm_status icm_batch_set_threads(icm_batch *b, int32_t threads)
{
    if (!b) return ICM_ERR_ARG;
    return apply_threads(b, threads);
}

icm_status icm_batch_autotune(icm_batch *b, uint32_t sweeps, int32_t *best_threads, float *best_ms)
{
    if (!b || sweeps == 0) return ICM_ERR_ARG;
    icm_ctx *ctx = b->ctx;
    icm::KParams &P = b->kp;
    const size_t nk = (size_t)b->n_inst * P.nT;
    // snapshot of everything a launch changes, restored after the trials
    struct Piece { void *dst; size_t bytes; void *save; };
    Piece pieces[] = {
        {P.spins, (size_t)b->n_inst * P.G * P.N * 4, nullptr},
        {b->gauss ? (void *)P.Ef : (void *)P.Ei, (size_t)b->n_inst * P.R * 4, nullptr},
        {P.tsweep, (size_t)b->n_inst * 4, nullptr},
        {P.accE, nk * 8, nullptr},
        {P.acc64, 4 * nk * 8, nullptr},
        {P.hist, nk * (P.N + 1) * 8, nullptr},
        {P.n_meas, (size_t)b->n_inst * 8, nullptr},
        {P.icm_stats, (size_t)b->n_inst * 16, nullptr},
    };
    icm_status st = ICM_OK;
    for (auto &pc : pieces) {
        if ((st = ctx_alloc(ctx, &pc.save, pc.bytes))) break;
        if (cudaMemcpyAsync(pc.save, pc.dst, pc.bytes, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
            st = fail(ctx, ICM_ERR_CUDA, "autotune snapshot copy");
            break;
        }
    }
    const int original = b->threads;
    int best = original;
    float best_t = 1e30f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!st && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(ctx, ICM_ERR_CUDA, "events");
    // the shared-memory widths when the instance fits them; wide CTAs when it
    // does not, or when a colour has more sites than 128 threads
    const bool fits = icm::smem_layout(P.N, P.Z, P.R, P.G, P.nT, b->n_icm, icm::kMaxThreads / 32, b->gauss,
                                       false).total <= ctx->max_smem_optin;
    // (cluster size, CTA width) candidates: one CTA per instance in shared
    // memory when it fits, wide CTAs when a colour has more than 128 sites,
    // and thread-block clusters for those large instances too
    std::vector<std::pair<int, int>> cand;
    if (fits)
        for (int th : {32, 64, 96, 128}) cand.push_back({0, th});
    if (!fits || P.N / 2 > icm::kMaxThreads) {
        for (int th : {256, 512, 1024}) cand.push_back({0, th});
        for (int K : {4, 8})
            for (int th : {256, 512}) cand.push_back({K, th});
    }
    const int original_k = b->cluster_k;
    int best_k = original_k;
    for (size_t ci = 0; !st && ci < cand.size(); ++ci) {
        const int K = cand[ci].first, th = cand[ci].second;
        if (apply_cluster(b, K, th) != ICM_OK) continue;
        if ((st = icm_run_sweeps(b, sweeps))) break;               // warm-up
        cudaEventRecord(e0, ctx->stream);
        if ((st = icm_run_sweeps(b, sweeps))) break;
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_t) {
            best_t = ms;
            best = th;
            best_k = K;
        }
        b->launches -= 2;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (auto &pc : pieces)
        if (pc.save) {
            cudaMemcpyAsync(pc.dst, pc.save, pc.bytes, cudaMemcpyDeviceToDevice, ctx->stream);
        }
    cudaStreamSynchronize(ctx->stream);
    for (auto &pc : pieces)
        if (pc.save) ctx_free(ctx, pc.save, pc.bytes);
    icm_status st2 = st ? apply_cluster(b, original_k, original) : apply_cluster(b, best_k, best);
    if (st) return st;
    if (st2) return st2;
    if (best_threads) *best_threads = best;
    if (best_ms) *best_ms = best_t;
    return ICM_OK;
}

}  // extern "C"

struct icm_group {
    icm_ctx *ctx = nullptr;
    std::vector<icm_batch *> batches;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t sweeps = 0;
    int64_t launches = 0;
    // shared form: one launch of the team kernel over every batch's instances
    bool shared = false;
    void *d_items = nullptr;               // icm::TeamItem [n_items] (device)
    size_t items_bytes = 0;
    std::vector<int> team_threads, tile;   // per batch: threads per instance, instances per tile
    int grid = 0, smem = 0, n_items = 0;
    bool counted = false;                  // the batches count this group (icm_batch::groups)
};

static void destroy_group(icm_group *g)
{
    if (!g) return;
    if (g->counted)
        for (auto *b : g->batches) --b->groups;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (auto e : g->events) cudaEventDestroy(e);
    for (auto s : g->streams) cudaStreamDestroy(s);
    if (g->d_items) ctx_free(g->ctx, g->d_items, g->items_bytes);
    delete g;
}

// Instances per tile of a batch in the shared group kernel at `w` threads per
// instance (0 if it does not fit), and the batch's parameters laid out for
// that width.
static int team_fit(const icm_batch *b, int w, int max_smem, icm::KParams &P)
{
    const icm::KParams &B = b->kp;
    if (w < 32 || w % 32 || icm::kTeamThreads % w) return 0;
    const int half = B.N / 2;
    if (((half + w - 1) / w) * B.Z >= 256 || (B.N + w - 1) / w >= 256) return 0;   // observable counters
    const icm::SmemLayout sm = icm::smem_layout(B.N, B.Z, B.R, B.G, B.nT, b->n_icm, w / 32, b->gauss, false);
    int k = icm::kTeamThreads / w;
    if (k * sm.total > max_smem) k = max_smem / sm.total;
    if (k < 1) return 0;
    P = B;
    P.sm = sm;
    P.wide = 0;
    P.scratch = nullptr;
    P.scratch_words = 0;
    P.small_counts = (((half + w - 1) / w) * B.Z < 16 && (B.N + w - 1) / w < 16) ? 1 : 0;
    return k;
}

extern "C" {

icm_status icm_group_create(icm_ctx *ctx, icm_batch *const *batches, int32_t n, uint32_t sweeps_per_launch,
                            icm_group **out)
{
    if (!ctx || !batches || n < 1 || !out || sweeps_per_launch == 0) return ICM_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!batches[i] || batches[i]->ctx != ctx) return fail(ctx, ICM_ERR_ARG, "batches must belong to the context");
    icm_group *g = new (std::nothrow) icm_group();
    if (!g) return ICM_ERR_OOM;
    g->ctx = ctx;
    g->batches.assign(batches, batches + n);
    g->sweeps = sweeps_per_launch;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        cudaStream_t s;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) g->streams.push_back(s);
    }
    for (int i = 0; i < n + 1 && e == cudaSuccess; ++i) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) g->events.push_back(ev);
    }
    // capture: fork one stream per batch from the context stream, join back
    cudaStream_t origin = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(g->events[n], origin);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        icm_batch *b = g->batches[i];
        e = cudaStreamWaitEvent(g->streams[i], g->events[n], 0);
        if (e != cudaSuccess) break;
        icm::KParams P = b->kp;
        P.icm_every = b->sched.icm_every;
        P.swap_every = b->sched.swap_every;
        P.enable_2a = b->sched.enable_2a;
        P.enable_metropolis = b->sched.enable_metropolis;
        P.trace = b->sched.trace;
        P.t_meas = b->sched.t_meas;
        P.active = b->d_active;
        P.t_meas_inst = b->d_tmeas;
        e = launch_batch(b, P, sweeps_per_launch, g->streams[i]);
        if (e == cudaSuccess) e = cudaEventRecord(g->events[i], g->streams[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, g->events[i], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(origin, &graph);
    if (e == cudaSuccess) e = ec;
    g->graph = graph;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (origin) cudaStreamDestroy(origin);
    if (e != cudaSuccess) {
        destroy_group(g);
        return cuda_fail(ctx, e, "group capture");
    }
    for (auto *b : g->batches) ++b->groups;
    g->counted = true;
    *out = g;
    return ICM_OK;
}

icm_status icm_group_create_shared(icm_ctx *ctx, icm_batch *const *batches, int32_t n, uint32_t sweeps_per_launch,
                                   const int32_t *team_threads, icm_group **out)
{
    if (!ctx || !batches || n < 1 || !out || sweeps_per_launch == 0) return ICM_ERR_ARG;
    *out = nullptr;
    if (n > icm::kTeamClasses)
        return fail(ctx, ICM_ERR_UNSUPPORTED, "a shared group takes at most " + std::to_string(icm::kTeamClasses) +
                                                  " batches");
    for (int i = 0; i < n; ++i) {
        const icm_batch *b = batches[i];
        if (!b || b->ctx != ctx) return fail(ctx, ICM_ERR_ARG, "batches must belong to the context");
        if (b->gauss != batches[0]->gauss || b->kp.Z != batches[0]->kp.Z)
            return fail(ctx, ICM_ERR_UNSUPPORTED, "a shared group takes one disorder kind and one lattice degree");
        if (b->seed != batches[0]->seed)
            return fail(ctx, ICM_ERR_UNSUPPORTED, "a shared group takes batches of one seed (instance ids tell them apart)");
        if (b->cluster_k || b->kp.diluted)
            return fail(ctx, ICM_ERR_UNSUPPORTED, "a shared group takes undiluted batches outside the cluster layout");
    }
    icm_group *g = new (std::nothrow) icm_group();
    if (!g) return ICM_ERR_OOM;
    std::unique_ptr<icm::TeamParams> TP(new (std::nothrow) icm::TeamParams());
    if (!TP) {
        delete g;
        return ICM_ERR_OOM;
    }
    g->ctx = ctx;
    g->batches.assign(batches, batches + n);
    g->sweeps = sweeps_per_launch;
    g->shared = true;
    for (int i = 0; i < 20; ++i) TP->key[i] = batches[0]->kp.key[i];
    // per batch: threads per instance (given, or the width that keeps most
    // threads of the CTA busy, the narrower on a tie) and instances per tile
    static const int kWidths[] = {32, 64, 128, 224, 448, 896};
    std::vector<icm::TeamItem> items;
    std::vector<double> work;
    for (int c = 0; c < n; ++c) {
        icm_batch *b = batches[c];
        int best_w = 0, best_k = 0;
        icm::KParams best{}, P{};
        if (team_threads && team_threads[c] > 0) {
            best_k = team_fit(b, team_threads[c], ctx->max_smem_optin, best);
            best_w = team_threads[c];
        } else {
            for (int w : kWidths) {
                const int k = team_fit(b, w, ctx->max_smem_optin, P);
                if (k > 0 && k * w > best_k * best_w) {
                    best_w = w;
                    best_k = k;
                    best = P;
                }
            }
        }
        if (best_k < 1) {
            destroy_group(g);
            return fail(ctx, ICM_ERR_UNSUPPORTED, "batch " + std::to_string(c) +
                                                      ": no team width (a divisor of " +
                                                      std::to_string(icm::kTeamThreads) +
                                                      ") fits the shared memory and the counters");
        }
        best.icm_every = b->sched.icm_every;
        best.swap_every = b->sched.swap_every;
        best.enable_2a = b->sched.enable_2a;
        best.enable_metropolis = b->sched.enable_metropolis;
        best.trace = b->sched.trace;
        best.t_meas = b->sched.t_meas;
        best.active = b->d_active;
        best.t_meas_inst = b->d_tmeas;
        TP->cls[c] = best;
        TP->team_threads[c] = best_w;
        g->team_threads.push_back(best_w);
        g->tile.push_back(best_k);
        g->smem = std::max(g->smem, best_k * best.sm.total);
        for (int s0 = 0; s0 < b->n_inst; s0 += best_k) {
            items.push_back({c, s0, std::min(best_k, b->n_inst - s0)});
            work.push_back((double)items.back().count * best.N * best.R);
        }
    }
    // the tiles in descending order of work (spin updates per sweep): the
    // CTAs take the next one whenever they are free, largest first
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
    std::vector<icm::TeamItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    g->n_items = (int)sorted.size();
    // tile list, then the two work counters (16-byte aligned after it)
    const size_t list_bytes = (sorted.size() * sizeof(icm::TeamItem) + 15) / 16 * 16;
    g->items_bytes = list_bytes + 16;
    icm_status st = ctx_alloc(ctx, &g->d_items, g->items_bytes);
    if (st) {
        g->d_items = nullptr;
        destroy_group(g);
        return st;
    }
    cudaError_t e = cudaMemcpy(g->d_items, sorted.data(), sorted.size() * sizeof(icm::TeamItem),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset((char *)g->d_items + list_bytes, 0, 16);
    TP->items = (const icm::TeamItem *)g->d_items;
    TP->n_items = g->n_items;
    TP->counters = (int *)((char *)g->d_items + list_bytes);
    int ctas = 0;
    if (e == cudaSuccess) e = icm::team_occupancy(batches[0]->gauss, batches[0]->kp.Z, g->smem, &ctas);
    if (e == cudaSuccess && ctas < 1) {
        destroy_group(g);
        return fail(ctx, ICM_ERR_UNSUPPORTED, "the shared group kernel does not fit an SM");
    }
    g->grid = std::min(g->n_items, ctx->num_sms * ctas);
    // capture the one launch
    cudaStream_t origin = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = icm::launch_team(*TP, batches[0]->gauss, batches[0]->kp.Z, g->grid, g->smem, sweeps_per_launch, origin);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(origin, &graph);
        if (e == cudaSuccess) e = ec;
        g->graph = graph;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (origin) cudaStreamDestroy(origin);
    if (e != cudaSuccess) {
        destroy_group(g);
        return cuda_fail(ctx, e, "shared group capture");
    }
    for (auto *b : g->batches) ++b->groups;
    g->counted = true;
    *out = g;
    return ICM_OK;
}

icm_status icm_group_info(const icm_group *g, int32_t *team_threads, int32_t *tile, int32_t *grid, int32_t *smem,
                          int32_t *n_items)
{
    if (!g) return ICM_ERR_ARG;
    for (size_t c = 0; c < g->batches.size(); ++c) {
        if (team_threads) team_threads[c] = g->shared ? g->team_threads[c] : g->batches[c]->threads;
        if (tile) tile[c] = g->shared ? g->tile[c] : 1;
    }
    if (grid) *grid = g->shared ? g->grid : 0;
    if (smem) *smem = g->shared ? g->smem : 0;
    if (n_items) *n_items = g->shared ? g->n_items : 0;
    return ICM_OK;
}

icm_status icm_group_run(icm_group *g, uint32_t n_launches)
{
    if (!g) return ICM_ERR_ARG;
    for (uint32_t i = 0; i < n_launches; ++i) {
        ICM_CUDA(g->ctx, cudaGraphLaunch(g->exec, g->ctx->stream));
        g->launches += 1;
        for (auto *b : g->batches) b->launches += 1;
    }
    return ICM_OK;
}

icm_status icm_group_destroy(icm_group *g)
{
    if (!g) return ICM_ERR_ARG;
    cudaStreamSynchronize(g->ctx->stream);
    destroy_group(g);
    return ICM_OK;
}

icm_status icm_set_temperatures(icm_batch *b, const double *T, int32_t n_T, double T_icm)
{
    if (!b || !T) return ICM_ERR_ARG;
    icm::KParams &P = b->kp;
    if (n_T != P.nT) return fail(b->ctx, ICM_ERR_ARG, "a batch keeps its number of temperatures");
    for (int k = 0; k < n_T; ++k) {
        if (!(T[k] > 0.0) || !std::isfinite(T[k])) return fail(b->ctx, ICM_ERR_ARG, "temperatures must be finite and > 0");
        if (k && !(T[k] > T[k - 1])) return fail(b->ctx, ICM_ERR_ARG, "temperatures must be strictly ascending");
    }
    TempTables tt;
    temperature_tables(T, n_T, P.Nb, P.Z, tt);
    if (!tt.swap_monotone) return fail(b->ctx, ICM_ERR_STATE, "swap thresholds not monotone in the energy difference");
    icm_status st;
    if (tt.thr_swap.size() > b->thr_swap_cap) {
        uint32_t *d = nullptr;
        if ((st = dalloc(b, &d, tt.thr_swap.size()))) return st;
        P.thr_swap = d;
        b->thr_swap_cap = tt.thr_swap.size();
    }
    cudaStream_t s = b->ctx->stream;
#define UPV(dst, vec) cudaMemcpyAsync((void *)(dst), (vec).data(), (vec).size() * sizeof((vec)[0]), cudaMemcpyHostToDevice, s)
    ICM_CUDA(b->ctx, UPV(P.thr_metro, tt.thr_metro));
    ICM_CUDA(b->ctx, UPV(P.b2l, tt.b2l));
    ICM_CUDA(b->ctx, UPV(P.beta, tt.beta));
    ICM_CUDA(b->ctx, UPV(P.dbeta_l2e, tt.dbeta_l2e));
    ICM_CUDA(b->ctx, UPV(P.thr_swap, tt.thr_swap));
    ICM_CUDA(b->ctx, UPV(P.swap_off, tt.swap_off));
    ICM_CUDA(b->ctx, UPV(P.swap_len, tt.swap_len));
#undef UPV
    ICM_CUDA(b->ctx, cudaStreamSynchronize(s));   // the host tables are read by the copies
    int n_icm = 0;
    while (n_icm < n_T && T[n_icm] <= T_icm) ++n_icm;
    b->T.assign(T, T + n_T);
    b->T_icm = T_icm;
    b->n_icm = n_icm;
    P.n_icm = n_icm;
    // the shared-memory layout depends on n_icm; a clustered batch stays clustered
    return b->cluster_k ? apply_cluster(b, b->cluster_k, b->threads) : apply_threads(b, b->threads);
}

// ---------------------------------------------------------------- checkpoint / resume

namespace {
struct BlobHeader {
    char magic[8];            // "ICMPTCK1"
    uint32_t version;         // 1
    int32_t lattice, L, disorder, n_inst, nT, N, R, G;
    int32_t has_slots;
    uint64_t seed;
    double T_icm;
    icm_schedule sched;
};

struct BlobPart {
    void *dev;
    size_t bytes;
};

std::vector<BlobPart> blob_parts(icm_batch *b)
{
    icm::KParams &P = b->kp;
    const size_t nk = (size_t)b->n_inst * P.nT;
    std::vector<BlobPart> v = {
        {b->raw_coup, (size_t)b->n_inst * P.Nb * (b->gauss ? 4 : 1)},
        {P.spins, (size_t)b->n_inst * P.G * P.N * 4},
        {b->gauss ? (void *)P.Ef : (void *)P.Ei, (size_t)b->n_inst * P.R * 4},
        {P.tsweep, (size_t)b->n_inst * 4},
        {const_cast<uint32_t *>(P.inst_id), (size_t)b->n_inst * 4},
        {P.accE, nk * 8},
        {P.acc64, 4 * nk * 8},
        {P.hist, nk * (P.N + 1) * 8},
        {P.n_meas, (size_t)b->n_inst * 8},
    };
    if (b->d_active) {
        v.push_back({b->d_active, (size_t)b->n_inst});
        v.push_back({b->d_tmeas, (size_t)b->n_inst * 8});
    }
    return v;
}
}  // namespace

icm_status icm_save(icm_batch *b, void *buf, size_t *len)
{
    if (!b || !len) return ICM_ERR_ARG;
    const std::vector<BlobPart> parts = blob_parts(b);
    size_t need = sizeof(BlobHeader) + b->nT * sizeof(double);
    for (const auto &pt : parts) need += pt.bytes;
    if (!buf) {
        *len = need;
        return ICM_OK;
    }
    if (*len < need) return fail(b->ctx, ICM_ERR_ARG, "checkpoint buffer too small");
    BlobHeader h{};
    std::memcpy(h.magic, "ICMPTCK1", 8);
    h.version = 1;
    h.lattice = b->lattice; h.L = b->L; h.disorder = b->disorder; h.n_inst = b->n_inst; h.nT = b->nT;
    h.N = b->kp.N; h.R = b->kp.R; h.G = b->kp.G; h.has_slots = b->d_active ? 1 : 0;
    h.seed = b->seed; h.T_icm = b->T_icm; h.sched = b->sched;
    unsigned char *o = (unsigned char *)buf;
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    std::memcpy(o, b->T.data(), b->nT * sizeof(double));
    o += b->nT * sizeof(double);
    for (const auto &pt : parts) {
        ICM_CUDA(b->ctx, cudaMemcpyAsync(o, pt.dev, pt.bytes, cudaMemcpyDeviceToHost, b->ctx->stream));
        o += pt.bytes;
    }
    ICM_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
    *len = need;
    return ICM_OK;
}

icm_status icm_load(icm_batch *b, const void *buf, size_t len)
{
    if (!b || !buf) return ICM_ERR_ARG;
    BlobHeader h;
    if (len < sizeof h) return fail(b->ctx, ICM_ERR_ARG, "checkpoint too short");
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, "ICMPTCK1", 8) || h.version != 1) return fail(b->ctx, ICM_ERR_ARG, "not a checkpoint of this library");
    if (h.lattice != b->lattice || h.L != b->L || h.disorder != b->disorder || h.n_inst != b->n_inst ||
        h.nT != b->nT || h.N != b->kp.N || h.R != b->kp.R || h.G != b->kp.G)
        return fail(b->ctx, ICM_ERR_ARG, "checkpoint of a batch with another shape");
    if (h.seed != b->seed) return fail(b->ctx, ICM_ERR_ARG, "checkpoint of a batch with another seed");
    if (h.has_slots) {
        icm_status st;
        if ((st = ensure_slot_arrays(b))) return st;
    }
    const unsigned char *in = (const unsigned char *)buf + sizeof h;
    std::vector<double> T(h.nT);
    std::memcpy(T.data(), in, h.nT * sizeof(double));
    in += h.nT * sizeof(double);
    const std::vector<BlobPart> parts = blob_parts(b);
    size_t need = sizeof h + h.nT * sizeof(double);
    for (const auto &pt : parts) need += pt.bytes;
    if (len < need) return fail(b->ctx, ICM_ERR_ARG, "checkpoint truncated");
    icm_status st;
    if (T != b->T || h.T_icm != b->T_icm)
        if ((st = icm_set_temperatures(b, T.data(), h.nT, h.T_icm))) return st;
    for (const auto &pt : parts) {
        ICM_CUDA(b->ctx, cudaMemcpyAsync(pt.dev, in, pt.bytes, cudaMemcpyHostToDevice, b->ctx->stream));
        in += pt.bytes;
    }
    icm::KParams &P = b->kp;
    ICM_CUDA(b->ctx, icm::launch_expand_couplings(b->raw_coup, b->gauss, b->edge_bond, b->n_inst, P.N, P.Z, P.Nb,
                                                  const_cast<float *>(P.Jd), const_cast<uint8_t *>(P.Jb),
                                                  b->ctx->stream));
    if ((st = refresh_dilution(b, 0, b->n_inst))) return st;
    if (h.has_slots) {
        ICM_CUDA(b->ctx, cudaMemcpy(b->h_active.data(), b->d_active, b->n_inst, cudaMemcpyDeviceToHost));
        ICM_CUDA(b->ctx, cudaMemcpy(b->h_tmeas.data(), b->d_tmeas, b->n_inst * 8, cudaMemcpyDeviceToHost));
    }
    b->sched = h.sched;
    return ICM_OK;
}

icm_status icm_batch_info(const icm_batch *b, int32_t *threads, int32_t *ctas_per_sm, int32_t *grid,
                          int32_t *smem_bytes, int64_t *launches)
{
    if (!b) return ICM_ERR_ARG;
    if (threads) *threads = b->threads;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    if (grid) *grid = b->grid;
    if (smem_bytes) *smem_bytes = b->cluster_k ? b->cl.total : b->kp.sm.total;
    if (launches) *launches = b->launches;
    return ICM_OK;
}

}  // extern "C"
