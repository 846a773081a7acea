// pt_icm.cu -- GB300 kernels for parallel tempering with isoenergetic
// cluster moves (the paper's "Isoenergetic cluster algorithm", steps 1, 2a,
// 2b, 3, plus the observables of "Benchmark model and observables").
//
// Design (one CTA per disorder instance, whole instance resident in shared
// memory for all sweeps of a launch; nothing here is a dense contraction, so
// no tensor cores are used).  Instances too large for one CTA's shared memory
// run the same code in a global-resident layout with wider CTAs (up to 1024
// threads): their spins and couplings are updated in place in global memory
// (L1/L2-resident), the small per-instance tables stay in shared memory.
//
//  * Spins are multispin-coded across replicas: the word of site position p
//    holds one bit per replica position r = 2k + c (bit set = spin -1), two
//    32-bit words per site when 2 N_T > 32.  Sites are stored colour-major
//    (colour 0 first), in ascending site index within a colour, so that a
//    checkerboard half-sweep walks contiguous words.
//  * Step 1 (Metropolis, checkerboard): a thread updates all replica bits of
//    one site word.  +-J: the number of unsatisfied bonds of all 32 replicas
//    is counted bit-sliced, then each bit draws its Philox word and compares
//    it with an integer threshold.  Gaussian: the local field of every bit is
//    summed in fp32 from sign-injected couplings, accept via ex2.
//    The energies of all replicas fall out of the colour-1 half-sweep
//    (every bond touches exactly one colour-1 site).
//  * Steps 2a/2b: overlap masks of all ICM pairs by a warp bit transpose; one thread
//    per pair counts, decides the copy-1 reversal and picks the seed by rank;
//    the clusters of all pairs grow at once, bit-parallel (bit 2k of a site's
//    cluster word = member of pair k's cluster), until a round adds nothing;
//    both copies flip by XOR, E_a is recomputed and E_b = (E_a+E_b) - E_a.
//  * Step 3: the draws of all swaps are turned into the form of their test in
//    parallel; one warp runs both copies' sequential passes (a half-warp
//    each) as chains of loads and compares; accepted swaps are then applied
//    to every site word as bit transpositions.
//  * Observables: vertical (bit-sliced) counters of q_i = -1 sites and of
//    bonds with q_i q_j = -1 for every pair at once.
#include "icm_internal.h"
#include "icm_device.cuh"

#include <cstdio>
#include <type_traits>

// The file is compiled three times so that the fused-kernel variants build in
// parallel: ICM_PART 0 = layout kernels and host entry points (the default),
// 1 = fused kernels for +-J couplings, 2 = fused kernels for Gaussian couplings
// (fused_pmj.cu and fused_gauss.cu define the macro and include this file).
#ifndef ICM_PART
#define ICM_PART 0
#endif

namespace icm {
cudaError_t launch_fused_pmj(const KParams &P, int threads, int grid, uint32_t n_sweeps, cudaStream_t st);
cudaError_t launch_fused_gauss(const KParams &P, int threads, int grid, uint32_t n_sweeps, cudaStream_t st);
cudaError_t launch_team_pmj(const TeamParams &TP, int Z, int grid, int smem, uint32_t n_sweeps, cudaStream_t st);
cudaError_t launch_team_gauss(const TeamParams &TP, int Z, int grid, int smem, uint32_t n_sweeps, cudaStream_t st);
cudaError_t team_occupancy_pmj(int Z, int smem, int *ctas);
cudaError_t team_occupancy_gauss(int Z, int smem, int *ctas);
cudaError_t fused_occupancy_pmj(int Z, bool wide, int threads, int smem, int *ctas);
cudaError_t fused_occupancy_gauss(int Z, bool wide, int threads, int smem, int *ctas);
int debug_phase_cycles_pmj(unsigned long long *out, int reset);
int debug_phase_cycles_gauss(unsigned long long *out, int reset);
int debug_check_pmj(unsigned int *out, int reset);
int debug_check_gauss(unsigned int *out, int reset);
}  // namespace icm

// Optional per-phase cycle counters (compile with -DICM_PHASE_TIMERS): thread 0
// of every CTA adds the clock64() cycles between phase marks to a global
// table, read back by icm_debug_phase_cycles().  Off by default; no work is
// skipped either way.
#ifdef ICM_PHASE_TIMERS
static __device__ unsigned long long g_icm_phase_cycles[16];   // one table per compiled part
#define PHASE_INIT() long long ph_last_ = clock64(); long long ph_acc_[8] = {0, 0, 0, 0, 0, 0, 0, 0}
#define PHASE_MARK(i) do { if (threadIdx.x == 0) { const long long n_ = clock64(); ph_acc_[i] += n_ - ph_last_; ph_last_ = n_; } } while (0)
#define PHASE_FLUSH() do { if (threadIdx.x == 0) for (int i_ = 0; i_ < 7; ++i_) atomicAdd(&g_icm_phase_cycles[i_], (unsigned long long)ph_acc_[i_]); } while (0)
#define ICM_SUB_INIT() long long icm_t0_ = clock64()
#define ICM_SUB(i) do { if (threadIdx.x == 0) { const long long n_ = clock64(); atomicAdd(&g_icm_phase_cycles[i], (unsigned long long)(n_ - icm_t0_)); icm_t0_ = n_; } } while (0)
#else
#define ICM_SUB_INIT() do { } while (0)
#define ICM_SUB(i) do { } while (0)
#define PHASE_INIT() do { } while (0)
#define PHASE_MARK(i) do { } while (0)
#define PHASE_FLUSH() do { } while (0)
#endif

namespace icm {

namespace {

struct Sm {
    uint32_t *s;
    uint16_t *nbr;
    uint8_t *zdeg;
    float *Jd;
    uint8_t *Jb;
    void *E;
    void *Epart;
    uint32_t *thr;
    float *b2l;
    uint32_t *mask;
    uint32_t *C;
    uint32_t *swap_x;
    int *swap_list;
    int *swap_n;
    uint64_t *swap_mask;
    float *sw_dbl;       // [32] (beta_k - beta_{k+1}) log2(e)
    int *sw_off, *sw_len;  // [32] +-J swap threshold table of pair k
    uint32_t *flipw;
    int *icm_seed;
    void *icm_esum_raw;
    int *cnt_n;
    int *cnt_d;
    double *accE;
    long long *acc64;
    long long *nmeas;
    unsigned long long *icmst;
    int tie;         // this instance is diluted: a zero-energy proposal is accepted with probability 1/2
    int nb;          // bonds present in this instance
};

__device__ __forceinline__ Sm make_sm(unsigned char *base, const SmemLayout &L)
{
    Sm S;
    S.s = (uint32_t *)(base + L.spins);
    S.nbr = (uint16_t *)(base + L.nbr);
    S.zdeg = (uint8_t *)(base + L.zdeg);
    S.Jd = (float *)(base + L.coup);
    S.Jb = (uint8_t *)(base + L.coup);
    S.E = base + L.E;
    S.Epart = base + L.Epart;
    S.thr = (uint32_t *)(base + L.rtab);
    S.b2l = (float *)(base + L.rtab);
    S.mask = (uint32_t *)(base + L.icm_mask);
    S.C = (uint32_t *)(base + L.icm_C);
    S.swap_x = (uint32_t *)(base + L.swap_x);
    S.swap_list = (int *)(base + L.swap_list);
    S.swap_n = (int *)(base + L.swap_n);
    S.swap_mask = (uint64_t *)(base + L.swap_mask);
    S.sw_dbl = (float *)(base + L.swap_tab);
    S.sw_off = (int *)(base + L.swap_tab + 128);
    S.sw_len = (int *)(base + L.swap_tab + 256);
    S.flipw = (uint32_t *)(base + L.flipw);
    S.icm_seed = (int *)(base + L.icm_seed);
    S.icm_esum_raw = base + L.icm_esum;
    S.cnt_n = (int *)(base + L.cnt_n);
    S.cnt_d = (int *)(base + L.cnt_d);
    S.accE = (double *)(base + L.accE);
    S.acc64 = (long long *)(base + L.acc64);
    S.nmeas = (long long *)(base + L.nmeas);
    S.icmst = (unsigned long long *)(base + L.icmst);
    return S;
}

// A 32-bit word of shared memory by its shared-window address.  Volatile: the
// cluster growth reads words that other threads rewrite during the same round.
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}

// The threads that run one instance: the whole CTA (the fused kernels), or
// one of several teams of a persistent CTA that runs instances of several
// sizes side by side (the shared group kernel).  A team is whole warps; its
// barrier is the CTA barrier (bar 0), a named barrier of its own (bar 1..15)
// or, for a one-warp team, a warp barrier (bar -1).
struct Team {
    int tid;   // thread index in the team
    int nth;   // threads of the team, a multiple of 32
    int bar;
};

__device__ __forceinline__ void team_sync(const Team &T)
{
    if (T.bar == 0) __syncthreads();
    else if (T.bar < 0) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(T.bar), "r"(T.nth) : "memory");
}

// Barrier of the team that returns whether pred was set in any of its threads.
__device__ __forceinline__ int team_sync_or(const Team &T, int pred)
{
    if (T.bar == 0) return __syncthreads_or(pred);
    if (T.bar < 0) {
        __syncwarp();
        return __any_sync(kFull, pred);
    }
    int r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
                 "selp.s32 %0, 1, 0, q;\n\t}"
                 : "=r"(r) : "r"(pred), "r"(T.bar), "r"(T.nth) : "memory");
    return r;
}

// Neighbour positions of position p (padding entries repeat p), read as
// 32-bit pairs from the [N][Z] uint16 table (Z even, so rows are 4-byte aligned).
template <int Z>
__device__ __forceinline__ void load_nbrs(const uint16_t *nbr, int p, int (&q)[Z])
{
    const uint32_t *w = (const uint32_t *)(nbr + p * Z);
#pragma unroll
    for (int i = 0; i < Z / 2; ++i) {
        const uint32_t v = w[i];
        q[2 * i] = (int)(v & 0xffffu);
        q[2 * i + 1] = (int)(v >> 16);
    }
}

// ---------------------------------------------------------------------------
// Step 1: one pass of a checkerboard half-sweep (colour COLOR) over the 16
// replica bits [32 g + 16 H, 32 g + 16 H + 16) of every site word of that
// colour.  Bits at or above R ("ghost" replicas of a partly used last word)
// are updated at beta = 0 and never read, so the inner loop has no guards.
// Two Philox4x32-10 blocks are generated together (8 draws) so that their
// dependency chains interleave.  The sites are taken by threads j0, j0 +
// jstride, ...; when other threads run another pass over the same words at
// the same time (tiny instances), the flips go in by atomic XOR (each pass
// owns its 16 bits, so the result does not depend on the order).
template <bool GAUSS, int Z, bool WIDE, bool DIL, bool SHARED>
__device__ __forceinline__ void sweep_pass(const KParams &P, const uint32_t (&key)[20], const Sm &S, const Team &T,
                                           uint32_t t, uint32_t inst, int g, int COLOR, int H, int j0, int jstride)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31, warp = T.tid >> 5;
    const int N = P.N, half = P.half;
    [[maybe_unused]] const int nth = T.nth;   // the bound of a checked index
    const int rbase = 32 * g + 16 * H;
    const int sh0 = 16 * H;                       // first bit of this pass inside the word
    const int npairs8 = (P.R - rbase + 7) >> 3;   // 8-bit groups holding at least one live replica (1 or 2)
    uint32_t *sg = S.s + g * N;
    ET acc[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) acc[b] = ET(0);
    for (int j = j0; j < half; j += jstride) {
        const int p = COLOR * half + j;
        const uint32_t sw0 = sg[p];
        const uint32_t sw = sw0 >> sh0;                 // this pass's bits at 0..15: constant shifts below
        const uint32_t site = __ldg(P.pos2site + p);
        uint32_t flip = 0;                              // bits 0..15 of this pass
        if constexpr (GAUSS) {
            // h = sum_d J_d s_d = Jsum - 2 sum_{d: s_d = -1} J_d: one bit test and one
            // predicated add per neighbour and bit
            float J2[Z];
            uint32_t nw[Z];
            int q[Z];
            load_nbrs<Z>(S.nbr, p, q);
            float Jsum = 0.f;
#pragma unroll
            for (int d = 0; d < Z; ++d) {
                nw[d] = sg[ICM_IDX(q[d], N, 1)] >> sh0;
                const float J = S.Jd[ICM_IDX(p * Z + d, N * Z, 2)];
                Jsum += J;
                J2[d] = 2.f * J;
            }
            const float *b2l = S.b2l + rbase;
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
                if (qq < npairs8) {
                    uint32_t x[4], y[4];
                    philox10x2(site, t, (uint32_t)(rbase >> 2) + 2 * qq, inst, key, x, y);
                    uint32_t f8 = 0u;                           // this group's accepted bits
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int b = 8 * qq + i;               // compile-time bit of the pass
                        float h = Jsum;
#pragma unroll
                        for (int d = 0; d < Z; ++d)
                            if ((nw[d] >> b) & 1u) h -= J2[d];
                        // sh = s_i h_i, Delta E = 2 sh; accept iff x < 2^32 exp(-2 beta sh),
                        // compared as rz(x) < 2^(32 + b2l sh) in fp32 (b2l = -2 beta log2 e):
                        // for sh <= 0 the right side is >= 2^32 > rz(x), so Delta E <= 0 is
                        // always accepted
                        const float sh = ((sw >> b) & 1u) ? -h : h;
                        const uint32_t xr = i < 4 ? x[i] : y[i - 4];
                        const float lim = ex2_approx(fmaf(b2l[b], sh, 32.f));
                        bool a;
                        if constexpr (DIL) {
                            // diluted instance: Delta E = 0 (a site without bonds) is
                            // accepted with probability 1/2
                            a = (sh < 0.f) || (sh == 0.f ? (!S.tie || xr < 0x80000000u) : (__uint2float_rz(xr) < lim));
                        } else {
                            a = __uint2float_rz(xr) < lim;
                        }
                        f8 |= (uint32_t)a << i;
                        acc[b] -= sh;                           // e = -s'h: -sh, or +sh after a flip
                        if (a) acc[b] += 2.f * sh;
                    }
                    flip |= f8 << (8 * qq);
                }
            }
        } else {
            uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;   // bit-planes of u = # unsatisfied bonds
            const uint32_t jb = S.Jb[ICM_IDX(p, N, 3)];
            int q[Z];
            load_nbrs<Z>(S.nbr, p, q);
            uint32_t u[Z];
#pragma unroll
            for (int d = 0; d < Z; ++d) u[d] = sw0 ^ sg[ICM_IDX(q[d], N, 1)] ^ (0u - ((jb >> d) & 1u));
            csa_count<Z>(u, c0, c1, c2, c3);
            c0 >>= sh0;
            c1 >>= sh0;
            c2 >>= sh0;
            c3 >>= sh0;
            const int z = (!DIL && P.const_z) ? P.const_z : (int)S.zdeg[ICM_IDX(p, N, 3)];   // degree = bonds present
            // m = z - 2u <= 0  <=>  u >= ceil(z/2): always accepted; on a diluted
            // instance only m < 0 (u >= floor(z/2) + 1), m = 0 takes the 1/2 entry
            if constexpr (DIL) {
                flip = ge_bitsliced(c0, c1, c2, c3, S.tie ? (z >> 1) + 1 : (z + 1) >> 1) & 0xFFFFu;
            } else if constexpr (Z > 7) {
                flip = (c3 | c2) & 0xFFFFu;         // z = 8: u >= 4
            } else {
                flip = ((z <= 4) ? (c2 | c1) : (c2 | (c1 & c0))) & 0xFFFFu;
            }
            constexpr int TS = thr_stride(Z);
            const uint32_t *thr = S.thr + rbase * TS;
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
                if (qq < npairs8) {
                    uint32_t x[4], y[4];
                    philox10x2(site, t, (uint32_t)(rbase >> 2) + 2 * qq, inst, key, x, y);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int b = 8 * qq + i;
                        const int u = (int)(((c0 >> b) & 1u) | (((c1 >> b) & 1u) << 1) | (((c2 >> b) & 1u) << 2) |
                                            (((c3 >> b) & 1u) << 3));
                        const int m = z - 2 * u;
                        const uint32_t xr = i < 4 ? x[i] : y[i - 4];
                        const uint32_t th = thr[b * TS + ICM_IDX(m > 0 ? m : 0, TS, 4)];
                        flip |= (uint32_t)(xr < th) << b;
                        acc[b] += ((flip >> b) & 1u) ? m : -m;
                    }
                }
            }
        }
        if constexpr (SHARED) atomicXor(sg + p, flip << sh0);
        else sg[p] = sw0 ^ (flip << sh0);
    }
    if (COLOR == 1) {   // energies: every bond touches exactly one colour-1 site
        const ET v = transpose_reduce16(acc, lane);
        const int r = rbase + (lane >> 1);
        if (!(lane & 1) && r < P.R) ((ET *)S.Epart)[ICM_IDX(warp * P.R + r, (nth >> 5) * (P.R > 32 ? P.R : 32), 5)] = v;
    }
}

// Tiny instances with at least twice the threads a colour needs: the
// threads split into groups of whole warps that run different passes at the
// same time; every warp writes its energy slots, the ones of passes it did not
// run as 0.
template <bool GAUSS, int Z, bool WIDE, bool DIL>
__device__ __forceinline__ void metropolis_sweep_concurrent(const KParams &P, const uint32_t (&key)[20], const Sm &S,
                                                         const Team &T, uint32_t t, uint32_t inst, int npass, int gthr,
                                                         int conc)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int group = T.tid / gthr;
    const int nslot = (T.nth >> 5) * P.R;
    for (int i = T.tid; i < nslot; i += T.nth) ((ET *)S.Epart)[i] = ET(0);
    team_sync(T);
    for (int color = 0; color < 2; ++color) {
        for (int p0 = 0; p0 < npass; p0 += conc) {
            const int pass = p0 + group;
            if (group < conc && pass < npass)    // whole warps: gthr is a multiple of 32
                sweep_pass<GAUSS, Z, WIDE, DIL, true>(P, key, S, T, t, inst, pass >> 1, color, pass & 1,
                                                      T.tid - group * gthr, gthr);
        }
        team_sync(T);
    }
}

// Step 1 for all replicas: colour 0 then colour 1, each as 16-bit passes over
// the site words.  One call site, so the pass body exists once in the kernel
// (the instruction cache is shared by all CTAs of the SM).
template <bool GAUSS, int Z, bool WIDE, bool DIL>
__device__ __forceinline__ void metropolis_sweep(const KParams &P, const uint32_t (&key)[20], const Sm &S, const Team &T,
                                                 uint32_t t, uint32_t inst)
{
    const int npass = (P.R + 15) >> 4;          // 16-bit passes per colour
    const int gthr = (P.half + 31) & ~31;        // threads of one pass
    const int conc = min(T.nth / gthr, npass);   // passes at a time
    if (conc >= 2) {
        metropolis_sweep_concurrent<GAUSS, Z, WIDE, DIL>(P, key, S, T, t, inst, npass, gthr, conc);
        return;
    }
    for (int it = 0; it < 2 * npass; ++it) {
        const int color = it >= npass;
        const int pass = it - color * npass;
        sweep_pass<GAUSS, Z, WIDE, DIL, false>(P, key, S, T, t, inst, pass >> 1, color, pass & 1, T.tid, T.nth);
        if (pass == npass - 1) team_sync(T);
    }
}

// ---------------------------------------------------------------------------
// Energies of copy cb (bit 2k + cb; cb = 0: copy a) of the pairs flagged in
// act0/act1 (bit 2k), from the spins: +-J via bit-sliced unsatisfied-bond
// counts (E = 2U - N_b), Gaussian via per-bit fp32 local fields; summed in a
// fixed order.  Every thread ends with partial sums in S.Epart[warp][k]; the
// caller adds warps.
template <bool GAUSS, int Z, bool WIDE>
__device__ __forceinline__ void pair_energies(const KParams &P, const Sm &S, const Team &T, uint32_t act0, uint32_t act1,
                                              int cb)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31, warp = T.tid >> 5;
    const int N = P.N, half = P.half, nth = T.nth;
    ET *part = (ET *)S.Epart;
    for (int g = 0; g < P.G; ++g) {
        const uint32_t act = g ? act1 : act0;
        if (!act) continue;                      // uniform
        const uint32_t *sg = S.s + g * N;
        ET acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = ET(0);
        for (int i = T.tid; i < half; i += nth) {
            const int p = half + i;              // colour-1 sites: every bond once
            const uint32_t sw = sg[p] >> cb;
            int q[Z];
            load_nbrs<Z>(S.nbr, p, q);
            if constexpr (GAUSS) {
                float J2[Z];
                uint32_t nw[Z];
                float Jsum = 0.f;
#pragma unroll
                for (int d = 0; d < Z; ++d) {
                    nw[d] = sg[ICM_IDX(q[d], N, 6)] >> cb;
                    const float J = S.Jd[ICM_IDX(p * Z + d, N * Z, 2)];
                    Jsum += J;
                    J2[d] = 2.f * J;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (!((act >> (2 * j)) & 1u)) continue;   // uniform
                    const int b = 2 * j;
                    float h = Jsum;                            // h = sum_d J_d s_d
#pragma unroll
                    for (int d = 0; d < Z; ++d)
                        if ((nw[d] >> b) & 1u) h -= J2[d];
                    acc[j] += ((sw >> b) & 1u) ? h : -h;       // e = -s_p h_p
                }
            } else {
                uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
                const uint32_t jb = S.Jb[ICM_IDX(p, N, 3)];
                uint32_t u[Z];
#pragma unroll
                for (int d = 0; d < Z; ++d) u[d] = sw ^ (sg[ICM_IDX(q[d], N, 6)] >> cb) ^ (0u - ((jb >> d) & 1u));
                csa_count<Z>(u, c0, c1, c2, c3);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int b = 2 * j;
                    acc[j] += (int)(((c0 >> b) & 1u) | (((c1 >> b) & 1u) << 1) | (((c2 >> b) & 1u) << 2) |
                                    (((c3 >> b) & 1u) << 3));
                }
            }
        }
        const ET v = transpose_reduce16(acc, lane);
        if (!(lane & 1)) part[ICM_IDX(warp * 32 + 16 * g + (lane >> 1), (nth >> 5) * 32, 7)] = v;
    }
}

// ---------------------------------------------------------------------------
// Steps 2a and 2b at every ICM temperature k < n_icm.
//  (a) overlap masks of all pairs by a warp bit-matrix transpose (bit 2k of s ^ (s >> 1));
//  (b) one thread per pair: n, the step-2a decision, the seed by rank;
//  (c) copy-1 reversal of the flagged pairs, then the clusters of all pairs
//      at once: C_p (bit 2k = site p in pair k's cluster, bit 2k + 1 the same
//      for pair 16 + k) grows by
//      C_p |= domain_p & OR(C of the neighbours) in rounds until a round
//      changes nothing -- the fixed point is each seed's connected component
//      of {q = -1};
//  (d) flip in both copies (bits 2k, 2k + 1 of the spin word of the pair), then E_a from
//      the spins and E_b = (E_a + E_b)_before - E_a (the move is isoenergetic).
//      A traced sweep also recomputes E_b from the spins and records
//      E_a + E_b of the two recomputed energies, so that the trace tests the
//      conservation of E_a + E_b instead of restating it.
template <bool GAUSS, int Z, bool WIDE>
__device__ void cluster_moves(const KParams &P, const uint32_t (&key)[20], const Sm &S, const Team &T, uint32_t t,
                              uint32_t inst, int slot, bool trace)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31, warp = T.tid >> 5, nwarps = T.nth >> 5;
    const int tid = T.tid, nth = T.nth;
    const int N = P.N, NW = P.NW, nicm = P.n_icm, G = P.G;
    ET *E = (ET *)S.E;
    ET *esum = (ET *)S.icm_esum_raw;
    ICM_SUB_INIT();

    // (a) masks; clear the cluster words
    for (int m = warp; m < NW; m += nwarps) {
        const int p = 32 * m + lane;
        uint32_t x = 0u;       // bit 2j: q of pair j (first word); bit 2j + 1: q of pair 16 + j
        if (p < N) {
            const uint32_t w0 = S.s[p];
            x = (w0 ^ (w0 >> 1)) & 0x55555555u;
            if (G > 1) {
                const uint32_t w1 = S.s[N + p];
                x |= ((w1 ^ (w1 >> 1)) & 0x55555555u) << 1;
            }
        }
        const uint32_t col = warp_transpose32(x, lane);   // lane l: bit l of the 32 sites' x
        const int k = (lane >> 1) + 16 * (lane & 1);
        if (k < nicm) S.mask[ICM_IDX(k * NW + m, nicm * NW, 8)] = col;
    }
    for (int i = tid; i < N; i += nth) S.C[i] = 0u;
    if (tid < 2) S.flipw[tid] = 0u;
    team_sync(T);

    // (b) per pair: n, step 2a, seed (planted into C)
    for (int k = tid; k < nicm; k += nth) {
        uint32_t *Mk = S.mask + k * NW;
        int n = 0;
        for (int m = 0; m < NW; ++m) n += __popc(Mk[m]);
        const int n_pre = n;
        int flipped = 0;
        if (P.enable_2a && 2 * n > N) {
            for (int m = 0; m < NW; ++m) {
                const int rem = N - 32 * m;
                Mk[m] = ~Mk[m] & (rem >= 32 ? kFull : ((1u << rem) - 1u));
            }
            n = N - n;
            flipped = 1;
            atomicOr(&S.flipw[(2 * k + 1) >> 5], 1u << ((2 * k + 1) & 31));
        }
        int seed = -1;
        if (n > 0) {
            uint32_t x[4];
            philox10k((uint32_t)k, t, 0u, (1u << 24) | inst, key, x);
            uint32_t rank = (uint32_t)(((uint64_t)x[0] * (uint32_t)n) >> 32);
            for (int m = 0; m < NW; ++m) {
                const uint32_t w = Mk[m];
                const uint32_t c = (uint32_t)__popc(w);
                if (rank < c) {
                    seed = 32 * m + nth_set_bit(w, rank);
                    break;
                }
                rank -= c;
            }
            atomicOr(&S.C[ICM_IDX(seed, N, 9)], 1u << (2 * (k & 15) + (k >> 4)));
        }
        S.icm_seed[k] = seed;
        esum[k] = E[2 * k] + E[2 * k + 1];
        if (trace) {
            const size_t o = (size_t)slot * P.nT + k;
            P.tr_n_pre[o] = n_pre;
            P.tr_flip2a[o] = flipped;
            P.tr_seed[o] = seed >= 0 ? (int)__ldg(P.pos2site + seed) : -1;
            P.tr_csize[o] = 0;
            P.tr_eb[o] = (float)(E[2 * k] + E[2 * k + 1]);
            P.tr_ea[o] = (float)(E[2 * k] + E[2 * k + 1]);
        }
    }
    team_sync(T);
    ICM_SUB(8);

    // (c) which pairs move, then copy-1 reversal and cluster growth.  One
    // cluster word per site holds every pair: bit 2j = pair j, bit 2j + 1 =
    // pair 16 + j (the bit of pair j's copy a in the first spin word, and the
    // one below pair 16 + j's copy a in the second), so that the domain word
    // is q of the first word | q of the second word << 1.
    uint32_t act0 = 0u, act1 = 0u;
    for (int k = 0; k < nicm; ++k)
        if (S.icm_seed[k] >= 0) {
            if (k < 16) act0 |= 1u << (2 * k);
            else act1 |= 1u << (2 * (k - 16));
        }
    const uint32_t actc = act0 | (act1 << 1);
    const uint32_t f0 = S.flipw[0], f1 = S.flipw[1];
    uint32_t *C = S.C;
    int rounds = 0;
    if (N <= 4 * nth) {
        // each thread owns sites tid + j nth (j < 4) and keeps, across rounds,
        // their neighbour positions, their domain words (the q = -1 bits of
        // the moving pairs, fixed during the growth) and their own cluster
        // words (written only by this thread) in registers
        // shared-memory layout: the neighbours' cluster words by their
        // shared-window addresses (one load each); wide layout: by position
        uint32_t qa[4][WIDE ? Z / 2 : Z];
        uint32_t dm[4], cw[4];
        uint32_t todo = 0u;                    // bit j: site j not yet absorbed
        [[maybe_unused]] const uint32_t cbase = WIDE ? 0u : (uint32_t)__cvta_generic_to_shared(C);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = tid + j * nth;
            const bool ok = p < N;
            const uint32_t *row = (const uint32_t *)(S.nbr + (ok ? p : 0) * Z);
#pragma unroll
            for (int i = 0; i < Z / 2; ++i) {
                const uint32_t v = row[i];
                if constexpr (WIDE) {
                    qa[j][i] = v;
                } else {
                    qa[j][2 * i] = cbase + 4u * ICM_IDX(v & 0xffffu, N, 10);
                    qa[j][2 * i + 1] = cbase + 4u * ICM_IDX(v >> 16, N, 10);
                }
            }
            dm[j] = cw[j] = 0u;
            if (ok) {
                const uint32_t w0 = S.s[p] ^ f0;             // step 2a
                S.s[p] = w0;
                uint32_t w1 = 0u;
                if (G > 1) {
                    w1 = S.s[N + p] ^ f1;
                    S.s[N + p] = w1;
                }
                dm[j] = (((w0 ^ (w0 >> 1)) & 0x55555555u) | (((w1 ^ (w1 >> 1)) & 0x55555555u) << 1)) & actc;
                cw[j] = C[p];
                if (dm[j] != cw[j]) todo |= 1u << j;
            }
        }
        if (actc) {
            int grew;
            do {
                grew = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (!((todo >> j) & 1u)) continue;
                    uint32_t nb = 0u;
                    if constexpr (WIDE) {
#pragma unroll
                        for (int i = 0; i < Z / 2; ++i)
                            nb |= C[ICM_IDX(qa[j][i] & 0xffffu, N, 10)] | C[ICM_IDX(qa[j][i] >> 16, N, 10)];
                    } else {
#pragma unroll
                        for (int i = 0; i < Z; ++i) nb |= lds_u32(qa[j][i]);
                    }
                    const uint32_t nw = cw[j] | (dm[j] & nb);
                    if (nw != cw[j]) {
                        C[tid + j * nth] = nw;
                        cw[j] = nw;
                        grew = 1;
                        if (nw == dm[j]) todo &= ~(1u << j);
                    }
                }
                ++rounds;
            } while (team_sync_or(T, grew));
            // (d) flip the owned sites in both copies of every moving pair
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = tid + j * nth;
                if (p < N && cw[j]) {
                    const uint32_t e0 = cw[j] & 0x55555555u, e1 = (cw[j] >> 1) & 0x55555555u;
                    S.s[p] ^= e0 | (e0 << 1);
                    if (G > 1) S.s[N + p] ^= e1 | (e1 << 1);
                }
            }
        }
    } else {
        for (int p = tid; p < N; p += nth) {
            S.s[p] ^= f0;
            if (G > 1) S.s[N + p] ^= f1;
        }
        team_sync(T);
        if (actc) {
            int grew;
            do {
                grew = 0;
                for (int p = tid; p < N; p += nth) {
                    const uint32_t w0 = S.s[p], w1 = G > 1 ? S.s[N + p] : 0u;
                    const uint32_t d = (((w0 ^ (w0 >> 1)) & 0x55555555u) | (((w1 ^ (w1 >> 1)) & 0x55555555u) << 1)) & actc;
                    const uint32_t c = C[p];
                    if (d == c) continue;
                    int q[Z];
                    load_nbrs<Z>(S.nbr, p, q);
                    uint32_t nb = 0u;
#pragma unroll
                    for (int dd = 0; dd < Z; ++dd) nb |= C[ICM_IDX(q[dd], N, 10)];
                    const uint32_t nw = c | (d & nb);
                    if (nw != c) {
                        C[p] = nw;
                        grew = 1;
                    }
                }
                ++rounds;
            } while (team_sync_or(T, grew));
            for (int p = tid; p < N; p += nth) {
                const uint32_t c = C[p];
                if (c) {
                    const uint32_t e0 = c & 0x55555555u, e1 = (c >> 1) & 0x55555555u;
                    S.s[p] ^= e0 | (e0 << 1);
                    if (G > 1) S.s[N + p] ^= e1 | (e1 << 1);
                }
            }
        }
    }
#ifdef ICM_PHASE_TIMERS
    if (tid == 0) atomicAdd(&g_icm_phase_cycles[11], (unsigned long long)rounds);
#endif
    if (tid == 0) {
        S.icmst[0] += (unsigned)__popc(actc);
        S.icmst[1] += (unsigned)rounds;
    }
    ICM_SUB(9);
    if (!actc) {
        team_sync(T);
        return;
    }
    if (trace) {
        // cluster sizes: counted once per cluster site; the cluster words as
        // [N][2] words, bit 2(k & 15) of word k >> 4 = site in pair k's cluster
        for (int p = tid; p < N; p += nth) {
            const uint32_t c = S.C[p];
            for (uint32_t b = c; b; b &= b - 1u) {
                const int bit = __ffs(b) - 1;
                atomicAdd(&S.cnt_d[(bit >> 1) + 16 * (bit & 1)], 1);
            }
            if (P.tr_cmask) {
                P.tr_cmask[(size_t)slot * 2 * N + 2 * p] = c & 0x55555555u;
                P.tr_cmask[(size_t)slot * 2 * N + 2 * p + 1] = (c >> 1) & 0x55555555u;
            }
        }
    }
    team_sync(T);
    pair_energies<GAUSS, Z, WIDE>(P, S, T, act0, act1, 0);
    team_sync(T);
    for (int k = tid; k < nicm; k += nth) {
        if (S.icm_seed[k] < 0) continue;
        ET ea = ET(0);
        for (int w = 0; w < nwarps; ++w) ea += ((const ET *)S.Epart)[w * 32 + k];
        if constexpr (!GAUSS) ea = 2 * ea - S.nb;            // E = 2 U - N_b (bonds present)
        E[2 * k] = ea;
        E[2 * k + 1] = esum[k] - ea;
        if (trace) P.tr_csize[(size_t)slot * P.nT + k] = S.cnt_d[k];
    }
    team_sync(T);
    if (trace) {
        // E_b of the moved pairs on its own, from the flipped spins
        pair_energies<GAUSS, Z, WIDE>(P, S, T, act0, act1, 1);
        team_sync(T);
        for (int k = tid; k < nicm; k += nth) {
            if (S.icm_seed[k] < 0) continue;
            ET eb = ET(0);
            for (int w = 0; w < nwarps; ++w) eb += ((const ET *)S.Epart)[w * 32 + k];
            if constexpr (!GAUSS) eb = 2 * eb - S.nb;
            P.tr_ea[(size_t)slot * P.nT + k] = (float)(E[2 * k] + eb);
        }
        for (int k = tid; k < 32; k += nth) S.cnt_d[k] = 0;
        team_sync(T);
    }
    ICM_SUB(10);
}

// ---------------------------------------------------------------------------
// Step 3: the PT pass of each copy (see pt_warp), then the configuration swaps.
template <bool GAUSS, bool WIDE>
__device__ void pt_pass(const KParams &P, const uint32_t (&key)[20], const Sm &S, const Team &T, uint32_t t,
                        uint32_t inst, int slot, bool trace)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int nT = P.nT, np = nT - 1, N = P.N;
    // draws of all (copy, pair) in parallel, in the form of their test
    for (int i = T.tid; i < 2 * np; i += T.nth) {
        const int c = i / np, k = i % np;
        uint32_t x[4];
        philox10k((uint32_t)k, t, (uint32_t)c, (2u << 24) | inst, key, x);
        if constexpr (GAUSS) S.swap_x[c * 32 + k] = pt_word_gauss(x[0]);
        else S.swap_x[c * 32 + k] = pt_word_pmj(x[0], P.thr_swap + S.sw_off[k], S.sw_len[k], P.dbeta_l2e[k]);
    }
    team_sync(T);
    // warp 0 runs both copies (a half-warp each).  Accepted swaps (k,k+1), ...,
    // (m,m+1) in a row form a run: the configuration at k bubbles up to m+1
    // and those at k+1..m+1 move down one slot; the words are permuted below
    // from the runs and the mask of bits that move down.
    if (T.tid < 32)
        pt_warp<GAUSS, ET>((ET *)S.E, P.R, np, S.swap_x, S.sw_dbl, S.swap_list, S.swap_n, S.swap_mask,
                           trace ? P.tr_swap + (size_t)slot * 2 * np : nullptr);
    team_sync(T);
    const int n0 = S.swap_n[0], n1 = S.swap_n[1];
    if (n0 + n1 > 0) {
        const SwapMasks m = swap_masks(S.swap_list, n0, n1, S.swap_mask);
        const bool two = P.G > 1;
        for (int p = T.tid; p < N; p += T.nth) {
            const uint64_t x = (uint64_t)S.s[p] | (two ? (uint64_t)S.s[N + p] << 32 : 0ull);
            const uint64_t y = swap_apply(m, x);
            S.s[p] = (uint32_t)y;
            if (two) S.s[N + p] = (uint32_t)(y >> 32);
        }
    }
    team_sync(T);
}

// ---------------------------------------------------------------------------
// Observables: per pair k, n = #{q_i = -1} and d = #{bonds, q_i q_j = -1}.
template <bool GAUSS, int Z, int NPL, bool WIDE>
__device__ void measure(const KParams &P, const Sm &S, const Team &T, int slot)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31;
    const int N = P.N, half = P.half, nT = P.nT;
    for (int g = 0; g < P.G; ++g) {
        const int npair = min(16, nT - 16 * g);
        const uint32_t *sg = S.s + g * N;
        uint32_t pl[NPL];   // even bit 2k: q = -1 sites of pair k; odd bit 2k+1: its q_i q_j = -1 bonds
#pragma unroll
        for (int i = 0; i < NPL; ++i) pl[i] = 0u;
        for (int p = T.tid; p < N; p += T.nth) {
            const uint32_t w = sg[p];
            vadd(pl, (w ^ (w >> 1)) & 0x55555555u);
        }
        for (int p = half + T.tid; p < N; p += T.nth) {
            const uint32_t w = sg[p];
            const uint32_t qp = (w ^ (w >> 1)) & 0x55555555u;
            int qn[Z];
            load_nbrs<Z>(S.nbr, p, qn);
            uint32_t x[Z];                 // an absent bond points at p itself: x = 0
#pragma unroll
            for (int d = 0; d < Z; ++d) {
                const uint32_t wq = sg[ICM_IDX(qn[d], N, 13)];
                x[d] = (qp ^ ((wq ^ (wq >> 1)) & 0x55555555u)) << 1;
            }
            uint32_t c0, c1, c2, c3;
            csa_count<Z>(x, c0, c1, c2, c3);
            vadd4(pl, c0, c1, c2, c3);
        }
        const int v = warp_vsum(pl, lane);   // lane 2k: n of pair k, lane 2k+1: d of pair k
        if (lane < 2 * npair) atomicAdd(((lane & 1) ? S.cnt_d : S.cnt_n) + 16 * g + (lane >> 1), v);
    }
    team_sync(T);
    for (int k = T.tid; k < nT; k += T.nth) {
        const long long n = S.cnt_n[k], d = S.cnt_d[k];
        S.cnt_n[k] = 0;
        S.cnt_d[k] = 0;
        const ET *E = (const ET *)S.E;
        S.accE[k] += (double)E[2 * k] + (double)E[2 * k + 1];
        S.acc64[0 * nT + k] += n;
        S.acc64[1 * nT + k] += (N - 2 * n) * (N - 2 * n);
        S.acc64[2 * nT + k] += n < N - n ? n : N - n;
        S.acc64[3 * nT + k] += d;
        atomicAdd(&P.hist[((size_t)slot * nT + k) * (N + 1) + ICM_IDX(n, N + 1, 14)], 1ull);
    }
    if (T.tid == 0) S.nmeas[0] += 1;
    team_sync(T);
}

// ---------------------------------------------------------------------------
// The per-batch tables of a team's shared memory: the neighbour table (the
// shared-memory layout of an undiluted batch), degrees, temperature and swap
// tables, cleared counters.
template <bool GAUSS, int Z, bool WIDE, bool DIL>
__device__ __forceinline__ void load_tables(const KParams &P, Sm &S, const Team &T)
{
    const int tid = T.tid, nth = T.nth;
    const int N = P.N, R = P.R, nT = P.nT, G = P.G;
    if constexpr (!WIDE && !DIL) {
        for (int i = tid; i < N * Z; i += nth) S.nbr[i] = P.nbr[i];
        if (!GAUSS && !P.const_z)
            for (int i = tid; i < N; i += nth) S.zdeg[i] = P.zdeg[i];
    }
    S.tie = 0;
    S.nb = P.Nb;
    for (int k = tid; k < nT - 1; k += nth) {
        if constexpr (GAUSS) {
            S.sw_dbl[k] = P.dbeta_l2e[k];
        } else {
            S.sw_off[k] = P.swap_off[k];
            S.sw_len[k] = P.swap_len[k];
        }
    }
    if constexpr (GAUSS) {
        for (int r = tid; r < 32 * G; r += nth) S.b2l[r] = r < R ? P.b2l[r] : 0.f;
    } else {
        constexpr int TS = thr_stride(Z);
        for (int i = tid; i < 32 * G * TS; i += nth) S.thr[i] = i < R * TS ? P.thr_metro[i] : 0u;
    }
    if (tid < 32) {
        S.cnt_n[tid] = 0;
        S.cnt_d[tid] = 0;
    }
}

// n_sweeps simulation steps of the instance in slot `slot`, run by team T:
// load its state into the team's shared memory (the spins and couplings stay
// in global memory in the wide layout), run the steps, store the state back.
template <bool GAUSS, int Z, bool WIDE, bool DIL>
__device__ __forceinline__ void run_instance(const KParams &P, const uint32_t (&key)[20], Sm &S, const Team &T,
                                             int slot, uint32_t n_sweeps)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    PHASE_INIT();
    const int tid = T.tid, nth = T.nth, nwarps = nth >> 5;
    const int N = P.N, R = P.R, nT = P.nT, G = P.G;
    if constexpr (DIL) {
        const uint16_t *nb_src = P.nbr_inst + (size_t)slot * N * Z;
        const uint8_t *zd_src = P.zdeg_inst + (size_t)slot * N;
        if constexpr (WIDE) {
            S.nbr = const_cast<uint16_t *>(nb_src);
            S.zdeg = const_cast<uint8_t *>(zd_src);
        } else {
            const uint32_t *src = (const uint32_t *)nb_src;     // N Z even: whole 32-bit pairs
            uint32_t *dst = (uint32_t *)S.nbr;
            for (int i = tid; i < (N * Z) / 2; i += nth) dst[i] = src[i];
            for (int i = tid; i < N; i += nth) S.zdeg[i] = zd_src[i];
        }
        S.nb = P.nb_inst[slot];
        S.tie = S.nb < P.Nb;
    }
    if constexpr (WIDE) {
        S.s = P.spins + (size_t)slot * G * N;
        S.Jd = const_cast<float *>(P.Jd) + (size_t)slot * N * Z;
        S.Jb = const_cast<uint8_t *>(P.Jb) + (size_t)slot * N;
    } else {
        const uint32_t *gs = P.spins + (size_t)slot * G * N;
        for (int i = tid; i < G * N; i += nth) S.s[i] = gs[i];
        if constexpr (GAUSS) {
            const float4 *src = (const float4 *)(P.Jd + (size_t)slot * N * Z);
            float4 *dst = (float4 *)S.Jd;
            for (int i = tid; i < (N * Z) / 4; i += nth) dst[i] = src[i];
        } else {
            for (int i = tid; i < N; i += nth) S.Jb[i] = P.Jb[(size_t)slot * N + i];
        }
    }
    if constexpr (GAUSS) {
        for (int r = tid; r < R; r += nth) ((float *)S.E)[r] = P.Ef[(size_t)slot * R + r];
    } else {
        for (int r = tid; r < R; r += nth) ((int *)S.E)[r] = P.Ei[(size_t)slot * R + r];
    }
    for (int k = tid; k < nT; k += nth) {
        S.accE[k] = P.accE[(size_t)slot * nT + k];
        for (int a = 0; a < 4; ++a) S.acc64[a * nT + k] = P.acc64[((size_t)a * P.n_inst + slot) * nT + k];
    }
    if (tid == 0) {
        S.nmeas[0] = P.n_meas[slot];
        S.icmst[0] = S.icmst[1] = 0ull;
    }
    const uint32_t inst = P.inst_id[slot];
    const long long t_meas = P.t_meas_inst ? P.t_meas_inst[slot] : P.t_meas;
    uint32_t t = P.tsweep[slot];
    team_sync(T);

    PHASE_MARK(5);
    for (uint32_t step = 0; step < n_sweeps; ++step, ++t) {
        const bool trace = P.trace && step + 1 == n_sweeps;
        if (trace) {
            for (int k = tid; k < nT; k += nth) {
                const size_t o = (size_t)slot * nT + k;
                P.tr_n_pre[o] = -1;
                P.tr_flip2a[o] = 0;
                P.tr_seed[o] = -1;
                P.tr_csize[o] = 0;
                P.tr_eb[o] = 0.f;
                P.tr_ea[o] = 0.f;
            }
            for (int i = tid; i < 2 * (nT - 1); i += nth) P.tr_swap[(size_t)slot * 2 * (nT - 1) + i] = 0;
            if (P.tr_cmask)
                for (int i = tid; i < 2 * N; i += nth) P.tr_cmask[(size_t)slot * 2 * N + i] = 0u;
            team_sync(T);
        }
        if (P.enable_metropolis) {  // step 1
            metropolis_sweep<GAUSS, Z, WIDE, DIL>(P, key, S, T, t, inst);
            for (int r = tid; r < R; r += nth) {
                ET e = ET(0);
                for (int w = 0; w < nwarps; ++w) e += ((const ET *)S.Epart)[w * R + r];
                ((ET *)S.E)[r] = e;
            }
            team_sync(T);
        }
        PHASE_MARK(0);
        if (P.icm_every > 0 && t % (uint32_t)P.icm_every == 0 && P.n_icm > 0)  // steps 2a, 2b
            cluster_moves<GAUSS, Z, WIDE>(P, key, S, T, t, inst, slot, trace);
        PHASE_MARK(1);
        if (P.swap_every > 0 && t % (uint32_t)P.swap_every == 0 && nT > 1)  // step 3
            pt_pass<GAUSS, WIDE>(P, key, S, T, t, inst, slot, trace);
        PHASE_MARK(2);
        if ((long long)t >= t_meas) {
            if (P.small_counts) measure<GAUSS, Z, 4, WIDE>(P, S, T, slot);   // every per-thread count < 16
            else measure<GAUSS, Z, kPlanes, WIDE>(P, S, T, slot);
        }
        PHASE_MARK(3);
    }

    PHASE_MARK(4);
    if constexpr (!WIDE) {
        uint32_t *gd = P.spins + (size_t)slot * G * N;
        for (int i = tid; i < G * N; i += nth) gd[i] = S.s[i];
    }
    for (int r = tid; r < R; r += nth) {
        if constexpr (GAUSS) P.Ef[(size_t)slot * R + r] = ((float *)S.E)[r];
        else P.Ei[(size_t)slot * R + r] = ((int *)S.E)[r];
    }
    for (int k = tid; k < nT; k += nth) {
        P.accE[(size_t)slot * nT + k] = S.accE[k];
        for (int a = 0; a < 4; ++a) P.acc64[((size_t)a * P.n_inst + slot) * nT + k] = S.acc64[a * nT + k];
    }
    if (tid == 0) {
        P.n_meas[slot] = S.nmeas[0];
        P.tsweep[slot] = t;
        if (P.icm_stats) {
            P.icm_stats[2 * (size_t)slot] += S.icmst[0];
            P.icm_stats[2 * (size_t)slot + 1] += S.icmst[1];
        }
    }
    team_sync(T);
    PHASE_MARK(5);
    PHASE_FLUSH();
}

// The fused step loop.  WIDE = false: the whole instance lives in shared
// memory for the launch.  WIDE = true (instances too large for one CTA's
// shared memory): spins and couplings are updated in place in global memory,
// the neighbour table is read from global memory, and the cluster words and
// overlap masks use a per-CTA global scratch; the arithmetic is the same.
// DIL = true (some instance of the batch has absent bonds): the neighbour
// table and degrees are per instance (absent bonds point at the site itself,
// like padding) and a diluted instance takes the probability-1/2 rule for
// zero-energy proposals.  One CTA runs the instances blockIdx.x,
// blockIdx.x + gridDim.x, ... in turn.
template <bool GAUSS, int Z, bool WIDE, bool DIL>
__device__ __forceinline__ void fused_body(const KParams &P, uint32_t n_sweeps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Sm S = make_sm(smem, P.sm);
    const Team T{(int)threadIdx.x, (int)blockDim.x, 0};
    if constexpr (WIDE) {
        S.nbr = const_cast<uint16_t *>(P.nbr);
        S.zdeg = const_cast<uint8_t *>(P.zdeg);
        S.C = P.scratch + (size_t)blockIdx.x * P.scratch_words;
        S.mask = S.C + 2 * P.N;
    }
    load_tables<GAUSS, Z, WIDE, DIL>(P, S, T);
    for (int slot = blockIdx.x; slot < P.n_inst; slot += gridDim.x) {
        if (P.active && !P.active[slot]) continue;   // free slot of a serving batch
        run_instance<GAUSS, Z, WIDE, DIL>(P, P.key, S, T, slot, n_sweeps);
    }
}

template <bool GAUSS, int Z, bool DIL>
__global__ void __launch_bounds__(kMaxThreads, 7) fused_kernel(const KParams P, uint32_t n_sweeps)
{
    fused_body<GAUSS, Z, false, DIL>(P, n_sweeps);
}

template <bool GAUSS, int Z, bool DIL>
__global__ void __launch_bounds__(kMaxThreadsWide, 1) fused_wide_kernel(const KParams P, uint32_t n_sweeps)
{
    fused_body<GAUSS, Z, true, DIL>(P, n_sweeps);
}

// The shared group kernel (see TeamParams): each persistent CTA takes the
// next work item (a global counter) whenever it is free, so the tiles, in
// descending order of work, balance over the CTAs; a tile's teams run their
// instances side by side, and the CTA barrier after each item frees the
// shared memory for the next.  The last CTA to finish resets the counters
// for the next launch (launches on one stream run in order).  Which CTA runs
// an instance does not change its result: same arithmetic and random keys as
// the fused kernel, so a +-J instance follows the same chain in either.
template <bool GAUSS, int Z>
__global__ void __launch_bounds__(kTeamThreads, 1) team_kernel(const __grid_constant__ TeamParams TP, uint32_t n_sweeps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int next_item;
    for (;;) {
        if (threadIdx.x == 0) next_item = atomicAdd(&TP.counters[0], 1);
        __syncthreads();
        const int it = next_item;
        if (it >= TP.n_items) break;           // the same value in every thread
        const TeamItem w = TP.items[it];
        const KParams &P = TP.cls[w.cls];
        const int tw = TP.team_threads[w.cls];
        const int team = (int)threadIdx.x / tw;
        if (team < w.count) {
            const int slot = w.slot0 + team;
            if (!P.active || P.active[slot]) {
                const Team T{(int)threadIdx.x - team * tw, tw, tw == 32 ? -1 : team + 1};
                Sm S = make_sm(smem + (size_t)team * P.sm.total, P.sm);
                load_tables<GAUSS, Z, false, false>(P, S, T);
                run_instance<GAUSS, Z, false, false>(P, TP.key, S, T, slot, n_sweeps);
            }
        }
        __syncthreads();                       // also: every thread has read next_item
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&TP.counters[1], 1) == (int)gridDim.x - 1) {   // every CTA has taken its last item
            TP.counters[0] = 0;
            TP.counters[1] = 0;
        }
    }
}

#if ICM_PART == 0
// ---------------------------------------------------------------------------
// Layout kernels (run at load/read time, not per sweep).
__global__ void pack_spins_kernel(const int8_t *__restrict__ src, uint32_t *__restrict__ dst,
                                  const uint16_t *__restrict__ pos2site, int n_inst, int R, int G, int N)
{
    const size_t total = (size_t)n_inst * G * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx % N);
        const int g = (int)((idx / N) % G);
        const size_t inst = idx / ((size_t)N * G);
        const int site = pos2site[p];
        uint32_t w = 0;
        for (int b = 0; b < 32 && 32 * g + b < R; ++b)
            w |= (uint32_t)(src[(inst * R + 32 * g + b) * N + site] < 0) << b;
        dst[idx] = w;
    }
}

__global__ void unpack_spins_kernel(const uint32_t *__restrict__ src, int8_t *__restrict__ dst,
                                    const uint16_t *__restrict__ pos2site, int n_inst, int R, int G, int N)
{
    const size_t total = (size_t)n_inst * R * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx % N);
        const int r = (int)((idx / N) % R);
        const size_t inst = idx / ((size_t)N * R);
        const uint32_t w = src[(inst * G + (r >> 5)) * N + p];
        dst[(inst * R + r) * N + pos2site[p]] = ((w >> (r & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
    }
}

__global__ void expand_couplings_kernel(const void *__restrict__ bondJ, int gauss, const int32_t *__restrict__ edge_bond,
                                        int n_inst, int N, int Z, int Nb, float *__restrict__ Jd,
                                        uint8_t *__restrict__ Jb)
{
    const size_t total = (size_t)n_inst * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx % N);
        const size_t inst = idx / N;
        if (gauss) {
            const float *J = (const float *)bondJ + inst * Nb;
            for (int d = 0; d < Z; ++d) {
                const int b = edge_bond[p * Z + d];
                Jd[idx * Z + d] = b >= 0 ? J[b] : 0.f;
            }
        } else {
            const int8_t *J = (const int8_t *)bondJ + inst * Nb;
            uint32_t bits = 0;
            for (int d = 0; d < Z; ++d) {
                const int b = edge_bond[p * Z + d];
                if (b >= 0 && J[b] < 0) bits |= 1u << d;
            }
            Jb[idx] = (uint8_t)bits;
        }
    }
}

// Per-instance tables of a diluted batch (see launch_expand_dilution).  A
// bond is absent when its coupling is exactly 0; each bond present is counted
// once, at the endpoint with the smaller position.  Invalid couplings (not
// finite, or +-J values other than -1, 0, +1) are counted per instance into bad.
__global__ void expand_dilution_kernel(const void *__restrict__ bondJ, int gauss, const int32_t *__restrict__ edge_bond,
                                       const uint16_t *__restrict__ nbr, int n_inst, int N, int Z, int Nb,
                                       uint16_t *__restrict__ nbr_inst, uint8_t *__restrict__ zdeg_inst,
                                       int32_t *__restrict__ nb_inst, int32_t *__restrict__ bad)
{
    const size_t total = (size_t)n_inst * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int p = (int)(idx % N);
        const size_t inst = idx / N;
        int deg = 0, once = 0, invalid = 0;
        for (int d = 0; d < Z; ++d) {
            const int b = edge_bond[p * Z + d];
            bool present = false;
            if (b >= 0) {
                if (gauss) {
                    const float J = ((const float *)bondJ)[inst * Nb + b];
                    present = J != 0.f;
                    invalid += !isfinite(J);
                } else {
                    const int J = ((const int8_t *)bondJ)[inst * Nb + b];
                    present = J != 0;
                    invalid += J < -1 || J > 1;
                }
            }
            const int q = nbr[p * Z + d];
            nbr_inst[idx * Z + d] = (uint16_t)(present ? q : p);
            deg += present;
            once += present && p < q;
        }
        zdeg_inst[idx] = (uint8_t)deg;
        if (once) atomicAdd(&nb_inst[inst], once);
        if (invalid) atomicAdd(&bad[inst], invalid);
    }
}

// Energies of every replica from the spins: E = -sum over colour-1 sites of
// s_i h_i (every bond joins the two colours).  One CTA per instance.
template <bool GAUSS, int Z>
__global__ void init_energies_kernel(const KParams P)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    __shared__ ET red[kMaxThreads];
    const int N = P.N, half = P.half;
    for (int slot = blockIdx.x; slot < P.n_inst; slot += gridDim.x) {
        const uint32_t *s = P.spins + (size_t)slot * P.G * N;
        const uint16_t *nbr = P.diluted ? P.nbr_inst + (size_t)slot * N * Z : P.nbr;   // absent bonds: self
        for (int r = 0; r < P.R; ++r) {
            const uint32_t *sg = s + (r >> 5) * N;
            const int b = r & 31;
            ET acc = ET(0);
            for (int p = half + threadIdx.x; p < N; p += blockDim.x) {
                const int si = ((sg[p] >> b) & 1u) ? -1 : 1;
                for (int d = 0; d < Z; ++d) {
                    const int q = nbr[p * Z + d];
                    const int sj = ((sg[q] >> b) & 1u) ? -1 : 1;
                    if constexpr (GAUSS) {
                        acc -= P.Jd[((size_t)slot * N + p) * Z + d] * (float)(si * sj);
                    } else {
                        if (q == p) continue;
                        const int J = ((P.Jb[(size_t)slot * N + p] >> d) & 1u) ? -1 : 1;
                        acc -= J * si * sj;
                    }
                }
            }
            red[threadIdx.x] = acc;
            __syncthreads();
            for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
                if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                if constexpr (GAUSS) P.Ef[(size_t)slot * P.R + r] = red[0];
                else P.Ei[(size_t)slot * P.R + r] = red[0];
            }
            __syncthreads();
        }
    }
}

__global__ void energies_to_double_kernel(const float *Ef, const int32_t *Ei, int gauss, size_t n, double *out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = gauss ? (double)Ef[i] : (double)Ei[i];
}

#endif  // ICM_PART == 0

inline int grid_for(size_t n, int threads)
{
    size_t g = (n + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    return g > 0 ? (int)g : 1;
}

template <bool GAUSS, int Z, bool DIL>
cudaError_t launch_fused_t(const KParams &P, int threads, int grid, uint32_t n_sweeps, cudaStream_t st)
{
    if (P.wide && (threads > kMaxThreadsWide || !P.scratch)) return cudaErrorInvalidValue;
    if (!P.wide && threads > kMaxThreads) return cudaErrorInvalidValue;
    if (DIL && (!P.nbr_inst || !P.zdeg_inst || !P.nb_inst)) return cudaErrorInvalidValue;
    auto kern = P.wide ? fused_wide_kernel<GAUSS, Z, DIL> : fused_kernel<GAUSS, Z, DIL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, P.sm.total);
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, P.sm.total, st>>>(P, n_sweeps);
    return cudaGetLastError();
}

template <bool GAUSS, int Z>
cudaError_t occupancy_t(bool wide, int threads, int smem, int *ctas)
{
    // the diluted variants have the same register budget (launch bounds) and layout
    auto kern = wide ? fused_wide_kernel<GAUSS, Z, false> : fused_kernel<GAUSS, Z, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, kern, threads, smem);
}

}  // namespace

#if ICM_PART == 0
// ---------------------------------------------------------------------------
static int align_up(int v, int a) { return (v + a - 1) / a * a; }

SmemLayout smem_layout(int N, int Z, int R, int G, int nT, int n_icm, int nwarps, bool gauss, bool wide)
{
    const int in_smem = wide ? 0 : 1;   // the large arrays stay in global memory in the wide layout
    SmemLayout L{};
    const int NW = (N + 31) / 32;
    int o = 0;
    auto take = [&](int bytes, int align) {
        o = align_up(o, align);
        const int at = o;
        o += bytes;
        return at;
    };
    L.coup = take(in_smem * (gauss ? N * Z * 4 : N), 16);
    L.spins = take(in_smem * G * N * 4, 16);
    L.nbr = take(in_smem * N * Z * 2, 16);
    L.zdeg = take(in_smem * N, 16);
    L.E = take(R * 4, 16);
    L.Epart = take(nwarps * (R > 32 ? R : 32) * 4, 16);
    L.rtab = take(gauss ? G * 32 * 4 : G * 32 * thr_stride(Z) * 4, 16);   // every bit of the G words
    L.icm_mask = take(in_smem * n_icm * NW * 4, 16);
    L.icm_C = take(in_smem * N * 4, 16);
    L.swap_x = take(2 * 32 * 4, 16);
    L.swap_list = take(2 * 32 * 4, 16);
    L.swap_n = take(2 * 4, 16);
    L.swap_mask = take(2 * 8, 16);
    L.swap_tab = take(3 * 32 * 4, 16);
    L.flipw = take(2 * 4, 16);
    L.icm_seed = take(32 * 4, 16);
    L.icm_esum = take(32 * 4, 16);
    L.cnt_n = take(32 * 4, 16);
    L.cnt_d = take(32 * 4, 16);
    L.accE = take(nT * 8, 16);
    L.acc64 = take(4 * nT * 8, 16);
    L.nmeas = take(8, 16);
    L.icmst = take(16, 16);
    L.total = align_up(o, 16);
    return L;
}

int fused_threads(int N)
{
    const int half = N / 2;
    int t = (half + 31) / 32 * 32;
    if (t > kMaxThreads) t = kMaxThreads;
    if (t < 32) t = 32;
    return t;
}

int fused_threads_wide(int N)
{
    const int half = N / 2;
    int t = (half + 31) / 32 * 32;
    if (t > kMaxThreadsWide) t = kMaxThreadsWide;
    if (t < 32) t = 32;
    return t;
}

int wide_scratch_words(int N)
{
    const int NW = (N + 31) / 32;
    return (2 * N + 32 * NW + 3) / 4 * 4;
}

cudaError_t fused_occupancy(bool gauss, int Z, bool wide, int threads, int smem, int *ctas)
{
    return gauss ? fused_occupancy_gauss(Z, wide, threads, smem, ctas) : fused_occupancy_pmj(Z, wide, threads, smem, ctas);
}

cudaError_t launch_fused(const KParams &P, bool gauss, int threads, int grid, uint32_t n_sweeps, cudaStream_t st)
{
    return gauss ? launch_fused_gauss(P, threads, grid, n_sweeps, st) : launch_fused_pmj(P, threads, grid, n_sweeps, st);
}

cudaError_t launch_team(const TeamParams &TP, bool gauss, int Z, int grid, int smem, uint32_t n_sweeps,
                        cudaStream_t st)
{
    return gauss ? launch_team_gauss(TP, Z, grid, smem, n_sweeps, st) : launch_team_pmj(TP, Z, grid, smem, n_sweeps, st);
}

cudaError_t team_occupancy(bool gauss, int Z, int smem, int *ctas)
{
    return gauss ? team_occupancy_gauss(Z, smem, ctas) : team_occupancy_pmj(Z, smem, ctas);
}

cudaError_t launch_pack_spins(const int8_t *src, uint32_t *dst, const uint16_t *pos2site, int n_inst, int R, int G,
                              int N, cudaStream_t st)
{
    pack_spins_kernel<<<grid_for((size_t)n_inst * G * N, 256), 256, 0, st>>>(src, dst, pos2site, n_inst, R, G, N);
    return cudaGetLastError();
}

cudaError_t launch_unpack_spins(const uint32_t *src, int8_t *dst, const uint16_t *pos2site, int n_inst, int R, int G,
                                int N, cudaStream_t st)
{
    unpack_spins_kernel<<<grid_for((size_t)n_inst * R * N, 256), 256, 0, st>>>(src, dst, pos2site, n_inst, R, G, N);
    return cudaGetLastError();
}

cudaError_t launch_expand_couplings(const void *bond_J, bool gauss, const int32_t *edge_bond, int n_inst, int N, int Z,
                                    int Nb, float *Jd, uint8_t *Jb, cudaStream_t st)
{
    expand_couplings_kernel<<<grid_for((size_t)n_inst * N, 256), 256, 0, st>>>(bond_J, gauss ? 1 : 0, edge_bond,
                                                                                n_inst, N, Z, Nb, Jd, Jb);
    return cudaGetLastError();
}

cudaError_t launch_expand_dilution(const void *bond_J, bool gauss, const int32_t *edge_bond, const uint16_t *nbr,
                                   int n_inst, int N, int Z, int Nb, uint16_t *nbr_inst, uint8_t *zdeg_inst,
                                   int32_t *nb_inst, int32_t *bad, cudaStream_t st)
{
    expand_dilution_kernel<<<grid_for((size_t)n_inst * N, 256), 256, 0, st>>>(bond_J, gauss ? 1 : 0, edge_bond, nbr,
                                                                               n_inst, N, Z, Nb, nbr_inst,
                                                                               zdeg_inst, nb_inst, bad);
    return cudaGetLastError();
}

cudaError_t launch_init_energies(const KParams &P, bool gauss, cudaStream_t st)
{
    const int grid = P.n_inst < 152 * 8 ? P.n_inst : 152 * 8;
    switch (P.Z) {
    case 4:
        if (gauss) init_energies_kernel<true, 4><<<grid, kMaxThreads, 0, st>>>(P);
        else init_energies_kernel<false, 4><<<grid, kMaxThreads, 0, st>>>(P);
        break;
    case 6:
        if (gauss) init_energies_kernel<true, 6><<<grid, kMaxThreads, 0, st>>>(P);
        else init_energies_kernel<false, 6><<<grid, kMaxThreads, 0, st>>>(P);
        break;
    case 8:
        if (gauss) init_energies_kernel<true, 8><<<grid, kMaxThreads, 0, st>>>(P);
        else init_energies_kernel<false, 8><<<grid, kMaxThreads, 0, st>>>(P);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_energies_to_double(const KParams &P, bool gauss, double *out, cudaStream_t st)
{
    const size_t n = (size_t)P.n_inst * P.R;
    energies_to_double_kernel<<<grid_for(n, 256), 256, 0, st>>>(P.Ef, P.Ei, gauss ? 1 : 0, n, out);
    return cudaGetLastError();
}

#else  // ICM_PART 1 or 2: the fused kernels of one disorder kind

namespace {
constexpr bool kPartGauss = ICM_PART == 2;

template <bool DIL>
cudaError_t launch_fused_z(const KParams &P, int threads, int grid, uint32_t n_sweeps, cudaStream_t st)
{
    switch (P.Z) {
    case 4: return launch_fused_t<kPartGauss, 4, DIL>(P, threads, grid, n_sweeps, st);
    case 6: return launch_fused_t<kPartGauss, 6, DIL>(P, threads, grid, n_sweeps, st);
    case 8: return launch_fused_t<kPartGauss, 8, DIL>(P, threads, grid, n_sweeps, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_part(const KParams &P, int threads, int grid, uint32_t n_sweeps, cudaStream_t st)
{
    return P.diluted ? launch_fused_z<true>(P, threads, grid, n_sweeps, st)
                     : launch_fused_z<false>(P, threads, grid, n_sweeps, st);
}

template <int Z>
cudaError_t launch_team_t(const TeamParams &TP, int grid, int smem, uint32_t n_sweeps, cudaStream_t st)
{
    auto kern = team_kernel<kPartGauss, Z>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kTeamThreads, smem, st>>>(TP, n_sweeps);
    return cudaGetLastError();
}

cudaError_t launch_team_part(const TeamParams &TP, int Z, int grid, int smem, uint32_t n_sweeps, cudaStream_t st)
{
    switch (Z) {
    case 4: return launch_team_t<4>(TP, grid, smem, n_sweeps, st);
    case 6: return launch_team_t<6>(TP, grid, smem, n_sweeps, st);
    case 8: return launch_team_t<8>(TP, grid, smem, n_sweeps, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int Z>
cudaError_t team_occupancy_t(int smem, int *ctas)
{
    auto kern = team_kernel<kPartGauss, Z>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, kern, kTeamThreads, smem);
}

cudaError_t team_occupancy_part(int Z, int smem, int *ctas)
{
    switch (Z) {
    case 4: return team_occupancy_t<4>(smem, ctas);
    case 6: return team_occupancy_t<6>(smem, ctas);
    case 8: return team_occupancy_t<8>(smem, ctas);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_part(int Z, bool wide, int threads, int smem, int *ctas)
{
    switch (Z) {
    case 4: return occupancy_t<kPartGauss, 4>(wide, threads, smem, ctas);
    case 6: return occupancy_t<kPartGauss, 6>(wide, threads, smem, ctas);
    case 8: return occupancy_t<kPartGauss, 8>(wide, threads, smem, ctas);
    default: return cudaErrorInvalidValue;
    }
}

int check_part(unsigned int *out, int reset)
{
#ifdef ICM_CHECKED
    if (cudaMemcpyFromSymbol(out, g_icm_check, sizeof(unsigned int) * 4) != cudaSuccess) return -4;
    if (reset) {
        unsigned int z[4] = {};
        if (cudaMemcpyToSymbol(g_icm_check, z, sizeof(z)) != cudaSuccess) return -4;
    }
    return 0;
#else
    (void)out;
    (void)reset;
    return -7;
#endif
}

int phase_cycles_part(unsigned long long *out, int reset)
{
#ifdef ICM_PHASE_TIMERS
    if (cudaMemcpyFromSymbol(out, g_icm_phase_cycles, sizeof(unsigned long long) * 16) != cudaSuccess) return -4;
    if (reset) {
        unsigned long long z[16] = {};
        if (cudaMemcpyToSymbol(g_icm_phase_cycles, z, sizeof(z)) != cudaSuccess) return -4;
    }
    return 0;
#else
    (void)out;
    (void)reset;
    return -7;
#endif
}
}  // namespace

#if ICM_PART == 1
cudaError_t launch_fused_pmj(const KParams &P, int threads, int grid, uint32_t n_sweeps, cudaStream_t st)
{
    return launch_part(P, threads, grid, n_sweeps, st);
}
cudaError_t fused_occupancy_pmj(int Z, bool wide, int threads, int smem, int *ctas)
{
    return occupancy_part(Z, wide, threads, smem, ctas);
}
cudaError_t launch_team_pmj(const TeamParams &TP, int Z, int grid, int smem, uint32_t n_sweeps, cudaStream_t st)
{
    return launch_team_part(TP, Z, grid, smem, n_sweeps, st);
}
cudaError_t team_occupancy_pmj(int Z, int smem, int *ctas) { return team_occupancy_part(Z, smem, ctas); }
int debug_phase_cycles_pmj(unsigned long long *out, int reset) { return phase_cycles_part(out, reset); }
int debug_check_pmj(unsigned int *out, int reset) { return check_part(out, reset); }
#else
cudaError_t launch_fused_gauss(const KParams &P, int threads, int grid, uint32_t n_sweeps, cudaStream_t st)
{
    return launch_part(P, threads, grid, n_sweeps, st);
}
cudaError_t fused_occupancy_gauss(int Z, bool wide, int threads, int smem, int *ctas)
{
    return occupancy_part(Z, wide, threads, smem, ctas);
}
cudaError_t launch_team_gauss(const TeamParams &TP, int Z, int grid, int smem, uint32_t n_sweeps, cudaStream_t st)
{
    return launch_team_part(TP, Z, grid, smem, n_sweeps, st);
}
cudaError_t team_occupancy_gauss(int Z, int smem, int *ctas) { return team_occupancy_part(Z, smem, ctas); }
int debug_phase_cycles_gauss(unsigned long long *out, int reset) { return phase_cycles_part(out, reset); }
int debug_check_gauss(unsigned int *out, int reset) { return check_part(out, reset); }
#endif

#endif  // ICM_PART
}  // namespace icm

#if ICM_PART == 0 && defined(ICM_CHECKED)
// Checked builds: out[0] = guarded indices found out of range in the fused
// kernels (both disorder kinds), out[1..3] = site code, index and bound of the
// first one of the ±J part, or of the Gaussian part when the ±J part has none.
extern "C" int icm_debug_check(unsigned int *out, int reset)
{
    unsigned int a[4], b[4];
    int rc = icm::debug_check_pmj(a, reset);
    if (!rc) rc = icm::debug_check_gauss(b, reset);
    if (rc) return rc;
    out[0] = a[0] + b[0];
    for (int i = 1; i < 4; ++i) out[i] = a[0] ? a[i] : b[i];
    return 0;
}
#endif

#if ICM_PART == 0 && defined(ICM_PHASE_TIMERS)
// Cycles per phase summed over CTAs and over both fused-kernel parts: 0 sweep +
// energies, 1 ICM, 2 PT, 3 observables, 4 between the last step and the
// store, 5 load/store and instance changes.
extern "C" int icm_debug_phase_cycles(unsigned long long *out, int reset)
{
    unsigned long long a[16], b[16];
    int rc = icm::debug_phase_cycles_pmj(a, reset);
    if (!rc) rc = icm::debug_phase_cycles_gauss(b, reset);
    if (rc) return rc;
    for (int i = 0; i < 16; ++i) out[i] = a[i] + b[i];
    return 0;
}
#endif
