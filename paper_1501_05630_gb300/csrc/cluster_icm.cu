// cluster_icm.cu -- the simulation step of pt_icm.cu for one instance spread
// over a thread-block cluster of K CTAs (K SMs), for instances whose single
// CTA would be slow (2D L=128, 3D L=16 and larger).
//
// CTA r of the cluster owns the positions [c half + r hs, c half + (r+1) hs)
// of each colour c and keeps their spin words, couplings, cluster words and
// neighbour table in its own shared memory.  A neighbour's word is read
// through the cluster's distributed shared memory: the neighbour table holds
// the 32-bit cluster-window address (mapa) of the neighbour's spin word in
// its owner CTA, read with ld.shared::cluster.  Phases are separated by
// cluster barriers (barrier.cluster arrive.release / wait.acquire):
//  * sweep: colour 0, barrier, colour 1; each CTA sums its sites' energies,
//    barrier, every CTA adds the K shares in rank order (the same E in all);
//  * ICM: per-CTA overlap counts, barrier, every CTA finds the seed's owner
//    from the K counts (position order = (colour, rank, local)), the owner
//    plants it, barrier; growth in rounds of a few in-place scans without
//    barriers, each round ending with a barrier after which every CTA reads
//    the round stamp that growing warps pushed into all CTAs; flip, barrier,
//    copy-a energies summed as above;
//  * PT: every CTA holds the same energies and draws the same numbers, so
//    all make the same decisions and permute their own words; barrier;
//  * observables: per-CTA counts, barrier, rank 0 accumulates.
// Every buffer another CTA reads is rewritten only after a barrier that
// both have passed since the read.  Random keys are those of the
// single-CTA kernels, so the chain is the same, bit for bit for +-J.
#include "icm_internal.h"
#include "icm_device.cuh"

#include <type_traits>

namespace icm {
namespace {

__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cl_id()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cl_count()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

// Every thread of every CTA of the cluster; orders shared-memory accesses
// across the cluster (release before, acquire after).
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Cluster-window address of the shared-memory byte `local` (a shared-window
// address of this CTA) in CTA `rank`.
__device__ __forceinline__ uint32_t cl_map(uint32_t local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

__device__ __forceinline__ uint32_t cl_ld(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}


// A word of this CTA's shared memory by its shared-window address.
__device__ __forceinline__ uint32_t sh_ld(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ void cl_st(uint32_t addr, uint32_t v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Relaxed cluster-scope accesses of the union-find labels, which other
// threads of the cluster change while they are read.
__device__ __forceinline__ uint32_t cl_ld_rlx(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.relaxed.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t cl_cas(uint32_t addr, uint32_t cmp, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.relaxed.cluster.shared::cluster.cas.b32 %0, [%1], %2, %3;"
                 : "=r"(old) : "r"(addr), "r"(cmp), "r"(v) : "memory");
    return old;
}

template <typename T>
__device__ __forceinline__ T cl_ldT(uint32_t addr)
{
    const uint32_t v = cl_ld(addr);
    if constexpr (std::is_same<T, float>::value) return __uint_as_float(v);
    else return (T)(int)v;
}

// This CTA's view: pointers into its shared memory and cluster addresses.
struct CS {
    uint32_t *s, *C, *nb;
    float *Jd;
    uint8_t *Jb, *zdeg;
    void *E, *Epart, *Esw, *Epair, *esum;
    uint32_t *thr;
    float *b2l;
    uint32_t *mask, *lab, *sadr, *sroot;
    uint16_t *gord;
    int *cntloc, *flags, *seed, *csz, *cnt_n, *cnt_d;
    uint32_t *flipw;
    uint32_t *swap_x;
    int *swap_list, *swap_n;
    uint64_t *swap_mask;
    double *accE;
    long long *acc64, *nmeas;
    unsigned long long *icmst;
    uint32_t base;        // shared-window address of this CTA's dynamic shared memory
    uint32_t dCs;         // a neighbour-table entry (the neighbour's cluster word) minus this: its spin word 0
    uint32_t rank, K;
    int hs, nls;
};

__device__ __forceinline__ CS make_cs(unsigned char *smem, const ClusterLayout &L)
{
    CS S;
    S.s = (uint32_t *)(smem + L.s);
    S.C = (uint32_t *)(smem + L.C);
    S.nb = (uint32_t *)(smem + L.nb);
    S.Jd = (float *)(smem + L.coup);
    S.Jb = (uint8_t *)(smem + L.coup);
    S.zdeg = (uint8_t *)(smem + L.zdeg);
    S.E = smem + L.E;
    S.Epart = smem + L.Epart;
    S.Esw = smem + L.Esw;
    S.Epair = smem + L.Epair;
    S.esum = smem + L.esum;
    S.thr = (uint32_t *)(smem + L.rtab);
    S.b2l = (float *)(smem + L.rtab);
    S.mask = (uint32_t *)(smem + L.mask);
    S.lab = (uint32_t *)(smem + L.lab);
    S.sadr = (uint32_t *)(smem + L.sadr);
    S.sroot = (uint32_t *)(smem + L.sroot);
    S.gord = L.gord >= 0 ? (uint16_t *)(smem + L.gord) : nullptr;
    S.cntloc = (int *)(smem + L.cntloc);
    S.flags = (int *)(smem + L.flags);
    S.seed = (int *)(smem + L.seed);
    S.csz = (int *)(smem + L.csz);
    S.cnt_n = (int *)(smem + L.cnt_n);
    S.cnt_d = (int *)(smem + L.cnt_d);
    S.flipw = (uint32_t *)(smem + L.flipw);
    S.swap_x = (uint32_t *)(smem + L.swap_x);
    S.swap_list = (int *)(smem + L.swap_list);
    S.swap_n = (int *)(smem + L.swap_n);
    S.swap_mask = (uint64_t *)(smem + L.swap_mask);
    S.accE = (double *)(smem + L.accE);
    S.acc64 = (long long *)(smem + L.acc64);
    S.nmeas = (long long *)(smem + L.nmeas);
    S.icmst = (unsigned long long *)(smem + L.icmst);
    S.base = (uint32_t)__cvta_generic_to_shared(smem);
    S.dCs = (uint32_t)(L.C - L.s);
    S.rank = cl_rank();
    S.K = (uint32_t)L.K;
    S.hs = L.hs;
    S.nls = L.nls;
    return S;
}

// The Z neighbour addresses of own site li, in 16-byte loads when Z is a
// multiple of 4 (a row starts 16-byte aligned), else 8-byte loads: one
// shared-memory instruction instead of four for a 2D site.
template <int Z>
__device__ __forceinline__ void nb_row(const uint32_t *nb, int li, uint32_t (&e)[Z])
{
    const uint32_t *row = nb + li * Z;
    if constexpr (Z % 4 == 0) {
#pragma unroll
        for (int d = 0; d < Z; d += 4) {
            const uint4 v = *reinterpret_cast<const uint4 *>(row + d);
            e[d] = v.x;
            e[d + 1] = v.y;
            e[d + 2] = v.z;
            e[d + 3] = v.w;
        }
    } else if constexpr (Z % 2 == 0) {
#pragma unroll
        for (int d = 0; d < Z; d += 2) {
            const uint2 v = *reinterpret_cast<const uint2 *>(row + d);
            e[d] = v.x;
            e[d + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int d = 0; d < Z; ++d) e[d] = row[d];
    }
}

// Sum over the cluster, in rank order, of the ET value at byte offset `off`
// of every CTA's shared memory (the same result in every CTA).
template <typename ET>
__device__ __forceinline__ ET cl_sum(const CS &S, int off)
{
    ET v = ET(0);
    for (uint32_t r = 0; r < S.K; ++r) v += cl_ldT<ET>(cl_map(S.base + off, r));
    return v;
}

// Global position of local site li of CTA `rank`.
__device__ __forceinline__ int pos_of(const KParams &P, const CS &S, int li)
{
    const int c = li >= S.hs;
    return c * P.half + (int)S.rank * S.hs + (li - c * S.hs);
}

// ---------------------------------------------------------------------------
// Step 1, one 16-bit pass of colour COLOR over word g (see sweep_pass in
// pt_icm.cu: the same arithmetic, with neighbour words read through the
// cluster window).
template <bool GAUSS, int Z, bool DIL>
__device__ __forceinline__ void cl_sweep_pass(const KParams &P, const CS &S, uint32_t t, uint32_t inst, int g,
                                              int COLOR, int H, bool tie)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nth = blockDim.x;
    const int rbase = 32 * g + 16 * H;
    const int sh0 = 16 * H;
    const int npairs8 = (P.R - rbase + 7) >> 3;
    const uint32_t goff = (uint32_t)(g * S.nls * 4) - S.dCs;   // neighbour entry -> its spin word g
    uint32_t *sg = S.s + g * S.nls;
    ET acc[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) acc[b] = ET(0);
    for (int j = threadIdx.x; j < S.hs; j += nth) {
        const int li = COLOR * S.hs + j;
        const uint32_t sw0 = sg[li];
        const uint32_t sw = sw0 >> sh0;
        const uint32_t site = __ldg(P.pos2site + pos_of(P, S, li));
        uint32_t nw[Z];
        nb_row<Z>(S.nb, li, nw);
#pragma unroll
        for (int d = 0; d < Z; ++d) nw[d] = cl_ld(nw[d] + goff);
        uint32_t flip = 0;
        if constexpr (GAUSS) {
            float J2[Z];
            float Jsum = 0.f;
#pragma unroll
            for (int d = 0; d < Z; ++d) {
                nw[d] >>= sh0;
                const float J = S.Jd[li * Z + d];
                Jsum += J;
                J2[d] = 2.f * J;
            }
            const float *b2l = S.b2l + rbase;
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
                if (qq < npairs8) {
                    uint32_t x[4], y[4];
                    philox10x2(site, t, (uint32_t)(rbase >> 2) + 2 * qq, inst, P.key, x, y);
                    uint32_t f8 = 0u;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int b = 8 * qq + i;
                        float h = Jsum;
#pragma unroll
                        for (int d = 0; d < Z; ++d)
                            if ((nw[d] >> b) & 1u) h -= J2[d];
                        const float sh = ((sw >> b) & 1u) ? -h : h;
                        const uint32_t xr = i < 4 ? x[i] : y[i - 4];
                        const uint32_t thr = __float2uint_rz(ex2_approx(fmaf(b2l[b], sh, 32.f)));
                        bool a;
                        if constexpr (DIL)   // diluted instance: Delta E = 0 accepted with probability 1/2
                            a = (sh < 0.f) || (sh == 0.f ? (!tie || xr < 0x80000000u) : (xr < thr));
                        else
                            a = (sh <= 0.f) || (xr < thr);
                        f8 |= (uint32_t)a << i;
                        acc[b] -= sh;
                        if (a) acc[b] += 2.f * sh;
                    }
                    flip |= f8 << (8 * qq);
                }
            }
        } else {
            uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;   // bit-planes of u = # unsatisfied bonds
            const uint32_t jb = S.Jb[li];
            uint32_t u[Z];
#pragma unroll
            for (int d = 0; d < Z; ++d) u[d] = sw0 ^ nw[d] ^ (0u - ((jb >> d) & 1u));
            csa_count<Z>(u, c0, c1, c2, c3);
            c0 >>= sh0;
            c1 >>= sh0;
            c2 >>= sh0;
            c3 >>= sh0;
            const int z = (!DIL && P.const_z) ? P.const_z : (int)S.zdeg[li];   // bonds present
            // always accepted: m = z - 2u <= 0; on a diluted instance only m < 0
            // (m = 0 takes the threshold entry 2^31, probability 1/2)
            if constexpr (DIL) flip = ge_bitsliced(c0, c1, c2, c3, tie ? (z >> 1) + 1 : (z + 1) >> 1) & 0xFFFFu;
            else if constexpr (Z > 7) flip = (c3 | c2) & 0xFFFFu;   // z = 8: u >= 4
            else flip = ((z <= 4) ? (c2 | c1) : (c2 | (c1 & c0))) & 0xFFFFu;
            constexpr int TS = thr_stride(Z);
            const uint32_t *thr = S.thr + rbase * TS;
#pragma unroll
            for (int qq = 0; qq < 2; ++qq) {
                if (qq < npairs8) {
                    uint32_t x[4], y[4];
                    philox10x2(site, t, (uint32_t)(rbase >> 2) + 2 * qq, inst, P.key, x, y);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int b = 8 * qq + i;
                        const int u = (int)(((c0 >> b) & 1u) | (((c1 >> b) & 1u) << 1) | (((c2 >> b) & 1u) << 2) |
                                            (((c3 >> b) & 1u) << 3));
                        const int m = z - 2 * u;
                        const uint32_t xr = i < 4 ? x[i] : y[i - 4];
                        const uint32_t th = thr[b * TS + (m > 0 ? m : 0)];
                        flip |= (uint32_t)(xr < th) << b;
                        acc[b] += ((flip >> b) & 1u) ? m : -m;
                    }
                }
            }
        }
        sg[li] = sw0 ^ (flip << sh0);
    }
    if (COLOR == 1) {
        const ET v = transpose_reduce16(acc, lane);
        const int r = rbase + (lane >> 1);
        if (!(lane & 1) && r < P.R) ((ET *)S.Epart)[warp * P.R + r] = v;
    }
}

// Step 1 for all replicas; then every CTA's share of the energies, summed
// over the cluster in rank order.
template <bool GAUSS, int Z, bool DIL>
__device__ __forceinline__ void cl_metropolis(const KParams &P, const ClusterLayout &L, const CS &S, uint32_t t,
                                              uint32_t inst, bool tie)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int npass = (P.R + 15) >> 4;
    const int nwarps = blockDim.x >> 5;
    for (int it = 0; it < 2 * npass; ++it) {
        const int color = it >= npass;
        const int pass = it - color * npass;
        cl_sweep_pass<GAUSS, Z, DIL>(P, S, t, inst, pass >> 1, color, pass & 1, tie);
        if (pass == npass - 1) {
            if (color == 0) cl_sync();            // colour 1 reads colour-0 words of other CTAs
            else __syncthreads();
        }
    }
    for (int r = threadIdx.x; r < P.R; r += blockDim.x) {
        ET e = ET(0);
        for (int w = 0; w < nwarps; ++w) e += ((const ET *)S.Epart)[w * P.R + r];
        ((ET *)S.Esw)[r] = e;
    }
    cl_sync();
    for (int r = threadIdx.x; r < P.R; r += blockDim.x) ((ET *)S.E)[r] = cl_sum<ET>(S, L.Esw + 4 * r);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Union-find over the cluster's shared memory.  A label word holds the
// cluster-window address of its parent's label word; a root holds its own
// address.  Roots are linked by a fixed random priority of their addresses
// (a bijective hash): a root is hooked, by compare-and-swap on the root, only
// under a root of higher priority, so priorities increase strictly along
// every path (no cycle forms, a walk ends within N steps) and the trees stay
// shallow, where linking by address would chain the sites of a row.  Words
// of this CTA are reached through its own shared window, which is faster
// than the cluster window.  In the phase where only this CTA's threads touch
// its words (LOCAL) the accesses are plain; otherwise they are relaxed at
// cluster scope, so that compare-and-swaps from every CTA are atomic with
// one another.
struct Uf {
    uint32_t lab;     // cluster-window address of this CTA's first label word
    uint32_t loc;     // its shared-window address
    uint32_t span;    // bytes of this CTA's label words in use
    int limit;        // N + 1
};

__device__ __forceinline__ uint32_t uf_prio(uint32_t x)
{
    x *= 0x9E3779B1u;
    x ^= x >> 15;
    x *= 0x85EBCA77u;
    return x ^ (x >> 13);
}

template <bool LOCAL>
__device__ __forceinline__ uint32_t uf_ld(const Uf &U, uint32_t a)
{
    const uint32_t o = a - U.lab;
    uint32_t v;
    if (LOCAL) v = sh_ld(U.loc + o);
    else if (o < U.span)
        asm volatile("ld.relaxed.cluster.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(U.loc + o) : "memory");
    else v = cl_ld_rlx(a);
    return v;
}

template <bool LOCAL>
__device__ __forceinline__ uint32_t uf_cas(const Uf &U, uint32_t a, uint32_t cmp, uint32_t v)
{
    const uint32_t o = a - U.lab;
    uint32_t old;
    if (LOCAL)
        asm volatile("atom.shared.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "r"(U.loc + o), "r"(cmp), "r"(v) : "memory");
    else if (o < U.span)
        asm volatile("atom.relaxed.cluster.shared::cta.cas.b32 %0, [%1], %2, %3;"
                     : "=r"(old) : "r"(U.loc + o), "r"(cmp), "r"(v) : "memory");
    else old = cl_cas(a, cmp, v);
    return old;
}

// The root of x (after the unions: nothing changes the labels any more).
__device__ __forceinline__ uint32_t uf_root(const Uf &U, uint32_t x)
{
    for (int i = 0; i < U.limit; ++i) {
        const uint32_t p = uf_ld<false>(U, x);
        if (p == x) return x;
        x = p;
    }
    (void)ICM_IDX(U.limit, U.limit, 23);
    return x;
}

// Union over the bonds of this CTA's colour-1 sites whose two ends have
// q = -1 in a group pair, each bond once: those inside this CTA (REMOTE
// false) or those to other CTAs (REMOTE true).  The lanes of a warp run in
// lockstep: each iteration, every lane with a union in hand reads the
// parents of both ends and climbs one level, or, at two distinct roots,
// hooks the lower-priority root under the other (a failed swap goes on from
// the root's new parent); a lane without one first takes its next bond.
// Every iteration ends in a warp vote, so the lanes' loads issue together
// (lanes that ran their own loops fell apart and waited for their loads one
// by one).  `it` is bounded (never reached: each union ends within N climbs
// and N failed swaps).
template <int Z, bool REMOTE>
__device__ __forceinline__ void uf_unions(const Uf &U, const CS &S, uint32_t gm0, uint32_t gm1, int n0, uint32_t mys,
                                          uint32_t dlab, uint32_t qstride)
{
    const int nls = S.nls, hs = S.hs, nth = blockDim.x;
    int j = (int)threadIdx.x - nth, li = 0, d = Z;
    uint32_t x0 = 0u, x1 = 0u, y0 = 0u, y1 = 0u, ea = 0u, eb = 0u, a = 0u, b = 0u;
    bool more = true, busy = false;
    // iterations a lane can need: its bonds x pairs x (N climbs + N failed swaps + 1)
    const long long cap = (long long)(hs / nth + 1) * Z * 32 * (2ll * U.limit + 1);
    for (long long it = 0;; ++it) {
        if (!busy && more) {
            while (!(y0 | y1)) {                     // the next bond with a pair to link
                if (d == Z) {
                    j += nth;
                    if (j >= hs) {
                        more = false;
                        break;
                    }
                    li = hs + j;
                    const uint32_t w0 = S.s[li];
                    x0 = (w0 ^ (w0 >> 1)) & gm0;
                    x1 = 0u;
                    if (gm1) {
                        const uint32_t w1 = S.s[nls + li];
                        x1 = (w1 ^ (w1 >> 1)) & gm1;
                    }
                    d = (x0 | x1) ? 0 : Z;
                    ea = U.lab + 4u * (uint32_t)li;
                    continue;
                }
                const uint32_t e = S.nb[li * Z + d] - S.dCs;   // the neighbour's spin word 0
                ++d;
                const uint32_t o = e - mys;
                if ((o >= qstride) != REMOTE) continue;
                if (x0) {
                    const uint32_t v = REMOTE ? cl_ld(e) : S.s[o >> 2];
                    y0 = x0 & (v ^ (v >> 1));
                }
                if (x1) {
                    const uint32_t v = REMOTE ? cl_ld(e + qstride) : S.s[nls + (o >> 2)];
                    y1 = x1 & (v ^ (v >> 1));
                }
                eb = e + dlab;
            }
            if (y0 | y1) {
                uint32_t q;
                if (y0) {
                    q = (uint32_t)__popc(gm0 & ((y0 & (0u - y0)) - 1u));
                    y0 &= y0 - 1u;
                } else {
                    q = (uint32_t)(n0 + __popc(gm1 & ((y1 & (0u - y1)) - 1u)));
                    y1 &= y1 - 1u;
                }
                a = ea + q * qstride;
                b = eb + q * qstride;
                busy = true;
            }
        }
        if (!__any_sync(kFull, busy)) break;
        if (it >= cap) {
            (void)ICM_IDX(U.limit, U.limit, 23);
            break;
        }
        if (busy) {
            const uint32_t pa = uf_ld<!REMOTE>(U, a), pb = uf_ld<!REMOTE>(U, b);
            if (pa != a || pb != b) {
                a = pa;
                b = pb;
            } else if (a == b) {
                busy = false;
            } else {
                if (uf_prio(a) < uf_prio(b)) {
                    const uint32_t x = a;
                    a = b;
                    b = x;
                }
                const uint32_t old = uf_cas<!REMOTE>(U, b, b, a);   // hook the lower-priority root under the other
                if (old == b) busy = false;
                else b = old;
            }
        }
    }
}

// The own sites in the seed's component of each group pair: their cluster
// bits are set.  Lockstep as above: each iteration a lane climbs one level
// from its site's label toward the root.
__device__ __forceinline__ void uf_mark(const Uf &U, const CS &S, uint32_t gm0, uint32_t gm1, int n0)
{
    const int nls = S.nls, nth = blockDim.x;
    int li = (int)threadIdx.x - nth, q = 0;
    uint32_t x0 = 0u, x1 = 0u, bit = 0u, c = 0u, c0 = 0u, c1 = 0u;
    bool word1 = false, more = true, busy = false;
    const long long cap = (long long)(nls / nth + 1) * 32 * (U.limit + 1);   // sites x pairs x (N climbs + 1)
    for (long long it = 0;; ++it) {
        if (!busy && more) {
            while (!(x0 | x1)) {
                if (li >= 0 && (c0 | c1)) {          // the last site's bits are complete
                    S.C[li] |= c0 | (c1 << 1);
                    c0 = c1 = 0u;
                }
                li += nth;
                if (li >= nls) {
                    more = false;
                    break;
                }
                const uint32_t w0 = S.s[li];
                x0 = (w0 ^ (w0 >> 1)) & gm0;
                if (gm1) {
                    const uint32_t w1 = S.s[nls + li];
                    x1 = (w1 ^ (w1 >> 1)) & gm1;
                }
            }
            if (x0 | x1) {
                word1 = !x0;
                uint32_t &x = word1 ? x1 : x0;
                bit = x & (0u - x);
                x &= x - 1u;
                q = word1 ? n0 + __popc(gm1 & (bit - 1u)) : __popc(gm0 & (bit - 1u));
                c = U.lab + 4u * (uint32_t)(q * nls + li);
                busy = true;
            }
        }
        if (!__any_sync(kFull, busy)) break;
        if (it >= cap) {
            (void)ICM_IDX(U.limit, U.limit, 23);
            break;
        }
        if (busy) {
            const uint32_t p = uf_ld<false>(U, c);
            if (p != c) {
                c = p;
            } else {
                if (c == S.sroot[q]) (word1 ? c1 : c0) |= bit;
                busy = false;
            }
        }
    }
    if (li < nls && (c0 | c1)) S.C[li] |= c0 | (c1 << 1);
}

// Step 2b(c) by union-find: the seed's component of q = -1 sites of every
// moving pair, set in the cluster words of the own sites (the seed's
// bit is already set).  Pairs go in groups of L.ufg (act0 / act1: pair j of
// word w at bit 2j of act_w).  Per group: labels reset (every site its own
// root); union over the bonds inside this CTA, where every walk stays in this
// CTA; cluster barrier; union over the bonds to other CTAs; cluster barrier;
// every own site compares its root with the seed's.  The components are those
// of the propagation in the other branch, so the cluster words are the same,
// bit for bit.
template <int Z>
__device__ __forceinline__ void cl_grow_uf(const KParams &P, const ClusterLayout &L, const CS &S, uint32_t act0,
                                           uint32_t act1)
{
    const int tid = threadIdx.x, nth = blockDim.x;
    const int nls = S.nls, g = L.ufg;
    Uf U;
    U.lab = cl_map(S.base + L.lab, S.rank);
    U.loc = S.base + (uint32_t)L.lab;
    U.limit = P.N + 1;
    const uint32_t mys = cl_map(S.base + L.s, S.rank);      // this CTA's spin words in the cluster window
    const uint32_t dlab = (uint32_t)(L.lab - L.s);          // a site's spin word 0 -> its first label word
    const uint32_t qstride = 4u * (uint32_t)nls;            // label arrays of consecutive group pairs; word 0 -> 1
    uint32_t rest0 = act0, rest1 = act1;
    int groups = 0;
    while (rest0 | rest1) {
        uint32_t gm0 = 0u, gm1 = 0u;                 // the next (up to) g pairs, in pair order
        for (int q = 0; q < g && (rest0 | rest1); ++q) {
            if (rest0) {
                gm0 |= rest0 & (0u - rest0);
                rest0 &= rest0 - 1u;
            } else {
                gm1 |= rest1 & (0u - rest1);
                rest1 &= rest1 - 1u;
            }
        }
        const int n0 = __popc(gm0), ng = n0 + __popc(gm1);
        U.span = (uint32_t)ng * qstride;
        ++groups;
        for (int i = tid; i < ng * nls; i += nth) S.lab[i] = U.lab + 4u * (uint32_t)i;
        __syncthreads();
        uf_unions<Z, false>(U, S, gm0, gm1, n0, mys, dlab, qstride);
        cl_sync();                                   // every CTA's own unions are done
        uf_unions<Z, true>(U, S, gm0, gm1, n0, mys, dlab, qstride);
        cl_sync();
        if (tid < ng) {                              // the root of the tid-th group pair's seed
            uint32_t m0 = gm0, m1 = gm1;
            for (int q = 0; q < tid; ++q) {
                if (m0) m0 &= m0 - 1u;
                else m1 &= m1 - 1u;
            }
            const int k = m0 ? (__ffs(m0) - 1) >> 1 : 16 + ((__ffs(m1) - 1) >> 1);
            S.sroot[tid] = uf_root(U, S.sadr[k] + (uint32_t)L.lab + (uint32_t)tid * qstride);
        }
        __syncthreads();
        uf_mark(U, S, gm0, gm1, n0);
        if (rest0 | rest1) cl_sync();                // walks through these labels end before the reset
    }
    __syncthreads();
    if (S.rank == 0 && tid == 0) {
        S.icmst[0] += (unsigned)(__popc(act0) + __popc(act1));
        S.icmst[1] += 4u * (unsigned)groups;         // passes over the own sites
    }
}

// Steps 2a and 2b (see cluster_moves in pt_icm.cu).
template <bool GAUSS, int Z>
__device__ void cl_cluster_moves(const KParams &P, const ClusterLayout &L, const CS &S, uint32_t t, uint32_t inst,
                                 int slot, bool trace)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int N = P.N, nicm = P.n_icm, G = P.G, nls = S.nls, hs = S.hs, NWl = L.NWl;
    ET *E = (ET *)S.E;
    ET *esum = (ET *)S.esum;

    // (a) overlap masks of the own sites, per-colour-block counts
    for (int m = warp; m < NWl; m += nwarps) {
        const int li = 32 * m + lane;
        const uint32_t w0 = S.s[li];
        uint32_t x = (w0 ^ (w0 >> 1)) & 0x55555555u;   // bit 2j: pair j; bit 2j + 1: pair 16 + j
        if (G > 1) {
            const uint32_t w1 = S.s[nls + li];
            x |= ((w1 ^ (w1 >> 1)) & 0x55555555u) << 1;
        }
        const uint32_t col = warp_transpose32(x, lane);
        const int k = (lane >> 1) + 16 * (lane & 1);
        if (k < nicm) S.mask[k * NWl + m] = col;
    }
    for (int i = tid; i < nls; i += nth) S.C[i] = 0u;
    if (tid < 2) S.flipw[tid] = 0u;
    if (tid < 32) S.csz[tid] = 0;
    __syncthreads();
    for (int k = tid; k < nicm; k += nth)
        for (int c = 0; c < 2; ++c) {
            int n = 0;
            for (int m = c * (hs / 32); m < (c + 1) * (hs / 32); ++m) n += __popc(S.mask[k * NWl + m]);
            S.cntloc[c * 32 + k] = n;
        }
    cl_sync();

    // (b) per pair, in every CTA alike: n, step 2a, the seed's owner by rank;
    // the owner plants the seed
    for (int k = tid; k < nicm; k += nth) {
        int n = 0;
        for (int c = 0; c < 2; ++c)
            for (uint32_t r = 0; r < S.K; ++r) n += (int)cl_ld(cl_map(S.base + L.cntloc + 4 * (c * 32 + k), r));
        const int n_pre = n;
        const bool flipped = P.enable_2a && 2 * n > N;
        if (flipped) {
            n = N - n;
            atomicOr(&S.flipw[(2 * k + 1) >> 5], 1u << ((2 * k + 1) & 31));
        }
        int seed_pos = -1;
        if (n > 0) {
            uint32_t x[4];
            philox10k((uint32_t)k, t, 0u, (1u << 24) | inst, P.key, x);
            uint32_t rank = (uint32_t)(((uint64_t)x[0] * (uint32_t)n) >> 32);
            for (int c = 0; c < 2 && seed_pos < 0; ++c)
                for (uint32_t r = 0; r < S.K; ++r) {
                    int cnt = (int)cl_ld(cl_map(S.base + L.cntloc + 4 * (c * 32 + k), r));
                    if (flipped) cnt = hs - cnt;
                    if (rank < (uint32_t)cnt) {
                        if (r == S.rank) {             // this CTA owns the seed: find the local site
                            for (int m = c * (hs / 32); m < (c + 1) * (hs / 32); ++m) {
                                uint32_t w = S.mask[k * NWl + m];
                                if (flipped) w = ~w;
                                const uint32_t pc = (uint32_t)__popc(w);
                                if (rank < pc) {
                                    const int li = 32 * m + nth_set_bit(w, rank);
                                    atomicOr(S.C + ICM_IDX(li, nls, 21), 1u << (2 * (k & 15) + (k >> 4)));
                                    if (L.ufg) {       // the seed's site address, for the union-find roots
                                        const uint32_t sa = cl_map(S.base, S.rank) + 4u * (uint32_t)li;
                                        for (uint32_t r2 = 0; r2 < S.K; ++r2) cl_st(cl_map(S.base + L.sadr + 4 * k, r2), sa);
                                    }
                                    if (trace) P.tr_seed[(size_t)slot * P.nT + k] = (int)__ldg(P.pos2site + pos_of(P, S, li));
                                    break;
                                }
                                rank -= pc;
                            }
                        }
                        seed_pos = c * P.half + (int)r * hs;   // block of the seed (the owner records the site)
                        break;
                    }
                    rank -= (uint32_t)cnt;
                }
        }
        S.seed[k] = seed_pos >= 0;
        esum[k] = E[2 * k] + E[2 * k + 1];
        if (trace && S.rank == 0) {
            const size_t o = (size_t)slot * P.nT + k;
            P.tr_n_pre[o] = n_pre;
            P.tr_flip2a[o] = flipped;
            if (seed_pos < 0) P.tr_seed[o] = -1;
            P.tr_csize[o] = 0;
            P.tr_eb[o] = (float)(E[2 * k] + E[2 * k + 1]);
            P.tr_ea[o] = (float)(E[2 * k] + E[2 * k + 1]);
        }
    }
    cl_sync();

    // (c) step 2a on the own sites, then the clusters of all pairs at once
    uint32_t act0 = 0u, act1 = 0u;
    for (int k = 0; k < nicm; ++k)
        if (S.seed[k]) {
            if (k < 16) act0 |= 1u << (2 * k);
            else act1 |= 1u << (2 * (k - 16));
        }
    const uint32_t f0 = S.flipw[0], f1 = S.flipw[1];
    for (int li = tid; li < nls; li += nth) {
        S.s[li] ^= f0;
        if (G > 1) S.s[nls + li] ^= f1;
    }
    if (!(act0 | act1)) {
        __syncthreads();
        return;                                      // the same decision in every CTA
    }
    // One cluster word per site holds every pair: bit 2j = pair j, bit 2j + 1
    // = pair 16 + j, so that the domain word is q of the first spin word | q
    // of the second << 1 and a neighbour is one load.
    // Growth in cluster rounds of kScansPerRound in-place scans of the own
    // sites (6: 2D L=128 and 3D L=16 on 8 x 512 +3.3% and +1.3% against 4,
    // where a round that grows from 2 to 8 scans lost 2.7% on 3D L=16).
    // Within a round the CTAs scan without barriers, reading each other's
    // words as they are.  A warp that grew a site writes the round's
    // stamp into the stamp word of every CTA of the cluster; after the
    // round's barrier each CTA reads its own word, so all CTAs decide alike.
    // The growth ends after a round in which nothing grew: every read of that
    // round saw the state that the previous barrier published, and no site
    // could grow from it, so it is the fixed point, each seed's component of
    // q = -1.  Stamps are (t << 16) + round + 1 (at most N < 2^16 rounds), so
    // words need no reset; a stale equal value could only add one empty round.
    constexpr int kScansPerRound = 6;
    const uint32_t actc = act0 | (act1 << 1);
    // with at most four own sites per thread, each thread keeps their domain
    // and cluster words in registers across the scans and skips the sites
    // already absorbed (2D L=128 on 8 x 512: +8%, with 50-100 bytes of
    // register spills under the 64 registers of the launch bounds).  On 2D
    // lattices with four sites per thread the host gives each thread a 2 x 2
    // block of sites, taken around the block (S.gord): a scan then carries
    // the growth across the block and into the next lane's block (a model of
    // the in-place scans on this workload's domains: 118 scans per sweep
    // instead of 155).
    const bool in_regs = nls <= 4 * nth;
    auto own = [&](int j) { return S.gord ? (int)S.gord[4 * tid + j] : tid + j * nth; };
    uint32_t dm[4], cw[4];
    uint32_t todo = 0u;                              // bit j: own site j not yet absorbed
    if (!L.ufg && in_regs) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int li = own(j);
            dm[j] = cw[j] = 0u;
            if (tid + j * nth < nls) {
                const uint32_t w0 = S.s[li], w1 = G > 1 ? S.s[nls + li] : 0u;
                dm[j] = (((w0 ^ (w0 >> 1)) & 0x55555555u) | (((w1 ^ (w1 >> 1)) & 0x55555555u) << 1)) & actc;
                cw[j] = S.C[li];
                if (dm[j] != cw[j]) todo |= 1u << j;
            }
        }
    }
    if (L.ufg) cl_grow_uf<Z>(P, L, S, act0, act1);
    else for (int round = 0;; ++round) {
        int grew = 0;
        if (in_regs) {
            for (int scan = 0; scan < kScansPerRound; ++scan) {
                // the thread's four block sites in one 8-byte load
                uint2 o = make_uint2(0u, 0u);
                if (S.gord) o = *reinterpret_cast<const uint2 *>(S.gord + 4 * tid);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // absorbed sites are skipped, except on 2D lattices, where the
                    // test costs more than it saves (2D L=128: +3.9% without it;
                    // 3D L=16: -1.7%)
                    if constexpr (Z != 4) {
                        if (!((todo >> j) & 1u)) continue;
                    } else {
                        if (tid + j * nth >= nls) continue;
                    }
                    const int li = S.gord ? (int)(((j < 2 ? o.x : o.y) >> (16 * (j & 1))) & 0xFFFFu) : tid + j * nth;
                    uint32_t nb = 0u;
                    // the site's neighbour row in one 16-byte (Z = 4) or 8-byte loads
                    // (2D L=128 on 8 x 512: +22% against four 4-byte loads)
                    uint32_t e[Z];
                    nb_row<Z>(S.nb, li, e);
#pragma unroll
                    for (int d = 0; d < Z; ++d) nb |= cl_ld(e[d]);
                    const uint32_t n = cw[j] | (dm[j] & nb);
                    if (n != cw[j]) {
                        S.C[li] = n;
                        cw[j] = n;
                        grew = 1;
                        if constexpr (Z != 4)
                            if (n == dm[j]) todo &= ~(1u << j);
                    }
                }
            }
        } else {
            for (int scan = 0; scan < kScansPerRound; ++scan)
                for (int li = tid; li < nls; li += nth) {
                    const uint32_t w0 = S.s[li], w1 = G > 1 ? S.s[nls + li] : 0u;
                    const uint32_t dmw = (((w0 ^ (w0 >> 1)) & 0x55555555u) | (((w1 ^ (w1 >> 1)) & 0x55555555u) << 1)) & actc;
                    const uint32_t c = S.C[li];
                    if (dmw == c) continue;
                    uint32_t e[Z], nb = 0u;
                    nb_row<Z>(S.nb, li, e);
#pragma unroll
                    for (int d = 0; d < Z; ++d) nb |= cl_ld(e[d]);
                    const uint32_t n = c | (dmw & nb);
                    if (n != c) {
                        S.C[li] = n;
                        grew = 1;
                    }
                }
        }
        const uint32_t stamp = (t << 16) + (uint32_t)round + 1u;
        if (__any_sync(kFull, grew) && lane == 0)
            for (uint32_t r = 0; r < S.K; ++r) cl_st(cl_map(S.base + L.flags + 4 * (round & 1), r), stamp);
        cl_sync();
        if ((uint32_t)S.flags[round & 1] != stamp) {
            if (S.rank == 0 && tid == 0) {
                S.icmst[0] += (unsigned)(__popc(act0) + __popc(act1));
                S.icmst[1] += (unsigned)(round + 1) * kScansPerRound;   // scans of the own sites
            }
            break;
        }
    }

    // (d) flip the own sites; copy-a energies of the moved pairs
    for (int li = tid; li < nls; li += nth) {
        const uint32_t cw = S.C[li];
        const uint32_t c0 = cw & 0x55555555u, c1 = (cw >> 1) & 0x55555555u;
        if (c0) S.s[li] ^= c0 | (c0 << 1);
        if (c1) S.s[nls + li] ^= c1 | (c1 << 1);
        if (trace) {
            for (int w = 0; w < 2; ++w)
                for (uint32_t b = w ? c1 : c0; b; b &= b - 1u) atomicAdd(&S.csz[16 * w + ((__ffs(b) - 1) >> 1)], 1);
            if (P.tr_cmask) {
                uint32_t *cm = P.tr_cmask + ((size_t)slot * N + pos_of(P, S, li)) * 2;
                cm[0] = c0;
                cm[1] = c1;
            }
        }
    }
    cl_sync();                                       // flipped words of other CTAs are read below
    // copy-a energies of the moved pairs (cb = 0); a traced sweep then also
    // recomputes the copy-b energies (cb = 1) and records E_a + E_b of the two
    // recomputed energies, so that the trace tests the conservation of E_a + E_b
    ET *part = (ET *)S.Epart;
    for (int cb = 0; cb < (trace ? 2 : 1); ++cb) {
        if (cb) cl_sync();                           // every CTA has read the copy-a shares
        for (int g = 0; g < G; ++g) {
            const uint32_t act = g ? act1 : act0;
            if (!act) continue;
            const uint32_t goff = (uint32_t)(g * nls * 4) - S.dCs;   // neighbour entry -> its spin word g
            const uint32_t *sg = S.s + g * nls;
            ET acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = ET(0);
            for (int j = tid; j < hs; j += nth) {
                const int li = hs + j;               // colour-1 sites: every bond once
                const uint32_t sw = sg[li] >> cb;
                uint32_t nw[Z];
                nb_row<Z>(S.nb, li, nw);
#pragma unroll
                for (int d = 0; d < Z; ++d) nw[d] = cl_ld(nw[d] + goff) >> cb;
                if constexpr (GAUSS) {
                    float J2[Z];
                    float Jsum = 0.f;
#pragma unroll
                    for (int d = 0; d < Z; ++d) {
                        const float J = S.Jd[li * Z + d];
                        Jsum += J;
                        J2[d] = 2.f * J;
                    }
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        if (!((act >> (2 * jj)) & 1u)) continue;
                        const int b = 2 * jj;
                        float h = Jsum;
#pragma unroll
                        for (int d = 0; d < Z; ++d)
                            if ((nw[d] >> b) & 1u) h -= J2[d];
                        acc[jj] += ((sw >> b) & 1u) ? h : -h;
                    }
                } else {
                    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
                    const uint32_t jb = S.Jb[li];
                    uint32_t u[Z];
#pragma unroll
                    for (int d = 0; d < Z; ++d) u[d] = sw ^ nw[d] ^ (0u - ((jb >> d) & 1u));
                    csa_count<Z>(u, c0, c1, c2, c3);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int b = 2 * jj;
                        acc[jj] += (int)(((c0 >> b) & 1u) | (((c1 >> b) & 1u) << 1) | (((c2 >> b) & 1u) << 2) |
                                         (((c3 >> b) & 1u) << 3));
                    }
                }
            }
            const ET v = transpose_reduce16(acc, lane);
            if (!(lane & 1)) part[warp * 32 + 16 * g + (lane >> 1)] = v;
        }
        __syncthreads();
        for (int k = tid; k < nicm; k += nth) {
            ET e = ET(0);
            if (S.seed[k])
                for (int w = 0; w < nwarps; ++w) e += part[w * 32 + k];
            ((ET *)S.Epair)[k] = e;
        }
        cl_sync();
        for (int k = tid; k < nicm; k += nth) {
            if (!S.seed[k]) continue;
            ET e = cl_sum<ET>(S, L.Epair + 4 * k);
            if constexpr (!GAUSS) e = 2 * e - (P.diluted ? P.nb_inst[slot] : P.Nb);   // E = 2 U - N_b (bonds present)
            if (cb == 0) {
                E[2 * k] = e;
                E[2 * k + 1] = esum[k] - e;
            }
            if (trace && S.rank == 0) {
                const size_t o = (size_t)slot * P.nT + k;
                if (cb == 0) {
                    int cs = 0;
                    for (uint32_t r = 0; r < S.K; ++r) cs += (int)cl_ld(cl_map(S.base + L.csz + 4 * k, r));
                    P.tr_csize[o] = cs;
                } else {
                    P.tr_ea[o] = (float)(E[2 * k] + e);
                }
            }
        }
        __syncthreads();
    }
}

// Step 3 (see pt_pass in pt_icm.cu): the same energies and draws in every
// CTA give the same decisions; each CTA permutes its own words.
template <bool GAUSS>
__device__ void cl_pt_pass(const KParams &P, const CS &S, uint32_t t, uint32_t inst, int slot, bool trace)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int nT = P.nT, np = nT - 1, nls = S.nls;
    for (int i = threadIdx.x; i < 2 * np; i += blockDim.x) {
        const int c = i / np, k = i % np;
        uint32_t x[4];
        philox10k((uint32_t)k, t, (uint32_t)c, (2u << 24) | inst, P.key, x);
        if constexpr (GAUSS) S.swap_x[c * 32 + k] = pt_word_gauss(x[0]);
        else S.swap_x[c * 32 + k] = pt_word_pmj(x[0], P.thr_swap + P.swap_off[k], P.swap_len[k], P.dbeta_l2e[k]);
    }
    __syncthreads();
    // every CTA decides alike (the same energies and draws); rank 0 traces
    if (threadIdx.x < 32)
        pt_warp<GAUSS, ET>((ET *)S.E, P.R, np, S.swap_x, P.dbeta_l2e, S.swap_list, S.swap_n, S.swap_mask,
                           trace && S.rank == 0 ? P.tr_swap + (size_t)slot * 2 * np : nullptr);
    __syncthreads();
    const int n0 = S.swap_n[0], n1 = S.swap_n[1];
    if (n0 + n1 > 0) {
        const SwapMasks m = swap_masks(S.swap_list, n0, n1, S.swap_mask);
        const bool two = P.G > 1;
        for (int li = threadIdx.x; li < nls; li += blockDim.x) {
            const uint64_t x = (uint64_t)S.s[li] | (two ? (uint64_t)S.s[nls + li] << 32 : 0ull);
            const uint64_t y = swap_apply(m, x);
            S.s[li] = (uint32_t)y;
            if (two) S.s[nls + li] = (uint32_t)(y >> 32);
        }
    }
    cl_sync();                                       // the observables read other CTAs' words
}

// Observables (see measure in pt_icm.cu): per-CTA counts, summed by rank 0.
template <bool GAUSS, int Z>
__device__ void cl_measure(const KParams &P, const ClusterLayout &L, const CS &S, int slot)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31;
    const int N = P.N, nT = P.nT, nls = S.nls, hs = S.hs;
    if (threadIdx.x < 32) {
        S.cnt_n[threadIdx.x] = 0;
        S.cnt_d[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int g = 0; g < P.G; ++g) {
        const int npair = min(16, nT - 16 * g);
        const uint32_t goff = (uint32_t)(g * nls * 4) - S.dCs;   // neighbour entry -> its spin word g
        const uint32_t *sg = S.s + g * nls;
        uint32_t pl[kPlanes];   // even bit 2k: q = -1 sites of pair k; odd bit 2k+1: its q_i q_j = -1 bonds
#pragma unroll
        for (int i = 0; i < kPlanes; ++i) pl[i] = 0u;
        for (int li = threadIdx.x; li < nls; li += blockDim.x) {
            const uint32_t w = sg[li];
            vadd(pl, (w ^ (w >> 1)) & 0x55555555u);
        }
        for (int li = hs + threadIdx.x; li < nls; li += blockDim.x) {
            const uint32_t w = sg[li];
            const uint32_t qp = (w ^ (w >> 1)) & 0x55555555u;
            uint32_t x[Z];                 // a padding entry points at the site itself: x = 0
            nb_row<Z>(S.nb, li, x);
#pragma unroll
            for (int d = 0; d < Z; ++d) {
                const uint32_t wq = cl_ld(x[d] + goff);
                x[d] = (qp ^ ((wq ^ (wq >> 1)) & 0x55555555u)) << 1;
            }
            uint32_t c0, c1, c2, c3;
            csa_count<Z>(x, c0, c1, c2, c3);
            vadd4(pl, c0, c1, c2, c3);
        }
        const int v = warp_vsum(pl, lane);   // lane 2k: n of pair k, lane 2k+1: d of pair k
        if (lane < 2 * npair) atomicAdd(((lane & 1) ? S.cnt_d : S.cnt_n) + 16 * g + (lane >> 1), v);
    }
    cl_sync();
    if (S.rank == 0) {
        for (int k = threadIdx.x; k < nT; k += blockDim.x) {
            long long n = 0, d = 0;
            for (uint32_t r = 0; r < S.K; ++r) {
                n += (int)cl_ld(cl_map(S.base + L.cnt_n + 4 * k, r));
                d += (int)cl_ld(cl_map(S.base + L.cnt_d + 4 * k, r));
            }
            const ET *E = (const ET *)S.E;
            S.accE[k] += (double)E[2 * k] + (double)E[2 * k + 1];
            S.acc64[0 * nT + k] += n;
            S.acc64[1 * nT + k] += (N - 2 * n) * (N - 2 * n);
            S.acc64[2 * nT + k] += n < N - n ? n : N - n;
            S.acc64[3 * nT + k] += d;
            atomicAdd(&P.hist[((size_t)slot * nT + k) * (N + 1) + ICM_IDX(n, N + 1, 22)], 1ull);
        }
        if (threadIdx.x == 0) S.nmeas[0] += 1;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
template <bool GAUSS, int Z, bool DIL>
__global__ void __launch_bounds__(kMaxThreadsWide, 1) cluster_kernel(const KParams P, const ClusterLayout L,
                                                                    uint32_t n_sweeps)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const CS S = make_cs(smem, L);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int N = P.N, R = P.R, nT = P.nT, G = P.G, nls = S.nls, hs = S.hs, half = P.half;

    if (tid < 2) S.flags[tid] = 0;   // growth round stamps (the same in every CTA at all times)
    // neighbour table: cluster-window address of each neighbour's cluster word
    // (of the batch's lattice here; per instance for diluted batches, below)
    auto neighbour_table = [&](const uint16_t *nbr, const uint8_t *zdeg) {
        for (int i = tid; i < nls * Z; i += nth) {
            const int li = i / Z, d = i % Z;
            const int q = ICM_IDX(nbr[pos_of(P, S, li) * Z + d], N, 20);
            const int cq = q >= half;
            const int hq = q - cq * half;
            const uint32_t rq = (uint32_t)(hq / hs);
            const int lq = cq * hs + hq % hs;
            S.nb[i] = cl_map(S.base + L.C, rq) + 4u * (uint32_t)lq;
        }
        if (!GAUSS && (DIL || !P.const_z))
            for (int li = tid; li < nls; li += nth) S.zdeg[li] = zdeg[pos_of(P, S, li)];
    };
    if constexpr (!DIL) neighbour_table(P.nbr, P.zdeg);
    if (L.gord >= 0)
        for (int i = tid; i < nls; i += nth) S.gord[i] = P.cl_order[i];
    if constexpr (GAUSS) {
        for (int r = tid; r < 32 * G; r += nth) S.b2l[r] = r < R ? P.b2l[r] : 0.f;
    } else {
        constexpr int TS = thr_stride(Z);
        for (int i = tid; i < 32 * G * TS; i += nth) S.thr[i] = i < R * TS ? P.thr_metro[i] : 0u;
    }

    for (int slot = (int)cl_id(); slot < P.n_inst; slot += (int)cl_count()) {
        if (P.active && !P.active[slot]) continue;   // the same for every CTA of the cluster
        for (int i = tid; i < G * nls; i += nth) {
            const int g = i / nls, li = i % nls;
            S.s[i] = P.spins[((size_t)slot * G + g) * N + pos_of(P, S, li)];
        }
        if constexpr (GAUSS) {
            for (int i = tid; i < nls * Z; i += nth)
                S.Jd[i] = P.Jd[((size_t)slot * N + pos_of(P, S, i / Z)) * Z + i % Z];
            for (int r = tid; r < R; r += nth) ((float *)S.E)[r] = P.Ef[(size_t)slot * R + r];
        } else {
            for (int li = tid; li < nls; li += nth) S.Jb[li] = P.Jb[(size_t)slot * N + pos_of(P, S, li)];
            for (int r = tid; r < R; r += nth) ((int *)S.E)[r] = P.Ei[(size_t)slot * R + r];
        }
        if (S.rank == 0) {
            for (int k = tid; k < nT; k += nth) {
                S.accE[k] = P.accE[(size_t)slot * nT + k];
                for (int a = 0; a < 4; ++a) S.acc64[a * nT + k] = P.acc64[((size_t)a * P.n_inst + slot) * nT + k];
            }
            if (tid == 0) {
                S.nmeas[0] = P.n_meas[slot];
                S.icmst[0] = S.icmst[1] = 0ull;
            }
        }
        // a diluted instance: its own neighbour table (absent bonds point at the
        // site itself) and degrees, and zero-energy proposals accepted with
        // probability 1/2
        bool tie = false;
        if constexpr (DIL) {
            neighbour_table(P.nbr_inst + (size_t)slot * N * Z, P.zdeg_inst + (size_t)slot * N);
            tie = P.nb_inst[slot] < P.Nb;
        }
        const uint32_t inst = P.inst_id[slot];
        const long long t_meas = P.t_meas_inst ? P.t_meas_inst[slot] : P.t_meas;
        uint32_t t = P.tsweep[slot];
        cl_sync();

        for (uint32_t step = 0; step < n_sweeps; ++step, ++t) {
            const bool trace = P.trace && step + 1 == n_sweeps;
            if (trace && S.rank == 0) {
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
            }
            if (trace && P.tr_cmask)                 // every CTA clears its own positions
                for (int li = tid; li < nls; li += nth) {
                    uint32_t *cm = P.tr_cmask + ((size_t)slot * N + pos_of(P, S, li)) * 2;
                    cm[0] = 0u;
                    cm[1] = 0u;
                }
            cl_sync();                               // buffers read remotely in the last step are free again
            if (P.enable_metropolis) cl_metropolis<GAUSS, Z, DIL>(P, L, S, t, inst, tie);
            if (P.icm_every > 0 && t % (uint32_t)P.icm_every == 0 && P.n_icm > 0)
                cl_cluster_moves<GAUSS, Z>(P, L, S, t, inst, slot, trace);
            if (P.swap_every > 0 && t % (uint32_t)P.swap_every == 0 && nT > 1) cl_pt_pass<GAUSS>(P, S, t, inst, slot, trace);
            else cl_sync();                          // 2a and cluster flips visible to the observables
            if ((long long)t >= t_meas) cl_measure<GAUSS, Z>(P, L, S, slot);
        }

        for (int i = tid; i < G * nls; i += nth) {
            const int g = i / nls, li = i % nls;
            P.spins[((size_t)slot * G + g) * N + pos_of(P, S, li)] = S.s[i];
        }
        if (S.rank == 0) {
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
        }
        cl_sync();
    }
}

template <bool GAUSS, int Z, bool DIL>
cudaError_t launch_cluster_t(const KParams &P, const ClusterLayout &L, int threads, int n_clusters, uint32_t n_sweeps,
                             cudaStream_t st)
{
    auto kern = cluster_kernel<GAUSS, Z, DIL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_clusters * L.K), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)L.total;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)L.K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, P, L, n_sweeps);
}

template <bool GAUSS, int Z, bool DIL>
cudaError_t cluster_occupancy_t(int K, int threads, int smem, int *clusters)
{
    auto kern = cluster_kernel<GAUSS, Z, DIL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)K, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, kern, &cfg);
}

int align_up16(int v) { return (v + 15) / 16 * 16; }

}  // namespace

ClusterLayout cluster_layout(int N, int Z, int R, int G, int nT, int K, int nwarps, bool gauss, int ufg,
                             bool order)
{
    ClusterLayout L{};
    L.K = K;
    L.ufg = ufg;
    L.hs = (N / 2) / K;
    L.nls = 2 * L.hs;
    L.NWl = L.nls / 32;
    int o = 0;
    auto take = [&](int bytes) {
        o = align_up16(o);
        const int at = o;
        o += bytes;
        return at;
    };
    const int nls = L.nls;
    L.s = take(G * nls * 4);
    L.C = take(nls * 4);
    L.nb = take(nls * Z * 4);
    L.coup = take(gauss ? nls * Z * 4 : nls);
    L.zdeg = take(nls);
    L.E = take(R * 4);
    L.Epart = take(nwarps * (R > 32 ? R : 32) * 4);
    L.Esw = take(R * 4);
    L.Epair = take(32 * 4);
    L.rtab = take(gauss ? G * 32 * 4 : G * 32 * thr_stride(Z) * 4);
    // the overlap masks are dead once the seeds are planted: the union-find
    // labels take their place (one pair's labels are as large as the masks)
    L.lab = take((ufg > 1 ? ufg : 1) * nls * 4);
    L.mask = L.lab;
    L.sadr = take(32 * 4);
    L.sroot = take(kMaxUfGroup * 4);
    L.gord = order ? take(nls * 2) : -1;
    L.cntloc = take(2 * 32 * 4);
    L.flags = take(2 * 4);
    L.seed = take(32 * 4);
    L.esum = take(32 * 4);
    L.flipw = take(2 * 4);
    L.csz = take(32 * 4);
    L.swap_x = take(2 * 32 * 4);
    L.swap_list = take(2 * 32 * 4);
    L.swap_n = take(2 * 4);
    L.swap_mask = take(2 * 8);
    L.cnt_n = take(32 * 4);
    L.cnt_d = take(32 * 4);
    L.accE = take(nT * 8);
    L.acc64 = take(4 * nT * 8);
    L.nmeas = take(8);
    L.icmst = take(16);
    L.total = align_up16(o);
    return L;
}

cudaError_t launch_cluster(const KParams &P, const ClusterLayout &L, bool gauss, int threads, int n_clusters,
                           uint32_t n_sweeps, cudaStream_t st)
{
    if (threads > kMaxThreadsWide || L.K < 1 || L.hs % 32) return cudaErrorInvalidValue;
    if (P.diluted && (!P.nbr_inst || !P.zdeg_inst || !P.nb_inst)) return cudaErrorInvalidValue;
#define ICM_LAUNCH_CL(G_, Z_)                                                                          \
    (P.diluted ? launch_cluster_t<G_, Z_, true>(P, L, threads, n_clusters, n_sweeps, st)               \
               : launch_cluster_t<G_, Z_, false>(P, L, threads, n_clusters, n_sweeps, st))
    if (gauss) return P.Z == 4 ? ICM_LAUNCH_CL(true, 4) : P.Z == 6 ? ICM_LAUNCH_CL(true, 6) : ICM_LAUNCH_CL(true, 8);
    return P.Z == 4 ? ICM_LAUNCH_CL(false, 4) : P.Z == 6 ? ICM_LAUNCH_CL(false, 6) : ICM_LAUNCH_CL(false, 8);
#undef ICM_LAUNCH_CL
}

cudaError_t cluster_occupancy(bool gauss, int Z, bool dil, int K, int threads, int smem, int *clusters)
{
    if (Z != 4 && Z != 6 && Z != 8) return cudaErrorInvalidValue;
#define ICM_OCC_CL(G_, Z_)                                                                             \
    (dil ? cluster_occupancy_t<G_, Z_, true>(K, threads, smem, clusters)                                \
         : cluster_occupancy_t<G_, Z_, false>(K, threads, smem, clusters))
    if (gauss) return Z == 4 ? ICM_OCC_CL(true, 4) : Z == 6 ? ICM_OCC_CL(true, 6) : ICM_OCC_CL(true, 8);
    return Z == 4 ? ICM_OCC_CL(false, 4) : Z == 6 ? ICM_OCC_CL(false, 6) : ICM_OCC_CL(false, 8);
#undef ICM_OCC_CL
}

}  // namespace icm

#ifdef ICM_CHECKED
// Checked builds: the check word of the thread-block-cluster kernels (guarded
// neighbour positions, seed sites and histogram bins; site codes 20-22), read
// like icm_debug_check reads those of the fused kernels.
extern "C" int icm_debug_check_cluster(unsigned int *out, int reset)
{
    if (cudaMemcpyFromSymbol(out, icm::g_icm_check, sizeof(unsigned int) * 4) != cudaSuccess) return -4;
    if (reset) {
        unsigned int z[4] = {};
        if (cudaMemcpyToSymbol(icm::g_icm_check, z, sizeof(z)) != cudaSuccess) return -4;
    }
    return 0;
}
#endif
