// icm_device.cuh -- device helpers shared by the fused kernels (pt_icm.cu)
// and the thread-block-cluster kernel (cluster_icm.cu): Philox4x32-10, the
// ex2 approximation, warp reductions and bit-sliced (vertical) counters.
// Included into an anonymous namespace of each translation unit.
#pragma once
#include <cstdint>

namespace icm {
namespace {

constexpr uint32_t kFull = 0xffffffffu;

// Checked builds (-DICM_CHECKED): ICM_IDX(i, n, site) tests a data-dependent
// index against its bound.  An index out of range is counted in g_icm_check
// (count, then the site code, index and bound of the first one) and replaced
// by 0, so the access stays inside the array and the kernel runs on; the
// host reads the word with icm_debug_check.  In normal builds ICM_IDX is the
// index itself.  (The substitute for a memory checker on this pool.)
#ifdef ICM_CHECKED
static __device__ unsigned int g_icm_check[4];
__device__ __forceinline__ int icm_guard(int idx, int bound, int site)
{
    if ((unsigned)idx < (unsigned)bound) return idx;
    if (atomicAdd(&g_icm_check[0], 1u) == 0u) {
        g_icm_check[1] = (unsigned)site;
        g_icm_check[2] = (unsigned)idx;
        g_icm_check[3] = (unsigned)bound;
    }
    return 0;
}
#define ICM_IDX(i, n, site) icm_guard((int)(i), (int)(n), (site))
#else
#define ICM_IDX(i, n, site) (i)
#endif

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds, multipliers
// 0xD2511F53 / 0xCD9E8D57; the round keys are the Weyl sequence of the
// 64-bit key (increments 0x9E3779B9 / 0xBB67AE85), taken here from a table
// computed once per batch (key[2i], key[2i+1] = the key of round i, see
// KParams::key).
__device__ __forceinline__ void philox10k(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          const uint32_t (&key)[20], uint32_t (&o)[4])
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint64_t m0 = (uint64_t)c0 * 0xD2511F53ull;
        const uint64_t m1 = (uint64_t)c2 * 0xCD9E8D57ull;
        const uint32_t n0 = (uint32_t)(m1 >> 32) ^ c1 ^ key[2 * i];
        const uint32_t n2 = (uint32_t)(m0 >> 32) ^ c3 ^ key[2 * i + 1];
        c1 = (uint32_t)m1;
        c3 = (uint32_t)m0;
        c0 = n0;
        c2 = n2;
    }
    o[0] = c0; o[1] = c1; o[2] = c2; o[3] = c3;
}

// Two Philox4x32-10 blocks with counters {c0, c1, c2, c3} and {c0, c1, c2+1, c3},
// written as two independent chains so that the scheduler can interleave them;
// round keys from a table as in philox10k.
__device__ __forceinline__ void philox10x2(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           const uint32_t (&key)[20], uint32_t (&o)[4], uint32_t (&p)[4])
{
    uint32_t a0 = c0, a1 = c1, a2 = c2, a3 = c3;
    uint32_t b0 = c0, b1 = c1, b2 = c2 + 1u, b3 = c3;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t k0 = key[2 * i], k1 = key[2 * i + 1];
        const uint64_t ma0 = (uint64_t)a0 * 0xD2511F53ull, ma1 = (uint64_t)a2 * 0xCD9E8D57ull;
        const uint64_t mb0 = (uint64_t)b0 * 0xD2511F53ull, mb1 = (uint64_t)b2 * 0xCD9E8D57ull;
        const uint32_t na0 = (uint32_t)(ma1 >> 32) ^ a1 ^ k0, na2 = (uint32_t)(ma0 >> 32) ^ a3 ^ k1;
        const uint32_t nb0 = (uint32_t)(mb1 >> 32) ^ b1 ^ k0, nb2 = (uint32_t)(mb0 >> 32) ^ b3 ^ k1;
        a1 = (uint32_t)ma1; a3 = (uint32_t)ma0; a0 = na0; a2 = na2;
        b1 = (uint32_t)mb1; b3 = (uint32_t)mb0; b0 = nb0; b2 = nb2;
    }
    o[0] = a0; o[1] = a1; o[2] = a2; o[3] = a3;
    p[0] = b0; p[1] = b1; p[2] = b2; p[3] = b3;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Step 3 (the PT pass).  For each copy c the swaps (k, k+1), k = 0 .. np-1, are
// decided in ascending k; an accepted swap moves the configuration at k up to
// k+1, so the energy compared at step k+1 is the one carried up (or, after a
// rejection, the original energy at k+1).  The draw x of (c, k) is first
// turned into the form its test takes inside that sequential loop:
//  * Gaussian: accept iff Delta >= 0 or u < 2^Delta, with Delta = (beta_k -
//    beta_{k+1}) log2(e) (E_k - E_{k+1}) and u = (x >> 8) 2^-24, that is iff
//    Delta >= 0 or log2(u) < Delta: the word is log2(u) (fp32 bits);
//  * +-J: accept iff E_k >= E_{k+1} or x < thr[d - 1], d = (E_{k+1} - E_k) / 2
//    in 1..len (thr = floor(exp(-2 d (beta_k - beta_{k+1})) 2^32), non-
//    increasing in d), that is iff d <= d_lim, the number of leading
//    thresholds above x: the word is d_lim, found from the closed form of
//    thr and checked against the table.
__device__ __forceinline__ uint32_t pt_word_gauss(uint32_t x)
{
    return __float_as_uint(__log2f((float)(x >> 8) * (1.0f / 16777216.0f)));
}

__device__ __forceinline__ uint32_t pt_word_pmj(uint32_t x, const uint32_t *thr, int len, float dbl)
{
    // thr[d-1] > x iff exp(-2 d dbeta) 2^32 >= x + 1 iff d <= (32 - log2(x + 1)) / (2 dbl),
    // dbl = dbeta log2(e): start there, then step to the exact count against
    // the table (from any start: up while thr[d] > x, down while thr[d-1] <= x)
    const float est = (32.f - __log2f((float)x + 1.f)) / (2.f * dbl);
    int d = est >= (float)len ? len : (est > 0.f ? (int)est : 0);
    while (d < len && __ldg(thr + d) > x) ++d;
    while (d > 0 && __ldg(thr + d - 1) <= x) --d;
    return (uint32_t)d;
}

// The passes of both copies, run by one warp: lanes 16c .. 16c+15 run copy c.
// Each lane runs its copy's sequential decisions (loads and compares only:
// the energies at positions k+1 are read as they were before the pass); then
// lane h of copy c, for the positions k = h and h + 16, writes the energy of
// position k after the pass, the run of accepted swaps that starts at k as a
// (source, destination) pair of replica slots, and its trace byte; lane 0 of
// each half writes its copy's run count and the mask of replica slots whose
// configuration moves down one position.
//   E [R] energies, slot 2k + c; w [2][32] words of pt_word_* (copy c at 32 c);
//   dbl [np] (beta_k - beta_{k+1}) log2(e) (Gaussian); list [2][32];
//   nlist [2]; down [2]; trace [2][np] or null.
template <bool GAUSS, typename ET>
__device__ __forceinline__ void pt_warp(ET *E, int R, int np, const uint32_t *w, const float *dbl, int *list,
                                        int *nlist, uint64_t *down, uint8_t *trace)
{
    const int lane = threadIdx.x & 31, c = lane >> 4, h = lane & 15;
    const uint32_t *wc = w + 32 * c;
    uint32_t acc = 0u;
    ET ek = E[c];
#pragma unroll 4
    for (int k = 0; k < 31; ++k) {
        if (k < np) {
            const ET ek1 = E[ICM_IDX(2 * k + 2 + c, R, 11)];
            bool a;
            if constexpr (GAUSS) {
                const float delta = dbl[k] * (ek - ek1);
                a = (delta >= 0.f) || (__uint_as_float(wc[k]) < delta);
            } else {
                const int dE = ek - ek1;                   // even: +-J energies differ by 2 d
                a = (dE >= 0) || (((-dE) >> 1) <= (int)wc[k]);
            }
            acc |= (uint32_t)a << k;
            if (!a) ek = ek1;
        }
    }
    // position k after the pass: the configuration from k+1 if swap k was
    // accepted; else, if swap k-1 was, the one that started the run at rs;
    // else its own
    ET en[2];
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int k = h + 16 * it;
        en[it] = ET(0);
        if (k <= np) {
            if ((acc >> k) & 1u) en[it] = E[2 * k + 2 + c];
            else if (k > 0 && ((acc >> (k - 1)) & 1u)) en[it] = E[2 * (32 - __clz(~acc & ((1u << k) - 1u))) + c];
            else en[it] = E[2 * k + c];
        }
    }
    __syncwarp();
    const uint32_t starts = acc & ~(acc << 1);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int k = h + 16 * it;
        if (k <= np) E[2 * k + c] = en[it];
        if (k < np) {
            if ((starts >> k) & 1u) {
                const int end = k + __ffs(~(acc >> k)) - 1;    // the first rejected swap above k (or np)
                list[32 * c + ICM_IDX(__popc(starts & ((1u << k) - 1u)), 32, 12)] = ((2 * k + c) << 8) | (2 * end + c);
            }
            if (trace) trace[c * np + k] = (uint8_t)((acc >> k) & 1u);
        }
    }
    if (h == 0) {
        nlist[c] = __popc(starts);
        uint64_t D = 0;
        for (uint32_t b = acc; b; b &= b - 1u) D |= 1ull << (2 * (__ffs(b) - 1) + 2 + c);
        down[c] = D;
    }
}

// Bit position of the rank-th set bit of w, counting from bit 0 (rank <
// popc(w)): five halvings of the window by the popcount of its lower half.
__device__ __forceinline__ int nth_set_bit(uint32_t w, uint32_t rank)
{
    int pos = 0;
#pragma unroll
    for (int hw = 16; hw >= 1; hw >>= 1) {
        const uint32_t lo = w & ((1u << hw) - 1u);
        const uint32_t cl = (uint32_t)__popc(lo);
        if (rank >= cl) {
            rank -= cl;
            w >>= hw;
            pos += hw;
        } else {
            w = lo;
        }
    }
    return pos;
}

// The configuration moves of one PT pass as masks of the 64 replica bits of a
// site (two words).  A run of accepted swaps k..m, list entry
// (2k + c) << 8 | 2(m + 1) + c, moves the configuration at bit s = 2k + c up
// to e = 2(m + 1) + c, and the others of the run down one position (mask
// down).  With fw = the sum of 2^e - 2^s over the runs of copy c,
// ((x & st) + fw) & en carries every start bit to its end bit at once: the
// runs of one copy cover disjoint bit ranges, so no carry leaves its run.
struct SwapMasks {
    uint64_t keep, down, st[2], fw[2], en[2];
};

__device__ __forceinline__ SwapMasks swap_masks(const int *list, int n0, int n1, const uint64_t *down)
{
    SwapMasks m;
    m.down = down[0] | down[1];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        m.st[c] = m.fw[c] = m.en[c] = 0ull;
        const int n = c ? n1 : n0;
        for (int j = 0; j < n; ++j) {
            const int mv = list[32 * c + j];
            const uint64_t s = 1ull << (mv >> 8), e = 1ull << (mv & 0xff);
            m.st[c] |= s;
            m.en[c] |= e;
            m.fw[c] += e - s;
        }
    }
    m.keep = ~(m.down | m.st[0] | m.st[1]);
    return m;
}

__device__ __forceinline__ uint64_t swap_apply(const SwapMasks &m, uint64_t x)
{
    return (x & m.keep) | ((x & m.down) >> 2) | (((x & m.st[0]) + m.fw[0]) & m.en[0]) |
           (((x & m.st[1]) + m.fw[1]) & m.en[1]);
}

// Sum of a[j] over the 32 lanes, delivered to lane j (31 shuffles).
template <typename T>
__device__ __forceinline__ T transpose_reduce(T (&a)[32], int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            const T send = upper ? a[j] : a[j + s];
            const T keep = upper ? a[j + s] : a[j];
            a[j] = keep + __shfl_xor_sync(kFull, send, s);
        }
    }
    return a[0];
}

// Sum of a[j] over the 32 lanes, delivered to lanes 2j and 2j+1 (16 shuffles).
template <typename T>
__device__ __forceinline__ T transpose_reduce16(T (&a)[16], int lane)
{
#pragma unroll
    for (int s = 8; s >= 1; s >>= 1) {
        const bool upper = (lane & (2 * s)) != 0;
#pragma unroll
        for (int j = 0; j < s; ++j) {
            const T send = upper ? a[j] : a[j + s];
            const T keep = upper ? a[j + s] : a[j];
            a[j] = keep + __shfl_xor_sync(kFull, send, 2 * s);
        }
    }
    return a[0] + __shfl_xor_sync(kFull, a[0], 1);
}

template <typename T>
__device__ __forceinline__ T warp_sum_lane0(T v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Add one word to NPL bit-planes of per-bit counters (vertical counters).
template <int NPL>
__device__ __forceinline__ void vadd(uint32_t (&pl)[NPL], uint32_t w)
{
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const uint32_t c = pl[i] & w;
        pl[i] ^= w;
        w = c;
    }
}

// 32 x 32 bit-matrix transpose across a warp: lane j returns the word whose
// bit l is bit j of lane l's x.  Five butterfly stages; the one of stride s
// swaps the off-diagonal s x s blocks between lanes l and l ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                         : s == 2 ? 0x33333333u : 0x55555555u;     // bits whose index has bit s clear
        const uint32_t o = __shfl_xor_sync(kFull, x, s);
        x = (lane & s) ? ((x & ~m) | ((o >> s) & m)) : ((x & m) | ((o << s) & ~m));
    }
    return x;
}

// Full adder on whole words: per bit lane, a + b + c = s + 2 cy.
__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &cy)
{
    const uint32_t x = a ^ b;
    s = x ^ c;
    cy = (a & b) | (c & x);
}

// Per bit lane, the number of set bits among x[0..Z-1] (Z = 4, 6 or 8) as
// bit-planes c0..c3, by a carry-save adder tree (c2 = c3 = 0 where the
// count cannot reach them).
template <int Z>
__device__ __forceinline__ void csa_count(const uint32_t (&x)[Z], uint32_t &c0, uint32_t &c1, uint32_t &c2,
                                          uint32_t &c3)
{
    static_assert(Z == 4 || Z == 6 || Z == 8, "coordination 4, 6 or 8");
    uint32_t a, ca;
    full_add(x[0], x[1], x[2], a, ca);
    if constexpr (Z == 4) {
        c0 = a ^ x[3];
        const uint32_t h = a & x[3];
        c1 = ca ^ h;
        c2 = ca & h;
        c3 = 0u;
    } else if constexpr (Z == 6) {
        uint32_t b, cb;
        full_add(x[3], x[4], x[5], b, cb);
        c0 = a ^ b;
        full_add(ca, cb, a & b, c1, c2);
        c3 = 0u;
    } else {
        uint32_t b, cb, c, cc, t, e;
        full_add(x[3], x[4], x[5], b, cb);
        full_add(a, b, x[6], c, cc);
        c0 = c ^ x[7];
        const uint32_t h = c & x[7];             // weight 2: ca, cb, cc, h
        full_add(ca, cb, cc, t, e);
        c1 = t ^ h;
        const uint32_t f = t & h;                // weight 4: e, f
        c2 = e ^ f;
        c3 = e & f;
    }
}

// Add a number given as four bit-planes to NPL bit-planes of vertical
// counters (ripple carry over the planes).
template <int NPL>
__device__ __forceinline__ void vadd4(uint32_t (&pl)[NPL], uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3)
{
    const uint32_t in[4] = {c0, c1, c2, c3};
    uint32_t cy = 0u;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const uint32_t b = i < 4 ? in[i] : 0u;
        const uint32_t x = pl[i] ^ b;
        const uint32_t ncy = (pl[i] & b) | (cy & x);
        pl[i] = x ^ cy;
        cy = ncy;
    }
}

// Warp totals of vertical counters.  Every lane holds 32 counters as NPL
// bit-planes (bit b of plane i = binary digit i of counter b).  Five
// butterfly steps add the lanes' counters plane by plane (a ripple-carry
// adder on whole words, one plane wider per step), so every lane ends with
// the warp totals in NPL + 5 planes; lane b returns total b.
template <int NPL>
__device__ __forceinline__ int warp_vsum(const uint32_t (&pl)[NPL], int lane)
{
    uint32_t a[NPL + 5];
#pragma unroll
    for (int i = 0; i < NPL + 5; ++i) a[i] = i < NPL ? pl[i] : 0u;
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        uint32_t c = 0u;
#pragma unroll
        for (int i = 0; i < NPL + st; ++i) {
            const uint32_t o = __shfl_xor_sync(kFull, a[i], 16 >> st);
            const uint32_t x = a[i] ^ o;
            const uint32_t cn = (a[i] & o) | (c & x);
            a[i] = x ^ c;
            c = cn;
        }
        a[NPL + st] = c;
    }
    int v = 0;
#pragma unroll
    for (int i = 0; i < NPL + 5; ++i) v |= (int)((a[i] >> lane) & 1u) << i;
    return v;
}

// Per bit lane: u >= k, where u's binary digits are the bit-planes c3 c2 c1 c0
// and k (0..15) is the same for all lanes.
__device__ __forceinline__ uint32_t ge_bitsliced(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int k)
{
    const uint32_t c[4] = {c0, c1, c2, c3};
    uint32_t gt = 0u, eq = ~0u;
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        const uint32_t kb = 0u - (uint32_t)((k >> i) & 1);
        gt |= eq & c[i] & ~kb;
        eq &= ~(c[i] ^ kb);
    }
    return gt | eq;
}

}  // namespace
}  // namespace icm
