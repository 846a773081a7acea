// pt_icm.cu -- GB300 kernels for parallel tempering with isoenergetic
// cluster moves (the paper's "Isoenergetic cluster algorithm", steps 1, 2a,
// 2b, 3, plus the observables of "Benchmark model and observables").
//
// Design (one CTA per disorder instance, whole instance resident in shared
// memory for all sweeps of a launch; nothing here is a dense contraction, so
// no tensor cores are used):
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
//  * Steps 2a/2b: one warp per ICM temperature: overlap mask by warp ballot,
//    optional spin reversal of copy 1, seed by rank, breadth-first cluster
//    growth with shared-memory atomics, flip by atomic XOR, boundary energy.
//  * Step 3: one thread runs each copy's sequential PT pass on the energies;
//    accepted swaps are then applied to every site word as bit transpositions.
//  * Observables: vertical (bit-sliced) counters of q_i = -1 sites and of
//    bonds with q_i q_j = -1 for every pair at once.
#include "icm_internal.h"

#include <cstdio>
#include <type_traits>

namespace icm {

namespace {

constexpr uint32_t kFull = 0xffffffffu;

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds, multipliers
// 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ void philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                         uint32_t k1, uint32_t (&o)[4])
{
#pragma unroll
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

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
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

template <typename T>
__device__ __forceinline__ T warp_sum_lane0(T v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

// Add one word to 8 bit-planes of per-bit counters.
__device__ __forceinline__ void vadd(uint32_t (&pl)[kPlanes], uint32_t w)
{
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) {
        const uint32_t c = pl[i] & w;
        pl[i] ^= w;
        w = c;
    }
}

__device__ __forceinline__ int vget(const uint32_t (&pl)[kPlanes], int bit)
{
    int v = 0;
#pragma unroll
    for (int i = 0; i < kPlanes; ++i) v |= (int)((pl[i] >> bit) & 1u) << i;
    return v;
}

struct Sm {
    uint32_t *s;
    uint16_t *nbr;
    uint8_t *zdeg;
    uint16_t *pos2site;
    float *Jd;
    uint8_t *Jb;
    void *E;
    void *Epart;
    uint32_t *thr;
    float *b2l;
    uint32_t *mask;
    uint32_t *C;
    uint16_t *queue;
    int *tail;
    uint32_t *swap_x;
    int *swap_list;
    int *swap_n;
    int *cnt_n;
    int *cnt_d;
    double *accE;
    long long *acc64;
    long long *nmeas;
};

__device__ __forceinline__ Sm make_sm(unsigned char *base, const SmemLayout &L)
{
    Sm S;
    S.s = (uint32_t *)(base + L.spins);
    S.nbr = (uint16_t *)(base + L.nbr);
    S.zdeg = (uint8_t *)(base + L.zdeg);
    S.pos2site = (uint16_t *)(base + L.pos2site);
    S.Jd = (float *)(base + L.coup);
    S.Jb = (uint8_t *)(base + L.coup);
    S.E = base + L.E;
    S.Epart = base + L.Epart;
    S.thr = (uint32_t *)(base + L.rtab);
    S.b2l = (float *)(base + L.rtab);
    S.mask = (uint32_t *)(base + L.icm_mask);
    S.C = (uint32_t *)(base + L.icm_C);
    S.queue = (uint16_t *)(base + L.icm_queue);
    S.tail = (int *)(base + L.icm_tail);
    S.swap_x = (uint32_t *)(base + L.swap_x);
    S.swap_list = (int *)(base + L.swap_list);
    S.swap_n = (int *)(base + L.swap_n);
    S.cnt_n = (int *)(base + L.cnt_n);
    S.cnt_d = (int *)(base + L.cnt_d);
    S.accE = (double *)(base + L.accE);
    S.acc64 = (long long *)(base + L.acc64);
    S.nmeas = (long long *)(base + L.nmeas);
    return S;
}

// ---------------------------------------------------------------------------
// Step 1: one checkerboard half-sweep (colour COLOR) of every replica.
template <bool GAUSS, int Z, int COLOR>
__device__ __forceinline__ void half_sweep(const KParams &P, const Sm &S, uint32_t t, uint32_t inst)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int N = P.N, half = P.half, nth = blockDim.x;
    const int iters = (half + nth - 1) / nth;
    for (int g = 0; g < P.G; ++g) {
        const int nbits = min(32, P.R - 32 * g);
        uint32_t *sg = S.s + g * N;
        ET acc[32];
#pragma unroll
        for (int b = 0; b < 32; ++b) acc[b] = ET(0);
        for (int it = 0; it < iters; ++it) {
            const int j = threadIdx.x + it * nth;
            if (j >= half) continue;
            const int p = COLOR * half + j;
            const uint32_t sw = sg[p];
            const uint32_t site = S.pos2site[p];
            uint32_t flip = 0;
            uint32_t x[4] = {0u, 0u, 0u, 0u};
            if constexpr (GAUSS) {
                float Jv[Z];
                uint32_t nw[Z];
#pragma unroll
                for (int d = 0; d < Z; ++d) {
                    nw[d] = sg[S.nbr[p * Z + d]];
                    Jv[d] = S.Jd[p * Z + d];
                }
                const float *b2l = S.b2l + 32 * g;
#pragma unroll
                for (int b = 0; b < 32; ++b) {
                    if (b < nbits) {
                        if ((b & 3) == 0) philox10(site, t, (uint32_t)(32 * g + b) >> 2, inst, P.seed_lo, P.seed_hi, x);
                        float h = 0.f;
#pragma unroll
                        for (int d = 0; d < Z; ++d)
                            h += __uint_as_float(__float_as_uint(Jv[d]) ^ ((nw[d] << (31 - b)) & 0x80000000u));
                        const float sh = __uint_as_float(__float_as_uint(h) ^ ((sw << (31 - b)) & 0x80000000u));
                        const float u = __uint_as_float(0x3f800000u | (x[b & 3] >> 9)) - 1.0f;
                        const bool a = (sh <= 0.f) || (u < ex2_approx(b2l[b] * sh));
                        flip |= (uint32_t)a << b;
                        if (COLOR == 1) acc[b] += a ? sh : -sh;
                    }
                }
            } else {
                uint32_t c0 = 0, c1 = 0, c2 = 0;
                const uint32_t jb = S.Jb[p];
#pragma unroll
                for (int d = 0; d < Z; ++d) {
                    const uint32_t u = sw ^ sg[S.nbr[p * Z + d]] ^ (0u - ((jb >> d) & 1u));
                    const uint32_t t0 = c0 & u;
                    c0 ^= u;
                    const uint32_t t1 = c1 & t0;
                    c1 ^= t0;
                    c2 |= t1;
                }
                const int z = P.const_z ? P.const_z : (int)S.zdeg[p];
                // m = z - 2u <= 0  <=>  u >= ceil(z/2): always accepted
                flip = (z <= 4) ? (c2 | c1) : (c2 | (c1 & c0));
                const uint32_t *thr = S.thr + 32 * g * 8;
#pragma unroll
                for (int b = 0; b < 32; ++b) {
                    if (b < nbits) {
                        if ((b & 3) == 0) philox10(site, t, (uint32_t)(32 * g + b) >> 2, inst, P.seed_lo, P.seed_hi, x);
                        const int u = (int)(((c0 >> b) & 1u) | (((c1 >> b) & 1u) << 1) | (((c2 >> b) & 1u) << 2));
                        const int m = z - 2 * u;
                        const uint32_t th = thr[b * 8 + (m > 0 ? m : 0)];
                        flip |= (uint32_t)(x[b & 3] < th) << b;
                        if (COLOR == 1) acc[b] += ((flip >> b) & 1u) ? m : -m;
                    }
                }
            }
            sg[p] = sw ^ flip;
        }
        if (COLOR == 1) {
            const ET v = transpose_reduce(acc, lane);
            if (lane < nbits) ((ET *)S.Epart)[warp * P.R + 32 * g + lane] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Steps 2a and 2b for temperature position k, executed by one warp.
template <bool GAUSS, int Z>
__device__ void cluster_move(const KParams &P, const Sm &S, int k, uint32_t t, uint32_t inst, int slot,
                             bool trace)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int N = P.N, NW = P.NW;
    const int ra = 2 * k, g = ra >> 5, ba = ra & 31;
    uint32_t *sg = S.s + g * N;
    uint32_t *mask = S.mask + warp * NW;
    uint32_t *C = S.C + warp * NW;
    uint16_t *queue = S.queue + warp * N;
    int *tailp = S.tail + warp;
    ET *E = (ET *)S.E;

    // site overlap q_i = s_i^a s_i^b; bit set where q_i = -1
    int n = 0;
    for (int m = 0; m < NW; ++m) {
        const int p = 32 * m + lane;
        uint32_t bit = 0;
        if (p < N) {
            const uint32_t w = sg[p];
            bit = ((w >> ba) ^ (w >> (ba + 1))) & 1u;
        }
        const uint32_t word = __ballot_sync(kFull, bit);
        if (lane == 0) mask[m] = word;
        n += __popc(word);
    }
    const int n_pre = n;
    const float esum_before = (float)(E[ra] + E[ra + 1]);
    int flipped = 0;
    __syncwarp();
    if (P.enable_2a && 2 * n > N) {  // step 2a: reverse every spin of copy 1
        for (int p = lane; p < N; p += 32) atomicXor(&sg[p], 1u << (ba + 1));
        for (int m = lane; m < NW; m += 32) {
            const int rem = N - 32 * m;
            const uint32_t valid = rem >= 32 ? kFull : ((1u << rem) - 1u);
            mask[m] = ~mask[m] & valid;
        }
        n = N - n;
        flipped = 1;
    }
    __syncwarp();
    int seed = -1, csize = 0;
    if (n > 0) {  // step 2b: one Houdayer move
        if (lane == 0) {
            uint32_t x[4];
            philox10((uint32_t)k, t, 0u, (1u << 24) | inst, P.seed_lo, P.seed_hi, x);
            uint32_t rank = (uint32_t)(((uint64_t)x[0] * (uint32_t)n) >> 32);
            for (int m = 0; m < NW; ++m) {
                uint32_t w = mask[m];
                const uint32_t c = (uint32_t)__popc(w);
                if (rank < c) {
                    for (uint32_t r = 0; r < rank; ++r) w &= w - 1u;
                    seed = 32 * m + __ffs(w) - 1;
                    break;
                }
                rank -= c;
            }
        }
        seed = __shfl_sync(kFull, seed, 0);
        if (seed < 0) n = 0;   // unreachable when the mask holds n set bits
    }
    if (n > 0) {
        for (int m = lane; m < NW; m += 32) C[m] = 0u;
        __syncwarp();
        if (lane == 0) {
            C[seed >> 5] = 1u << (seed & 31);
            queue[0] = (uint16_t)seed;
            *tailp = 1;
        }
        __syncwarp();
        // breadth-first growth of the seed's component of {q = -1}
        int head = 0, tail = 1;
        while (head < tail) {
            for (int idx = head + lane; idx < tail; idx += 32) {
                const int p = queue[idx];
#pragma unroll
                for (int d = 0; d < Z; ++d) {
                    const int q = S.nbr[p * Z + d];
                    const uint32_t bq = 1u << (q & 31);
                    if (mask[q >> 5] & bq) {
                        const uint32_t old = atomicOr(&C[q >> 5], bq);
                        if (!(old & bq)) queue[atomicAdd(tailp, 1)] = (uint16_t)q;
                    }
                }
            }
            __syncwarp();
            head = tail;
            tail = *(volatile int *)tailp;
            __syncwarp();
        }
        csize = tail;
        // flip the cluster in both copies; boundary bonds give E_a's change
        ET delta = ET(0);
        for (int m = 0; m < NW; ++m) {
            const int p = 32 * m + lane;
            if (p < N && ((C[m] >> lane) & 1u)) {
                const uint32_t old = atomicXor(&sg[p], 3u << ba);
                const uint32_t ap = (old >> ba) & 1u;
#pragma unroll
                for (int d = 0; d < Z; ++d) {
                    const int q = S.nbr[p * Z + d];
                    if ((mask[q >> 5] >> (q & 31)) & 1u) continue;  // inside the domain (or padding)
                    const uint32_t aq = (sg[q] >> ba) & 1u;
                    if constexpr (GAUSS) {
                        const float J = S.Jd[p * Z + d];
                        delta += (ap ^ aq) ? -2.f * J : 2.f * J;
                    } else {
                        const uint32_t jneg = (S.Jb[p] >> d) & 1u;
                        delta += (jneg ^ ap ^ aq) ? -2 : 2;
                    }
                }
            }
        }
        delta = warp_sum_lane0(delta);
        if (lane == 0) {
            E[ra] += delta;
            E[ra + 1] -= delta;
        }
    }
    __syncwarp();
    if (trace && lane == 0) {
        const size_t o = (size_t)slot * P.nT + k;
        P.tr_n_pre[o] = n_pre;
        P.tr_flip2a[o] = flipped;
        P.tr_seed[o] = seed >= 0 ? (int)S.pos2site[seed] : -1;
        P.tr_csize[o] = csize;
        P.tr_eb[o] = esum_before;
        P.tr_ea[o] = (float)(E[ra] + E[ra + 1]);
    }
}

// ---------------------------------------------------------------------------
// Step 3: sequential PT pass per copy, then the configuration swaps.
template <bool GAUSS>
__device__ void pt_pass(const KParams &P, const Sm &S, uint32_t t, uint32_t inst, int slot, bool trace)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int nT = P.nT, np = nT - 1, N = P.N;
    for (int i = threadIdx.x; i < 2 * np; i += blockDim.x) {
        const int c = i / np, k = i % np;
        uint32_t x[4];
        philox10((uint32_t)k, t, (uint32_t)c, (2u << 24) | inst, P.seed_lo, P.seed_hi, x);
        S.swap_x[c * 32 + k] = x[0];
    }
    __syncthreads();
    const int second = blockDim.x > 32 ? 32 : 1;   // copy 1 runs on another warp when there is one
    if (threadIdx.x == 0 || threadIdx.x == second) {
        ET *E = (ET *)S.E;
        const int c = threadIdx.x == 0 ? 0 : 1;
        {
            int ns = 0;
            for (int k = 0; k < np; ++k) {
                const int ra = 2 * k + c, rb = ra + 2;
                const ET ek = E[ra], ek1 = E[rb];
                const uint32_t x = S.swap_x[c * 32 + k];
                bool acc;
                if constexpr (GAUSS) {
                    // log2(e) (beta_k - beta_{k+1}) (E_k - E_{k+1}); accept iff >= 0 or u < 2^delta
                    const float delta = P.dbeta_l2e[k] * (ek - ek1);
                    acc = (delta >= 0.f) || ((float)(x >> 8) * (1.0f / 16777216.0f) < ex2_approx(delta));
                } else {
                    const int dE = ek - ek1;
                    if (dE >= 0) {
                        acc = true;
                    } else {
                        const int d = (-dE) >> 1;
                        acc = d >= 1 && d <= P.swap_len[k] && x < P.thr_swap[P.swap_off[k] + d - 1];
                    }
                }
                if (acc) {
                    E[ra] = ek1;
                    E[rb] = ek;
                    S.swap_list[c * 32 + ns++] = k;
                }
                if (trace) P.tr_swap[((size_t)slot * 2 + c) * np + k] = (uint8_t)acc;
            }
            S.swap_n[c] = ns;
        }
    }
    __syncthreads();
    const int n0 = S.swap_n[0], n1 = S.swap_n[1];
    if (n0 + n1 > 0) {
        const bool two = P.G > 1;
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            uint32_t w0 = S.s[p], w1 = two ? S.s[N + p] : 0u;
            for (int c = 0; c < 2; ++c) {
                const int nc = c ? n1 : n0;
                for (int j = 0; j < nc; ++j) {
                    const int r1 = 2 * S.swap_list[c * 32 + j] + c, r2 = r1 + 2;
                    const uint32_t b1 = (r1 < 32 ? (w0 >> r1) : (w1 >> (r1 - 32))) & 1u;
                    const uint32_t b2 = (r2 < 32 ? (w0 >> r2) : (w1 >> (r2 - 32))) & 1u;
                    const uint32_t dlt = b1 ^ b2;
                    if (r1 < 32) w0 ^= dlt << r1; else w1 ^= dlt << (r1 - 32);
                    if (r2 < 32) w0 ^= dlt << r2; else w1 ^= dlt << (r2 - 32);
                }
            }
            S.s[p] = w0;
            if (two) S.s[N + p] = w1;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Observables: per pair k, n = #{q_i = -1} and d = #{bonds, q_i q_j = -1}.
template <bool GAUSS, int Z>
__device__ void measure(const KParams &P, const Sm &S, int slot)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    const int lane = threadIdx.x & 31;
    const int N = P.N, half = P.half, nT = P.nT;
    for (int g = 0; g < P.G; ++g) {
        const int npair = min(16, nT - 16 * g);
        const uint32_t *sg = S.s + g * N;
        uint32_t pn[kPlanes], pd[kPlanes];
#pragma unroll
        for (int i = 0; i < kPlanes; ++i) pn[i] = pd[i] = 0u;
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            const uint32_t w = sg[p];
            vadd(pn, (w ^ (w >> 1)) & 0x55555555u);
        }
        for (int p = half + threadIdx.x; p < N; p += blockDim.x) {
            const uint32_t w = sg[p];
            const uint32_t qp = (w ^ (w >> 1)) & 0x55555555u;
#pragma unroll
            for (int d = 0; d < Z; ++d) {
                const int q = S.nbr[p * Z + d];
                if (q == p) continue;
                const uint32_t wq = sg[q];
                vadd(pd, qp ^ ((wq ^ (wq >> 1)) & 0x55555555u));
            }
        }
        for (int j = 0; j < npair; ++j) {
            const int cn = __reduce_add_sync(kFull, vget(pn, 2 * j));
            const int cd = __reduce_add_sync(kFull, vget(pd, 2 * j));
            if (lane == 0) {
                atomicAdd(&S.cnt_n[16 * g + j], cn);
                atomicAdd(&S.cnt_d[16 * g + j], cd);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nT; k += blockDim.x) {
        const long long n = S.cnt_n[k], d = S.cnt_d[k];
        S.cnt_n[k] = 0;
        S.cnt_d[k] = 0;
        const ET *E = (const ET *)S.E;
        S.accE[k] += (double)E[2 * k] + (double)E[2 * k + 1];
        S.acc64[0 * nT + k] += n;
        S.acc64[1 * nT + k] += (N - 2 * n) * (N - 2 * n);
        S.acc64[2 * nT + k] += n < N - n ? n : N - n;
        S.acc64[3 * nT + k] += d;
        atomicAdd(&P.hist[((size_t)slot * nT + k) * (N + 1) + n], 1ull);
    }
    if (threadIdx.x == 0) S.nmeas[0] += 1;
    __syncthreads();
}

// ---------------------------------------------------------------------------
template <bool GAUSS, int Z>
__global__ void __launch_bounds__(kMaxThreads, 4) fused_kernel(const KParams P, uint32_t n_sweeps)
{
    using ET = typename std::conditional<GAUSS, float, int>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const Sm S = make_sm(smem, P.sm);
    const int tid = threadIdx.x, nth = blockDim.x, nwarps = nth >> 5, warp = tid >> 5;
    const int N = P.N, R = P.R, nT = P.nT, G = P.G;

    for (int i = tid; i < N * Z; i += nth) S.nbr[i] = P.nbr[i];
    for (int i = tid; i < N; i += nth) {
        S.pos2site[i] = P.pos2site[i];
        if (!GAUSS && !P.const_z) S.zdeg[i] = P.zdeg[i];
    }
    if constexpr (GAUSS) {
        for (int r = tid; r < R; r += nth) S.b2l[r] = P.b2l[r];
    } else {
        for (int i = tid; i < R * 8; i += nth) S.thr[i] = P.thr_metro[i];
    }
    if (tid < 32) {
        S.cnt_n[tid] = 0;
        S.cnt_d[tid] = 0;
    }

    for (int slot = blockIdx.x; slot < P.n_inst; slot += gridDim.x) {
        const uint32_t *gs = P.spins + (size_t)slot * G * N;
        for (int i = tid; i < G * N; i += nth) S.s[i] = gs[i];
        if constexpr (GAUSS) {
            const float4 *src = (const float4 *)(P.Jd + (size_t)slot * N * Z);
            float4 *dst = (float4 *)S.Jd;
            for (int i = tid; i < (N * Z) / 4; i += nth) dst[i] = src[i];
            for (int r = tid; r < R; r += nth) ((float *)S.E)[r] = P.Ef[(size_t)slot * R + r];
        } else {
            for (int i = tid; i < N; i += nth) S.Jb[i] = P.Jb[(size_t)slot * N + i];
            for (int r = tid; r < R; r += nth) ((int *)S.E)[r] = P.Ei[(size_t)slot * R + r];
        }
        for (int k = tid; k < nT; k += nth) {
            S.accE[k] = P.accE[(size_t)slot * nT + k];
            for (int a = 0; a < 4; ++a) S.acc64[a * nT + k] = P.acc64[((size_t)a * P.n_inst + slot) * nT + k];
        }
        if (tid == 0) S.nmeas[0] = P.n_meas[slot];
        const uint32_t inst = P.inst_id[slot];
        uint32_t t = P.tsweep[slot];
        __syncthreads();

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
                __syncthreads();
            }
            if (P.enable_metropolis) {  // step 1
                half_sweep<GAUSS, Z, 0>(P, S, t, inst);
                __syncthreads();
                half_sweep<GAUSS, Z, 1>(P, S, t, inst);
                __syncthreads();
                for (int r = tid; r < R; r += nth) {
                    ET e = ET(0);
                    for (int w = 0; w < nwarps; ++w) e += ((const ET *)S.Epart)[w * R + r];
                    ((ET *)S.E)[r] = e;
                }
                __syncthreads();
            }
            if (P.icm_every > 0 && t % (uint32_t)P.icm_every == 0 && P.n_icm > 0) {  // steps 2a, 2b
                for (int k = warp; k < P.n_icm; k += nwarps) cluster_move<GAUSS, Z>(P, S, k, t, inst, slot, trace);
                __syncthreads();
            }
            if (P.swap_every > 0 && t % (uint32_t)P.swap_every == 0 && nT > 1)  // step 3
                pt_pass<GAUSS>(P, S, t, inst, slot, trace);
            if ((long long)t >= P.t_meas) measure<GAUSS, Z>(P, S, slot);
        }

        uint32_t *gd = P.spins + (size_t)slot * G * N;
        for (int i = tid; i < G * N; i += nth) gd[i] = S.s[i];
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
        }
        __syncthreads();
    }
}

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
        for (int r = 0; r < P.R; ++r) {
            const uint32_t *sg = s + (r >> 5) * N;
            const int b = r & 31;
            ET acc = ET(0);
            for (int p = half + threadIdx.x; p < N; p += blockDim.x) {
                const int si = ((sg[p] >> b) & 1u) ? -1 : 1;
                for (int d = 0; d < Z; ++d) {
                    const int q = P.nbr[p * Z + d];
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

inline int grid_for(size_t n, int threads)
{
    size_t g = (n + threads - 1) / threads;
    if (g > 152 * 16) g = 152 * 16;
    return g > 0 ? (int)g : 1;
}

template <bool GAUSS, int Z>
cudaError_t launch_fused_t(const KParams &P, int threads, int grid, uint32_t n_sweeps, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<GAUSS, Z>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         P.sm.total);
    if (e != cudaSuccess) return e;
    fused_kernel<GAUSS, Z><<<grid, threads, P.sm.total, st>>>(P, n_sweeps);
    return cudaGetLastError();
}

template <bool GAUSS, int Z>
cudaError_t occupancy_t(int threads, int smem, int *ctas)
{
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<GAUSS, Z>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, fused_kernel<GAUSS, Z>, threads, smem);
}

}  // namespace

// ---------------------------------------------------------------------------
static int align_up(int v, int a) { return (v + a - 1) / a * a; }

SmemLayout smem_layout(int N, int Z, int R, int G, int nT, int nwarps, bool gauss)
{
    SmemLayout L{};
    const int NW = (N + 31) / 32;
    int o = 0;
    auto take = [&](int bytes, int align) {
        o = align_up(o, align);
        const int at = o;
        o += bytes;
        return at;
    };
    L.coup = take(gauss ? N * Z * 4 : N, 16);
    L.spins = take(G * N * 4, 16);
    L.nbr = take(N * Z * 2, 16);
    L.zdeg = take(N, 16);
    L.pos2site = take(N * 2, 16);
    L.E = take(R * 4, 16);
    L.Epart = take(nwarps * R * 4, 16);
    L.rtab = take(gauss ? R * 4 : R * 8 * 4, 16);
    L.icm_mask = take(nwarps * NW * 4, 16);
    L.icm_C = take(nwarps * NW * 4, 16);
    L.icm_queue = take(nwarps * N * 2, 16);
    L.icm_tail = take(nwarps * 4, 16);
    L.swap_x = take(2 * 32 * 4, 16);
    L.swap_list = take(2 * 32 * 4, 16);
    L.swap_n = take(2 * 4, 16);
    L.cnt_n = take(32 * 4, 16);
    L.cnt_d = take(32 * 4, 16);
    L.accE = take(nT * 8, 16);
    L.acc64 = take(4 * nT * 8, 16);
    L.nmeas = take(8, 16);
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

cudaError_t fused_occupancy(bool gauss, int Z, int threads, int smem, int *ctas)
{
    if (gauss) return Z == 4 ? occupancy_t<true, 4>(threads, smem, ctas) : occupancy_t<true, 6>(threads, smem, ctas);
    return Z == 4 ? occupancy_t<false, 4>(threads, smem, ctas) : occupancy_t<false, 6>(threads, smem, ctas);
}

cudaError_t launch_fused(const KParams &P, bool gauss, int threads, int grid, uint32_t n_sweeps, cudaStream_t st)
{
    if (gauss)
        return P.Z == 4 ? launch_fused_t<true, 4>(P, threads, grid, n_sweeps, st)
                        : launch_fused_t<true, 6>(P, threads, grid, n_sweeps, st);
    return P.Z == 4 ? launch_fused_t<false, 4>(P, threads, grid, n_sweeps, st)
                    : launch_fused_t<false, 6>(P, threads, grid, n_sweeps, st);
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

cudaError_t launch_init_energies(const KParams &P, bool gauss, cudaStream_t st)
{
    const int grid = P.n_inst < 152 * 8 ? P.n_inst : 152 * 8;
    if (gauss) {
        if (P.Z == 4) init_energies_kernel<true, 4><<<grid, kMaxThreads, 0, st>>>(P);
        else init_energies_kernel<true, 6><<<grid, kMaxThreads, 0, st>>>(P);
    } else {
        if (P.Z == 4) init_energies_kernel<false, 4><<<grid, kMaxThreads, 0, st>>>(P);
        else init_energies_kernel<false, 6><<<grid, kMaxThreads, 0, st>>>(P);
    }
    return cudaGetLastError();
}

cudaError_t launch_energies_to_double(const KParams &P, bool gauss, double *out, cudaStream_t st)
{
    const size_t n = (size_t)P.n_inst * P.R;
    energies_to_double_kernel<<<grid_for(n, 256), 256, 0, st>>>(P.Ef, P.Ei, gauss ? 1 : 0, n, out);
    return cudaGetLastError();
}

}  // namespace icm
