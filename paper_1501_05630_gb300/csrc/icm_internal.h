// Internal declarations shared by the host half (icm_api.cpp) and the device
// half (pt_icm.cu) of the library.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace icm {

constexpr int kMaxZ = 8;          // largest degree of the supported graphs (4D hypercubic)
constexpr int kMaxR = 64;         // replicas per instance (2 N_T, N_T <= 32)
constexpr int kMaxThreads = 128;  // threads per CTA of the fused kernel, shared-memory layout
constexpr int kMaxThreadsWide = 1024;  // threads per CTA of the fused kernel, global-resident layout
constexpr int kPlanes = 8;        // bit-planes of the vertical counters (counts < 256 per thread)

// Entries per replica of the +-J Metropolis threshold table, indexed by
// m = s_i h_i = 0..Z (m = 0: the probability-1/2 entry of diluted instances).
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr int thr_stride(int Z) { return Z > 7 ? 16 : 8; }

// Byte offsets into the fused kernel's dynamic shared memory.  In the
// global-resident ("wide") layout the spins, couplings, neighbour table,
// overlap masks and cluster words stay in global memory (size 0 here).
struct SmemLayout {
    int spins;      // uint32 [G][N]
    int nbr;        // uint16 [N][Z]   neighbour positions, padding = self
    int zdeg;       // uint8  [N]      degree (+-J only)
    int coup;       // float [N][Z] (Gaussian) or uint8 [N] bit d = (J < 0) (+-J)
    int E;          // float or int32 [R]
    int Epart;      // float or int32 [nwarps][max(R, 32)]
    int rtab;       // uint32 [R][thr_stride(Z)] thresholds (+-J) or float [R] -2 beta log2(e) (Gaussian)
    int icm_mask;   // uint32 [n_icm][NW] overlap masks per ICM pair
    int icm_C;      // uint32 [N]        cluster bits of every pair (bit 2k: pair k, bit 2k + 1: pair 16 + k)
    int swap_x;     // uint32 [2][32]
    int swap_list;  // int32 [2][32]   per run: (source bit << 8) | destination bit
    int swap_n;     // int32 [2]       runs per copy
    int swap_mask;  // uint64 [2]      bits moving down one slot, per copy
    int swap_tab;   // [3][32]         per neighbouring pair k: dbeta log2(e) (float), +-J table offset and length
    int flipw;      // uint32 [2]      step-2a reversal masks of the two words
    int icm_seed;   // int32 [32]      seed position per ICM pair (-1: none)
    int icm_esum;   // float or int32 [32]  E_a + E_b of each ICM pair before the move
    int cnt_n;      // int32 [32]
    int cnt_d;      // int32 [32]
    int accE;       // double [nT]
    int acc64;      // int64 [4][nT]  n, q2, pmin, d
    int nmeas;      // int64 [1]
    int icmst;      // uint64 [2]      this instance's cluster moves (pairs with n > 0) and growth scans
    int total;
};

// Everything the fused kernel reads or writes.  Device pointers.
struct KParams {
    int N, Nb, nT, R, G, Z, n_inst, n_icm, half, NW;
    int const_z;                  // degree when uniform (lattices), 0 = per-site table
    int wide;                     // 1: global-resident layout (instances too large for shared memory)
    int diluted;                  // 1: some instance has absent bonds (J = 0): per-instance tables below
    int scratch_words;            // wide layout: uint32 words of scratch per CTA (cluster words, masks)
    uint32_t *scratch;            // wide layout: [grid][scratch_words]
    int small_counts;             // per-thread observable counts fit 4 bit-planes
    // geometry, shared by all instances of the batch
    const uint16_t *nbr;          // [N][Z]
    const uint8_t *zdeg;          // [N]
    const uint16_t *pos2site;     // [N]
    // per instance, used when `diluted`: neighbour positions with absent bonds
    // replaced by the site itself, degree = bonds present, bonds present
    const uint16_t *nbr_inst;     // [n_inst][N][Z]
    const uint8_t *zdeg_inst;     // [n_inst][N]
    const int32_t *nb_inst;       // [n_inst]
    // per instance
    const float *Jd;              // [n_inst][N][Z]  (Gaussian)
    const uint8_t *Jb;            // [n_inst][N]     (+-J)
    uint32_t *spins;              // [n_inst][G][N]
    float *Ef;                    // [n_inst][R]     (Gaussian)
    int32_t *Ei;                  // [n_inst][R]     (+-J)
    uint32_t *tsweep;             // [n_inst]
    const uint32_t *inst_id;      // [n_inst]
    // temperature tables
    const uint32_t *thr_metro;    // [R][thr_stride(Z)]
    const float *b2l;             // [R]
    const double *beta;           // [nT]
    const float *dbeta_l2e;       // [nT-1] (beta_k - beta_{k+1}) log2(e)
    const uint32_t *thr_swap;     // concatenated per pair k
    const int32_t *swap_off;      // [nT-1]
    const int32_t *swap_len;      // [nT-1]
    // schedule
    int icm_every, swap_every, enable_2a, enable_metropolis, trace;
    long long t_meas;
    const long long *t_meas_inst;  // [n_inst] per-instance measurement start, or null (t_meas for all)
    const uint8_t *active;         // [n_inst] 0 = free slot (skipped), or null (all active)
    uint32_t seed_lo, seed_hi;
    // Philox4x32-10 key schedule of the seed: key[2i] = seed_lo + i 0x9E3779B9,
    // key[2i+1] = seed_hi + i 0xBB67AE85 (mod 2^32), the round keys i = 0..9;
    // read from the kernel parameters, so no round recomputes them
    uint32_t key[20];
    // observables
    double *accE;                 // [n_inst][nT]
    long long *acc64;             // [4][n_inst][nT]: n, (N-2n)^2, min(n,N-n), d
    unsigned long long *hist;     // [n_inst][nT][N+1]
    long long *n_meas;            // [n_inst]
    // ICM counters, accumulated over launches (cleared with the observables):
    // [n_inst][2] = pairs moved (n > 0 after step 2a), growth scans (passes over the sites)
    unsigned long long *icm_stats;
    // trace of the last sweep
    int32_t *tr_n_pre, *tr_flip2a, *tr_seed, *tr_csize;  // [n_inst][nT]
    float *tr_eb, *tr_ea;                                // [n_inst][nT]
    uint8_t *tr_swap;                                    // [n_inst][2][nT-1]
    uint32_t *tr_cmask;   // [n_inst][N][2] cluster words of the traced sweep, by position (NULL = off)
    // thread-block-cluster layout of 2D lattices: the own site that thread t
    // of a CTA grows as its j-th, at [4 t + j] (2 x 2 blocks of sites), or null
    const uint16_t *cl_order;     // [nls]
    SmemLayout sm;
};

// The shared group kernel (pt_icm.cu): one persistent CTA of kTeamThreads
// threads per SM runs tiles of instances of several batches (sizes) of one
// disorder kind and degree; a tile of batch c is `count` instances side by
// side, one team of team_threads[c] threads each (a divisor of
// kTeamThreads), each team with its own shared memory (KParams::sm of its
// batch, laid out for the team's width) and its own barrier.
constexpr int kTeamThreads = 896;   // 7 x 128: the threads of seven fused-kernel CTAs
constexpr int kTeamClasses = 8;     // batches per shared group
struct TeamItem {
    int cls, slot0, count;
};
struct TeamParams {
    KParams cls[kTeamClasses];
    int team_threads[kTeamClasses];
    const TeamItem *items;         // [n_items], in the order the CTAs take them
    int n_items;
    int *counters;                 // [2]: next item, CTAs done; zero between launches
    uint32_t key[20];              // Philox round keys of the common seed
};

// Host-built position tables of one lattice (see host_tables in icm_api.cpp).
struct HostTables {
    int N = 0, Nb = 0, Z = 0;
    std::vector<uint16_t> nbr;        // [N][Z]
    std::vector<uint16_t> pos2site;   // [N]
    std::vector<int32_t> edge_bond;   // [N][Z]
};
bool host_tables(int lattice, int L, HostTables &t);

SmemLayout smem_layout(int N, int Z, int R, int G, int nT, int n_icm, int nwarps, bool gauss, bool wide);

// Thread-block-cluster layout (cluster_icm.cu): one instance per cluster of
// K CTAs.  CTA r owns the positions [c half + r hs, c half + (r+1) hs) of
// each colour c (hs = half / K), stored as local index li = c hs + i; every
// per-site array has stride 4 bytes per local site, so the cluster-window
// address of a neighbour's spin word also locates its other words.  Byte
// offsets into each CTA's dynamic shared memory:
struct ClusterLayout {
    int K, hs, nls, NWl;   // CTAs, own sites per colour, own sites (2 hs), mask words (nls / 32)
    int s;          // uint32 [G][nls]   spin words
    int C;          // uint32 [nls]      cluster word: bit 2j = pair j, bit 2j + 1 = pair 16 + j
    int nb;         // uint32 [nls][Z]   cluster-window address of the neighbour's cluster word C
    int coup;       // float [nls][Z] (Gaussian) or uint8 [nls] sign bits (+-J)
    int zdeg;       // uint8 [nls]
    int E;          // float or int32 [R]       energies (the same in every CTA)
    int Epart;      // float or int32 [nwarps][max(R, 32)]
    int Esw;        // float or int32 [R]       this CTA's share of the sweep energies (read remotely)
    int Epair;      // float or int32 [32]      this CTA's share of the copy-a energies (read remotely)
    int rtab;       // thresholds (+-J) or -2 beta log2(e) (Gaussian), as in SmemLayout
    int mask;       // uint32 [32][NWl]         overlap masks of the ICM pairs (in the lab region)
    int lab;        // uint32 [max(ufg, 1)][nls] union-find parents: the cluster-window address of the
                    //                          parent's label word (a root holds its own address)
    int ufg;        // pairs per union-find group; 0 = growth by in-place scans (no labels)
    int sadr;       // uint32 [32]              cluster-window address of each pair's seed site (written remotely)
    int sroot;      // uint32 [8]               root of each group pair's seed
    int gord;       // uint16 [nls]             KParams::cl_order in shared memory, or -1 (site tid + j nth)
    int cntloc;     // int32 [2][32]            q = -1 sites per colour block and pair (read remotely)
    int flags;      // uint32 [2]               growth-round stamps, by round parity (written remotely)
    int seed;       // int32 [32]               1 = the pair moves
    int esum;       // float or int32 [32]
    int flipw;      // uint32 [2]
    int csz;        // int32 [32]               this CTA's cluster sites per pair (read remotely)
    int swap_x, swap_list, swap_n, swap_mask;   // as in SmemLayout
    int cnt_n, cnt_d;   // int32 [32]           this CTA's observable counts (read remotely)
    int accE, acc64, nmeas;                     // observables (rank 0)
    int icmst;      // uint64 [2]               cluster moves and growth scans of this instance (rank 0)
    int total;
};
// ufg: pairs per union-find group (1..kMaxUfGroup), or 0 for growth by scans.
constexpr int kMaxUfGroup = 8;
ClusterLayout cluster_layout(int N, int Z, int R, int G, int nT, int K, int nwarps, bool gauss, int ufg,
                             bool order);
cudaError_t launch_cluster(const KParams &P, const ClusterLayout &CL, bool gauss, int threads, int n_clusters,
                           uint32_t n_sweeps, cudaStream_t st);
cudaError_t cluster_occupancy(bool gauss, int Z, bool dil, int K, int threads, int smem, int *clusters);
int fused_threads(int N);
int fused_threads_wide(int N);
// uint32 words of per-CTA scratch of the wide layout (2 N cluster words, 32
// overlap-mask rows of NW words), rounded to 16 bytes.
int wide_scratch_words(int N);

// Host-callable launchers (pt_icm.cu).  Return a cudaError_t.
cudaError_t fused_occupancy(bool gauss, int Z, bool wide, int threads, int smem, int *ctas_per_sm);
cudaError_t launch_fused(const KParams &P, bool gauss, int threads, int grid, uint32_t n_sweeps,
                         cudaStream_t st);
cudaError_t launch_pack_spins(const int8_t *src, uint32_t *dst, const uint16_t *pos2site, int n_inst,
                              int R, int G, int N, cudaStream_t st);
cudaError_t launch_unpack_spins(const uint32_t *src, int8_t *dst, const uint16_t *pos2site, int n_inst,
                                int R, int G, int N, cudaStream_t st);
cudaError_t launch_expand_couplings(const void *bond_J, bool gauss, const int32_t *edge_bond, int n_inst,
                                    int N, int Z, int Nb, float *Jd, uint8_t *Jb, cudaStream_t st);
// Per-instance tables of a diluted batch from the bond couplings: neighbour
// positions (absent bond -> the site itself), degree and bonds present, and
// the number of invalid couplings (not finite; +-J outside -1, 0, +1) per
// instance in bad.  nb_inst and bad must be zero on entry (the kernel adds).
cudaError_t launch_expand_dilution(const void *bond_J, bool gauss, const int32_t *edge_bond, const uint16_t *nbr,
                                   int n_inst, int N, int Z, int Nb, uint16_t *nbr_inst, uint8_t *zdeg_inst,
                                   int32_t *nb_inst, int32_t *bad, cudaStream_t st);
cudaError_t launch_init_energies(const KParams &P, bool gauss, cudaStream_t st);
// The shared group kernel: grid persistent CTAs of kTeamThreads threads with
// `smem` bytes of dynamic shared memory each.
cudaError_t launch_team(const TeamParams &TP, bool gauss, int Z, int grid, int smem, uint32_t n_sweeps,
                        cudaStream_t st);
cudaError_t team_occupancy(bool gauss, int Z, int smem, int *ctas_per_sm);
cudaError_t launch_energies_to_double(const KParams &P, bool gauss, double *out, cudaStream_t st);

}  // namespace icm
