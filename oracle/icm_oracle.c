/*
 * icm_oracle.c -- plain, slow, single-threaded CPU oracle for parallel
 * tempering (PT) with isoenergetic cluster moves (ICM) on Ising spin glasses.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA library against an
 * independent, obviously correct restatement of the method.  It shares no
 * source, header, table or helper with the CUDA library.
 *
 * Arithmetic: fp64 for Gaussian couplings; exact integers (held in doubles
 * and int64) for +-J couplings.  Every step follows the paper in its order:
 *
 *   Model and observables      -- "Benchmark model and observables", Eq. 1
 *   Simulation step            -- "Isoenergetic cluster algorithm", steps
 *                                 1, 2a, 2b, 3 (with the Houdayer move of the
 *                                 "Reminder: Houdayer cluster algorithm")
 *
 * Readings of points the paper leaves open (the library implements the same
 * readings; they are listed once more in the design notes):
 *   R1 H = -sum over bonds <ij> (each bond once) of J_ij s_i s_j.
 *   R2 Site order of a sweep: all sites of colour 0, then all of colour 1;
 *      replicas independent.  Same-colour sites share no bond, so the order
 *      inside a colour class does not change the result.
 *   R3 Random draws come from Philox4x32-10 (Salmon et al., SC'11), key =
 *      (seed lo32, seed hi32), counters:
 *         Metropolis (t, r, i): ctr {i, t, r>>2, inst}          word r&3
 *         ICM seed   (t, k)   : ctr {k, t, 0,    (1<<24)|inst}  word 0
 *         PT swap    (t, c, k): ctr {k, t, c,    (2<<24)|inst}  word 0
 *      t = sweep index, r = 2k+c = temperature position k, copy c.
 *   R4 +-J Metropolis: m = s_i h_i (Delta E = 2m); accept iff m <= 0 or
 *      x < floor(exp((-2m) * beta) * 2^32).
 *      Gaussian: accept iff dE <= 0 or (x>>8)*2^-24 < exp(-beta dE).
 *   R5 Step 2a flips copy 1 when n_neg > N/2 (strict).
 *   R6 ICM at every k with T_k <= T_icm, ascending k.  Seed = the rank-th
 *      site with q_i = -1, rank = floor(x * n_neg / 2^32), sites ordered by
 *      (colour, index).  n_neg = 0: no move.
 *   R7 Cluster = connected component of the seed in the subgraph of the
 *      interaction graph induced by {i : q_i = -1}.
 *   R8 PT pass: for each copy c, k = 0 .. N_T-2 ascending, swap the
 *      configurations at k and k+1 with probability
 *      min(1, exp((beta_k - beta_{k+1})(E_k - E_{k+1}))).
 *      +-J: accept iff E_k >= E_{k+1} or
 *           x < floor(exp((-2d) * (beta_k - beta_{k+1})) * 2^32),
 *           d = (E_{k+1} - E_k)/2.
 *      Gaussian: accept iff Delta >= 0 or (x>>8)*2^-24 < exp(Delta).
 *   R9 Measurement after the PT pass when t >= t_meas.
 *  R10 Dilution (the remedy the introduction cites for the cluster move in
 *      three dimensions): a bond with J_ij = 0 is absent from the lattice.
 *      It is no edge of the interaction graph of R7, and it is not counted
 *      in the link overlap q_l (a sum over the bonds of the lattice, with
 *      N_b = the number of bonds present).  It adds nothing to H or to a
 *      local field either way.
 *  R11 On a diluted instance (some J_ij = 0) a Metropolis proposal with
 *      Delta E = 0 is accepted with probability 1/2 (x < 2^31) instead of
 *      always.  Dilution creates sites of degree 0, 1 and 2; there the
 *      checkerboard sweep with deterministic zero-energy flips is not
 *      ergodic (on a ring of four sites, s0 != s2 and s1 != s3 flips every
 *      site every half-sweep forever).  The acceptance ratio
 *      a(dE)/a(-dE) = exp(-beta dE) still holds, so the chain keeps the
 *      Boltzmann distribution.  Undiluted instances keep R4 unchanged.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_SQUARE 0
#define ORC_CUBIC 1
#define ORC_CHIMERA 2
#define ORC_HYPERCUBIC4 3

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
 * 32x32->64 multiplies with the Weyl-sequence key schedule.                 */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static uint32_t draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int word)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ------------------------------------------------------------------------ */
/* Geometry.  2D: site i = x + L y, bond b = 2i + d to the +x / +y neighbour.
 * 3D: i = x + L(y + L z), b = 3i + d.  Both periodic; colour (x+y[+z]) mod 2.
 * Chimera C_M: i = 8(rM + c) + 4h + k (h = shore).  In-cell K_{4,4}:
 * b = 16 cell + 4 k0 + k1 joins (h=0,k0)-(h=1,k1); then the vertical bonds
 * (r,c,0,k)-(r+1,c,0,k), b = 16M^2 + 4(rM + c) + k; then the horizontal
 * bonds (r,c,1,k)-(r,c+1,1,k), b = 16M^2 + 4M(M-1) + 4(r(M-1) + c) + k.
 * Open boundary; colour (r + c + h) mod 2.
 * 4D hypercubic: i = x + L(y + L(z + L w)), b = 4i + d, periodic, colour
 * (x+y+z+w) mod 2.                                                         */
int orc_geometry_sizes(int kind, int L, int32_t *N, int32_t *Nb)
{
    if (L < 1) return -1;
    if (kind == ORC_SQUARE) { *N = L * L; *Nb = 2 * L * L; return 0; }
    if (kind == ORC_CUBIC) { *N = L * L * L; *Nb = 3 * L * L * L; return 0; }
    if (kind == ORC_CHIMERA) { *N = 8 * L * L; *Nb = 16 * L * L + 8 * L * (L - 1); return 0; }
    if (kind == ORC_HYPERCUBIC4) { *N = L * L * L * L; *Nb = 4 * L * L * L * L; return 0; }
    return -1;
}

int orc_geometry(int kind, int L, int32_t *bi, int32_t *bj, uint8_t *color)
{
    int32_t N, Nb;
    if (orc_geometry_sizes(kind, L, &N, &Nb)) return -1;
    if (kind == ORC_SQUARE) {
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int i = x + L * y;
                color[i] = (uint8_t)((x + y) % 2);
                bi[2 * i + 0] = i; bj[2 * i + 0] = (x + 1) % L + L * y;
                bi[2 * i + 1] = i; bj[2 * i + 1] = x + L * ((y + 1) % L);
            }
    } else if (kind == ORC_CUBIC) {
        for (int z = 0; z < L; ++z)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    int i = x + L * (y + L * z);
                    color[i] = (uint8_t)((x + y + z) % 2);
                    bi[3 * i + 0] = i; bj[3 * i + 0] = (x + 1) % L + L * (y + L * z);
                    bi[3 * i + 1] = i; bj[3 * i + 1] = x + L * ((y + 1) % L + L * z);
                    bi[3 * i + 2] = i; bj[3 * i + 2] = x + L * (y + L * ((z + 1) % L));
                }
    } else if (kind == ORC_HYPERCUBIC4) {
        for (int w = 0; w < L; ++w)
            for (int z = 0; z < L; ++z)
                for (int y = 0; y < L; ++y)
                    for (int x = 0; x < L; ++x) {
                        int i = x + L * (y + L * (z + L * w));
                        color[i] = (uint8_t)((x + y + z + w) % 2);
                        bi[4 * i + 0] = i; bj[4 * i + 0] = (x + 1) % L + L * (y + L * (z + L * w));
                        bi[4 * i + 1] = i; bj[4 * i + 1] = x + L * ((y + 1) % L + L * (z + L * w));
                        bi[4 * i + 2] = i; bj[4 * i + 2] = x + L * (y + L * ((z + 1) % L + L * w));
                        bi[4 * i + 3] = i; bj[4 * i + 3] = x + L * (y + L * (z + L * ((w + 1) % L)));
                    }
    } else {
        int M = L;
        for (int r = 0; r < M; ++r)
            for (int c = 0; c < M; ++c)
                for (int h = 0; h < 2; ++h)
                    for (int k = 0; k < 4; ++k)
                        color[8 * (r * M + c) + 4 * h + k] = (uint8_t)((r + c + h) % 2);
        int b = 0;
        for (int cell = 0; cell < M * M; ++cell)
            for (int k0 = 0; k0 < 4; ++k0)
                for (int k1 = 0; k1 < 4; ++k1) {
                    bi[b] = 8 * cell + k0; bj[b] = 8 * cell + 4 + k1; ++b;
                }
        for (int r = 0; r + 1 < M; ++r)
            for (int c = 0; c < M; ++c)
                for (int k = 0; k < 4; ++k) {
                    bi[b] = 8 * (r * M + c) + k; bj[b] = 8 * ((r + 1) * M + c) + k; ++b;
                }
        for (int r = 0; r < M; ++r)
            for (int c = 0; c + 1 < M; ++c)
                for (int k = 0; k < 4; ++k) {
                    bi[b] = 8 * (r * M + c) + 4 + k; bj[b] = 8 * (r * M + c + 1) + 4 + k; ++b;
                }
        if (b != Nb) return -2;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t N, Nb, nT, pm;        /* pm = 1: +-J (integer arithmetic); 0: Gaussian */
    const int32_t *bi, *bj;       /* bond endpoints [Nb] */
    const double *J;              /* couplings [Nb] (exactly +-1 when pm) */
    const uint8_t *color;         /* [N] */
    const double *T;              /* [nT], ascending */
    double T_icm;                 /* ICM at every k with T_k <= T_icm */
    int32_t icm_every, swap_every, enable_2a, enable_metropolis;
    int64_t t_meas;
    uint64_t seed;
    uint32_t inst, pad2_;
} orc_problem;

typedef struct {
    int8_t *s;                    /* [2 nT][N], +-1, row r = 2k + c */
    double *E;                    /* [2 nT] energies at the end of the last sweep */
    double *accE;                 /* [nT] sum of E_{2k} + E_{2k+1} */
    int64_t *acc_n;               /* [nT] sum of n = #{q_i = -1} */
    int64_t *acc_q2;              /* [nT] sum of (N - 2n)^2 */
    int64_t *acc_pmin;            /* [nT] sum of min(n, N - n) */
    int64_t *acc_d;               /* [nT] sum of d = #{bonds present with q_i q_j = -1} */
    int64_t *hist;                /* [nT][N+1] histogram of n */
    int64_t *n_meas;              /* [1] */
    uint32_t t;                   /* sweep counter */
    uint32_t pad_;
} orc_state;

typedef struct {                  /* the last sweep only */
    int32_t *n_pre;               /* [nT] n before step 2a, -1 if no ICM at k */
    int32_t *flip2a;              /* [nT] 1 if step 2a flipped copy 1 */
    int32_t *seed_site;           /* [nT] seed site index, -1 if none */
    int32_t *csize;               /* [nT] cluster size */
    double *esum_before;          /* [nT] E_a + E_b before the cluster move */
    double *esum_after;           /* [nT] E_a + E_b after the cluster move */
    uint8_t *swap_acc;            /* [2][nT-1] */
    uint8_t *cmask;               /* [nT][N] 1 = site in the moved cluster at k, or NULL */
} orc_trace;

/* Adjacency built from the bond list: for every site its incident bonds.
 * With couplings given, bonds with J = 0 are absent (R10).                 */
typedef struct {
    int32_t *start;   /* [N+1] */
    int32_t *nbr;     /* [2 Nb] */
    int32_t *bond;    /* [2 Nb] */
} adjacency;

static int build_adjacency(const orc_problem *P, adjacency *A)
{
    int N = P->N, Nb = P->Nb;
    A->start = calloc((size_t)N + 1, sizeof(int32_t));
    A->nbr = malloc(sizeof(int32_t) * 2 * (size_t)(Nb > 0 ? Nb : 1));
    A->bond = malloc(sizeof(int32_t) * 2 * (size_t)(Nb > 0 ? Nb : 1));
    if (!A->start || !A->nbr || !A->bond) return -1;
    for (int b = 0; b < Nb; ++b) {
        if (P->J && P->J[b] == 0.0) continue;
        A->start[P->bi[b] + 1]++;
        A->start[P->bj[b] + 1]++;
    }
    for (int i = 0; i < N; ++i) A->start[i + 1] += A->start[i];
    int32_t *fill = calloc((size_t)N, sizeof(int32_t));
    if (!fill) return -1;
    for (int b = 0; b < Nb; ++b) {
        if (P->J && P->J[b] == 0.0) continue;
        int i = P->bi[b], j = P->bj[b];
        int pi = A->start[i] + fill[i]++, pj = A->start[j] + fill[j]++;
        A->nbr[pi] = j; A->bond[pi] = b;
        A->nbr[pj] = i; A->bond[pj] = b;
    }
    free(fill);
    return 0;
}

static void free_adjacency(adjacency *A) { free(A->start); free(A->nbr); free(A->bond); }

/* H = -sum_<ij> J_ij s_i s_j over the bond list (R1). */
static double energy(const orc_problem *P, const int8_t *s)
{
    double e = 0.0;
    for (int b = 0; b < P->Nb; ++b) e -= P->J[b] * (double)s[P->bi[b]] * (double)s[P->bj[b]];
    return e;
}

/* floor(exp(a) * 2^32), at most 2^32 - 1; a <= 0. */
static uint64_t threshold(double a)
{
    double v = floor(exp(a) * 4294967296.0);
    if (v >= 4294967295.0) return 4294967295ull;
    if (v < 0.0) return 0;
    return (uint64_t)v;
}

static double unit24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* Step 1: one Metropolis sweep of every replica (R2, R4, R11).  `tie` = 1 on
 * a diluted instance: a zero-energy proposal is accepted with probability 1/2. */
static void metropolis_sweep(const orc_problem *P, orc_state *S, const adjacency *A, int tie)
{
    int N = P->N, R = 2 * P->nT;
    for (int col = 0; col < 2; ++col)
        for (int r = 0; r < R; ++r) {
            double beta = 1.0 / P->T[r / 2];
            int8_t *s = S->s + (size_t)r * N;
            for (int i = 0; i < N; ++i) {
                if (P->color[i] != col) continue;
                double h = 0.0;
                for (int e = A->start[i]; e < A->start[i + 1]; ++e)
                    h += P->J[A->bond[e]] * (double)s[A->nbr[e]];
                uint32_t x = draw(P->seed, (uint32_t)i, S->t, (uint32_t)(r >> 2), P->inst, r & 3);
                int accept;
                if (P->pm) {
                    long m = (long)s[i] * lrint(h);
                    if (m < 0) accept = 1;
                    else if (m == 0) accept = tie ? (x < 0x80000000u) : 1;
                    else accept = (uint64_t)x < threshold((double)(-2 * m) * beta);
                } else {
                    double dE = 2.0 * (double)s[i] * h;
                    if (dE < 0.0) accept = 1;
                    else if (dE == 0.0) accept = tie ? (unit24(x) < 0.5) : 1;
                    else accept = unit24(x) < exp(-beta * dE);
                }
                if (accept) s[i] = (int8_t)(-s[i]);
            }
        }
}

/* Steps 2a and 2b at temperature position k (R5, R6, R7). */
static void cluster_move(const orc_problem *P, orc_state *S, const adjacency *A, int k,
                         const int32_t *site_order, int32_t *queue, uint8_t *in_cluster,
                         const orc_trace *tr)
{
    int N = P->N;
    int8_t *sa = S->s + (size_t)(2 * k) * N;
    int8_t *sb = S->s + (size_t)(2 * k + 1) * N;
    int n = 0;
    for (int i = 0; i < N; ++i) n += (sa[i] * sb[i] == -1);
    if (tr) { tr->n_pre[k] = n; tr->flip2a[k] = 0; tr->seed_site[k] = -1; tr->csize[k] = 0; }
    if (tr) tr->esum_before[k] = energy(P, sa) + energy(P, sb);
    if (P->enable_2a && 2 * n > N) {            /* step 2a: spin-reversal of copy 1 */
        for (int i = 0; i < N; ++i) sb[i] = (int8_t)(-sb[i]);
        n = N - n;
        if (tr) tr->flip2a[k] = 1;
    }
    if (n > 0) {                                 /* step 2b: one Houdayer move */
        uint32_t x = draw(P->seed, (uint32_t)k, S->t, 0u, (1u << 24) | P->inst, 0);
        uint32_t rank = (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32);
        int seed_site = -1;
        uint32_t seen = 0;
        for (int o = 0; o < N; ++o) {
            int i = site_order[o];
            if (sa[i] * sb[i] == -1) {
                if (seen == rank) { seed_site = i; break; }
                ++seen;
            }
        }
        memset(in_cluster, 0, (size_t)N);
        int head = 0, tail = 0;
        queue[tail++] = seed_site;
        in_cluster[seed_site] = 1;
        while (head < tail) {                    /* breadth-first search */
            int i = queue[head++];
            for (int e = A->start[i]; e < A->start[i + 1]; ++e) {
                int j = A->nbr[e];
                if (!in_cluster[j] && sa[j] * sb[j] == -1) { in_cluster[j] = 1; queue[tail++] = j; }
            }
        }
        for (int q = 0; q < tail; ++q) {         /* flip the cluster in both copies */
            int i = queue[q];
            sa[i] = (int8_t)(-sa[i]);
            sb[i] = (int8_t)(-sb[i]);
        }
        if (tr) { tr->seed_site[k] = seed_site; tr->csize[k] = tail; }
        if (tr && tr->cmask)
            for (int q = 0; q < tail; ++q) tr->cmask[(size_t)k * N + queue[q]] = 1;
    }
    if (tr) tr->esum_after[k] = energy(P, sa) + energy(P, sb);
}

/* Step 3: the PT pass (R8).  E holds the energies of the configurations. */
static void pt_pass(const orc_problem *P, orc_state *S, double *E, const orc_trace *tr)
{
    int N = P->N, nT = P->nT;
    int8_t *tmp = malloc((size_t)N);
    for (int c = 0; c < 2; ++c)
        for (int k = 0; k + 1 < nT; ++k) {
            int ra = 2 * k + c, rb = 2 * (k + 1) + c;
            double bk = 1.0 / P->T[k], bk1 = 1.0 / P->T[k + 1];
            uint32_t x = draw(P->seed, (uint32_t)k, S->t, (uint32_t)c, (2u << 24) | P->inst, 0);
            int accept;
            if (P->pm) {
                long dE = lrint(E[ra]) - lrint(E[rb]);
                if (dE >= 0) accept = 1;
                else {
                    long d = -dE / 2;
                    accept = (uint64_t)x < threshold((double)(-2 * d) * (bk - bk1));
                }
            } else {
                double delta = (bk - bk1) * (E[ra] - E[rb]);
                accept = (delta >= 0.0) || (unit24(x) < exp(delta));
            }
            if (tr) tr->swap_acc[c * (nT - 1) + k] = (uint8_t)accept;
            if (accept) {
                memcpy(tmp, S->s + (size_t)ra * N, (size_t)N);
                memcpy(S->s + (size_t)ra * N, S->s + (size_t)rb * N, (size_t)N);
                memcpy(S->s + (size_t)rb * N, tmp, (size_t)N);
                double e = E[ra]; E[ra] = E[rb]; E[rb] = e;
            }
        }
    free(tmp);
}

/* Observables of the benchmark model (R9): energy, site overlap q, the
 * negative-overlap fraction p and the link overlap q_l of each pair.        */
static void measure(const orc_problem *P, orc_state *S, const double *E)
{
    int N = P->N;
    for (int k = 0; k < P->nT; ++k) {
        const int8_t *sa = S->s + (size_t)(2 * k) * N;
        const int8_t *sb = S->s + (size_t)(2 * k + 1) * N;
        int64_t n = 0, d = 0;
        for (int i = 0; i < N; ++i) n += (sa[i] * sb[i] == -1);
        for (int b = 0; b < P->Nb; ++b) {
            if (P->J[b] == 0.0) continue;        /* absent bond (R10) */
            int i = P->bi[b], j = P->bj[b];
            d += ((sa[i] * sb[i]) * (sa[j] * sb[j]) == -1);
        }
        S->accE[k] += E[2 * k] + E[2 * k + 1];
        S->acc_n[k] += n;
        S->acc_q2[k] += (N - 2 * n) * (N - 2 * n);
        S->acc_pmin[k] += (n < N - n) ? n : N - n;
        S->acc_d[k] += d;
        S->hist[(size_t)k * (N + 1) + n] += 1;
    }
    S->n_meas[0] += 1;
}

/* Run n_sweeps simulation steps of one instance.  The trace (optional)
 * records the last sweep.  Returns 0 on success.                           */
int orc_run(const orc_problem *P, orc_state *S, uint32_t n_sweeps, const orc_trace *tr)
{
    int N = P->N, nT = P->nT, R = 2 * nT;
    if (N <= 0 || nT < 1) return -1;
    adjacency A;
    if (build_adjacency(P, &A)) return -2;
    int32_t *site_order = malloc(sizeof(int32_t) * (size_t)N);
    int32_t *queue = malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *in_cluster = malloc((size_t)N);
    double *E = malloc(sizeof(double) * (size_t)R);
    int o = 0;
    for (int col = 0; col < 2; ++col)
        for (int i = 0; i < N; ++i)
            if (P->color[i] == col) site_order[o++] = i;
    for (int r = 0; r < R; ++r) E[r] = energy(P, S->s + (size_t)r * N);
    int diluted = 0;                             /* R10, R11 */
    for (int b = 0; b < P->Nb; ++b) diluted |= (P->J[b] == 0.0);
    for (uint32_t step = 0; step < n_sweeps; ++step) {
        const orc_trace *trs = (tr && step + 1 == n_sweeps) ? tr : NULL;
        if (trs) {
            for (int k = 0; k < nT; ++k) {
                trs->n_pre[k] = -1; trs->flip2a[k] = 0; trs->seed_site[k] = -1; trs->csize[k] = 0;
                trs->esum_before[k] = 0.0; trs->esum_after[k] = 0.0;
            }
            for (int q = 0; q < 2 * (nT - 1); ++q) trs->swap_acc[q] = 0;
            if (trs->cmask) memset(trs->cmask, 0, (size_t)nT * N);
        }
        if (P->enable_metropolis) metropolis_sweep(P, S, &A, diluted); /* step 1 */
        if (P->icm_every > 0 && S->t % (uint32_t)P->icm_every == 0)   /* steps 2a, 2b */
            for (int k = 0; k < nT; ++k)
                if (P->T[k] <= P->T_icm) cluster_move(P, S, &A, k, site_order, queue, in_cluster, trs);
        for (int r = 0; r < R; ++r) E[r] = energy(P, S->s + (size_t)r * N);
        if (P->swap_every > 0 && S->t % (uint32_t)P->swap_every == 0)  /* step 3 */
            pt_pass(P, S, E, trs);
        if ((int64_t)S->t >= P->t_meas) measure(P, S, E);
        S->t += 1;
    }
    for (int r = 0; r < R; ++r) S->E[r] = E[r];
    free(site_order); free(queue); free(in_cluster); free(E);
    free_adjacency(&A);
    return 0;
}

/* Energy of one configuration, for tests. */
double orc_energy(const orc_problem *P, const int8_t *s) { return energy(P, s); }

/* ------------------------------------------------------------------------ */
/* Site percolation (Supplemental Material): size of the largest connected
 * cluster of occupied sites of each mask, by breadth-first search over the
 * bond list.  masks: [n][N] bytes (nonzero = occupied); smax: [n].          */
int orc_largest_clusters(int32_t N, int32_t Nb, const int32_t *bi, const int32_t *bj, int32_t n,
                         const uint8_t *masks, int32_t *smax)
{
    orc_problem P;
    memset(&P, 0, sizeof P);
    P.N = N; P.Nb = Nb; P.bi = bi; P.bj = bj;
    adjacency A;
    if (build_adjacency(&P, &A)) return -2;
    int32_t *queue = malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    uint8_t *seen = malloc((size_t)(N > 0 ? N : 1));
    for (int m = 0; m < n; ++m) {
        const uint8_t *occ = masks + (size_t)m * N;
        memset(seen, 0, (size_t)N);
        int best = 0;
        for (int s = 0; s < N; ++s) {
            if (!occ[s] || seen[s]) continue;
            int head = 0, tail = 0;
            queue[tail++] = s;
            seen[s] = 1;
            while (head < tail) {
                int i = queue[head++];
                for (int e = A.start[i]; e < A.start[i + 1]; ++e) {
                    int j = A.nbr[e];
                    if (occ[j] && !seen[j]) { seen[j] = 1; queue[tail++] = j; }
                }
            }
            if (tail > best) best = tail;
        }
        smax[m] = best;
    }
    free(queue); free(seen);
    free_adjacency(&A);
    return 0;
}
