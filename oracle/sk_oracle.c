/*
 * sk_oracle.c -- plain, slow FP64 CPU oracle for Many-Configuration
 * Markov-Chain Monte Carlo (MCMCMC) on the Sherrington-Kirkpatrick (SK)
 * spin glass (Simkovic & Rossi, arXiv:2102.05613).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA path: the Philox
 * generator, the weight tables and every step of the chain are written out
 * here a second time, from their published definitions.
 *
 * What it computes (citations are to the paper's sections and equations):
 *
 *  - Energy.  The paper's SK energy (Sec. IV.A) is (1/sqrt L) sum_{j<k} J S S
 *    with J ~ N(0,1).  We use the equivalent E = -scale * sum_{i<j} J_ij s_i s_j
 *    with J ~ N(0,1/N) (Gaussian) or J = +-1 (the +-J model), which is the same
 *    ensemble after J -> -J/sqrt(N).  Local fields h_i = sum_j J_ij s_j, so that
 *    E = -scale/2 sum_i s_i h_i; flipping site i changes E by 2 scale s_i h_i.
 *
 *  - Node rule.  Sec. A.2, Eq. (eq_det_balance_graph_solution): a node c of
 *    the undirected graph T is visited with P_node(c|T) proportional to
 *    P_eq(c) P_gen(T|c), normalised over V(T) (Eq. eq_normalization_p_c_T).
 *    The next graph is generated from the node chosen (Eq. eq_gen_graph).
 *
 *  - Graph.  App. B.2 (general graph populating process): a K-ary tree of
 *    depth one (the "star", K+1 slots) whose root slot is drawn uniformly,
 *    p_r = 1/(K+1), and whose edges are populated with the symmetric
 *    single-spin-flip proposal P_gen(c'|c) = 1/N.  Then P_gen(T|c) is the
 *    same for every slot (the "self-thermalizing tree"), so P_node is
 *    proportional to P_eq = exp(-beta E) alone.
 *      * root = centre (probability 1/(K+1)): slot 0 is the current state c,
 *        slot d = 1..K is c with site_d flipped;
 *      * root = a leaf (probability K/(K+1)): slot 0 is c, slot 1 (the
 *        centre) is c with a = site_1 flipped, slot d = 2..K is the centre
 *        with b = site_d flipped (a double flip, or c itself when b = a).
 *    All slots are labelled, so a configuration present in m slots is
 *    chosen with m times its weight.
 *
 *  - Root distribution.  App. B.2 leaves the root probabilities p_r free.
 *    With the centre drawn as the root with probability p_c and each leaf
 *    with p_l = (1 - p_c)/K, P_gen(T|c in slot j) = p_{r(j)} N^-K, so the
 *    node rule weights slot j by P_eq(c_j) p_{r(j)}: the centre slot by p_c,
 *    every leaf slot by p_l.  p_c = 1/(K+1) is the uniform root above.
 *
 *  - Node-weighted estimator.  Sec. A.2, Eq. (eq_monte_carlo_graph): an
 *    observable may be averaged over all nodes of each step's graph with
 *    their node probabilities.  For the energy of a state c and the graph T
 *    the next step generates from it, E_nw = sum_j P_node(j|T) E(c_j) =
 *    E(c) + sum_j P_node(j|T) dE_j, the expectation of the next state's
 *    energy given T; for the Metropolis comparator the same conditional
 *    expectation over accept / reject, E(c) + p_acc dE.  Records store it
 *    next to E(c), for the graph of the step after the record.
 *
 *  - K = 1 of the same rule is the two-node heat-bath chain of Sec. III.A,
 *    Eq. (eq_node_two_conf).  The "standard local Metropolis" comparator of
 *    Sec. IV.B uses the acceptance min(1, P_eq(c1)/P_eq(c0)) of Sec. II.
 *
 *  Readings where the paper is silent (random numbers, integer weight
 *  tables, tie-breaks, acceptance of an MCMCMC step) are spelt out at each
 *  function below.  Random numbers come from Philox4x32-10 (Salmon, Moraes,
 *  Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11),
 *  addressed by counter = (block, step, chain, domain<<24 | stream) and
 *  key = (seed low word, seed high word).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SKO_PM1 0
#define SKO_GAUSS 1
#define SKO_MCMCMC 0
#define SKO_METROPOLIS 1
#define SKO_MAX_K 256
#define SKO_MAXSLOT_GUARD (SKO_MAX_K + 1)

/* ------------------------------------------------------------------ */
/* Philox4x32-10, SC'11: ten rounds of two 32x32->64 multiplies with   */
/* the multipliers 0xD2511F53, 0xCD9E8D57; the key is bumped by the    */
/* Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.               */
/* ------------------------------------------------------------------ */
void sko_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One Philox block of the chain's stream. */
static void draw_block(uint64_t seed, uint32_t stream, uint32_t domain,
                       uint32_t chain, uint64_t step, uint32_t block, uint32_t out[4]) {
    uint32_t ctr[4] = {block, (uint32_t)step, chain, (domain << 24) | (stream & 0xFFFFFFu)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    sko_philox(ctr, key, out);
}

/* floor(x * n / 2^32): a 32-bit word mapped onto {0..n-1}. */
static uint32_t range32(uint32_t x, uint32_t n) {
    return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32);
}

/* floor(x * n / 2^64) for 64-bit x. */
static uint64_t range64(uint64_t x, uint64_t n) {
    return (uint64_t)(((unsigned __int128)x * (unsigned __int128)n) >> 64);
}

/* ------------------------------------------------------------------ */
/* Model                                                               */
/* ------------------------------------------------------------------ */
static double coupling(int kind, const void* J, int N, int i, int j) {
    if (kind == SKO_PM1) return (double)((const int8_t*)J)[(size_t)i * N + j];
    return (double)((const float*)J)[(size_t)i * N + j];
}

/* E = -scale * sum_{i<j} J_ij s_i s_j, written out as the double sum. */
double sko_energy(int N, int kind, const void* J, double scale, const int8_t* s) {
    double e = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j)
            e += coupling(kind, J, N, i, j) * (double)s[i] * (double)s[j];
    return -scale * e;
}

/*
 * Couplings drawn from a seed, the instance generator of the library's
 * sk_create_instance with couplings NULL, written out here separately:
 * Philox4x32-10 with key = (seed low, seed high), domain 2, one draw per pair
 * i < j shared by J_ij and J_ji:
 *   +-J (kind 0):      counter (j >> 7, i, 0, 2 << 24), bit j mod 128 of the
 *                      block (word (j mod 128) / 32, bit j mod 32): set -> -1;
 *   Gaussian (kind 1): counter (j, i, 1, 2 << 24) -> (w0, w1, w2, w3); the
 *                      53-bit uniforms u1 = (2^26 (w0 >> 5) + (w1 >> 6)) 2^-53
 *                      and u2 from (w2, w3); the Box-Muller normal (Box &
 *                      Muller 1958) z = sqrt(-2 ln(1 - u1)) cos(2 pi u2);
 *                      J_ij = (float)(z / sqrt(N)), so J ~ N(0, 1/N).
 * Zero diagonal.  out: N*N int8 (kind 0) or float (kind 1), row-major.
 */
void sko_gen_couplings(int N, int kind, uint64_t seed, void* out) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = 0; i < N; ++i) {
        if (kind == SKO_PM1) ((int8_t*)out)[(size_t)i * N + i] = 0;
        else ((float*)out)[(size_t)i * N + i] = 0.0f;
        for (int j = i + 1; j < N; ++j) {
            uint32_t w[4];
            if (kind == SKO_PM1) {
                const uint32_t ctr[4] = {(uint32_t)j >> 7, (uint32_t)i, 0u, 2u << 24};
                sko_philox(ctr, key, w);
                const int b = j % 128;
                const int8_t v = ((w[b / 32] >> (b % 32)) & 1u) ? (int8_t)-1 : (int8_t)1;
                ((int8_t*)out)[(size_t)i * N + j] = v;
                ((int8_t*)out)[(size_t)j * N + i] = v;
            } else {
                const uint32_t ctr[4] = {(uint32_t)j, (uint32_t)i, 1u, 2u << 24};
                sko_philox(ctr, key, w);
                const double u1 = ((double)(w[0] >> 5) * 67108864.0 + (double)(w[1] >> 6)) * ldexp(1.0, -53);
                const double u2 = ((double)(w[2] >> 5) * 67108864.0 + (double)(w[3] >> 6)) * ldexp(1.0, -53);
                const double z = sqrt(-2.0 * log(1.0 - u1)) * cos(6.283185307179586476925286766559 * u2);
                const float v = (float)(z / sqrt((double)N));
                ((float*)out)[(size_t)i * N + j] = v;
                ((float*)out)[(size_t)j * N + i] = v;
            }
        }
    }
}

/* h_i = sum_j J_ij s_j (unscaled). */
void sko_fields(int N, int kind, const void* J, const int8_t* s, double* h) {
    for (int i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int j = 0; j < N; ++j) acc += coupling(kind, J, N, i, j) * (double)s[j];
        h[i] = acc;
    }
}

/* Random start: domain 1, 128 spins per Philox block, bit set -> -1. */
void sko_init_spins(uint64_t seed, uint32_t stream, uint32_t chain, int N, int8_t* s) {
    for (int i = 0; i < N; i += 128) {
        uint32_t w[4];
        draw_block(seed, stream, 1u, chain, 0, (uint32_t)(i / 128), w);
        for (int k = 0; k < 128 && i + k < N; ++k) {
            uint32_t bit = (w[k / 32] >> (k % 32)) & 1u;
            s[i + k] = bit ? (int8_t)-1 : (int8_t)1;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Integer weight tables for the +-J model (reading of the paper's     */
/* P_eq ratios in exact integer arithmetic, so that two independent    */
/* implementations take identical decisions).                          */
/*   MCMCMC:     W[d] = round(2^52 exp(-2 beta_eff d)), d = (dE-min)/2, */
/*               cut at the first entry that rounds to zero.           */
/*   Metropolis: M[k] = round(2^53 exp(-2 beta_eff k)), k = dE/2 >= 1.  */
/* ------------------------------------------------------------------ */
int sko_weight_table(double beta_eff, int dmax, uint64_t* W) {
    int len = 0;
    for (int d = 0; d <= dmax; ++d) {
        double v = nearbyint(ldexp(exp(-2.0 * beta_eff * (double)d), 52));
        if (v <= 0.0) break;
        W[d] = (uint64_t)v;
        len = d + 1;
    }
    return len;
}

int sko_metropolis_table(double beta_eff, int kmax, uint64_t* M) {
    for (int k = 0; k <= kmax; ++k) {
        double v = nearbyint(ldexp(exp(-2.0 * beta_eff * (double)k), 53));
        M[k] = (uint64_t)v;
    }
    return kmax + 1;
}

/* ------------------------------------------------------------------ */
/* One chain                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    int N, kind, K, rule;
    const void* J;
    double scale, beta;
    uint64_t seed;
    uint32_t stream;
    /* +-J integer tables */
    uint64_t* W;
    int wlen;
    uint64_t* M;
    int mlen;
    /* root distribution: p_center = 0 is the uniform root 1/(K+1) */
    double p_center;
    uint64_t root_thr;    /* non-uniform: the centre is the root iff U0 < root_thr */
    double f_c, f_l;      /* slot weight factors p_c / max(p_c, p_l), p_l / max(..) */
    uint64_t F_c, F_l;    /* the same as integers round(f 2^20) for the +-J tables */
} sko_ctx;

typedef struct {
    int n_moves;      /* 0, 1 or 2 spins to flip */
    int site[2];
    int slot;         /* selected slot, 0..K */
} sko_move;

/*
 * Candidate energies of the K+1 slots (Sec. A.2 node rule on the App. B.2
 * star).  Returns in dE[j] the unscaled energy change of slot j relative to
 * the current state, and in flips[j] the spins that slot j differs by.
 */
static void star_candidates(const sko_ctx* c, const int8_t* s, const double* h,
                            int leaf_root, const uint32_t* sites,
                            double* dE, int (*flips)[2], int* nflip) {
    const int K = c->K;
    dE[0] = 0.0;
    nflip[0] = 0;
    if (!leaf_root) {
        for (int d = 1; d <= K; ++d) {
            int i = (int)sites[d];
            dE[d] = 2.0 * (double)s[i] * h[i];
            flips[d][0] = i;
            nflip[d] = 1;
        }
        return;
    }
    int a = (int)sites[1];
    double dEa = 2.0 * (double)s[a] * h[a];
    dE[1] = dEa;
    flips[1][0] = a;
    nflip[1] = 1;
    for (int d = 2; d <= K; ++d) {
        int b = (int)sites[d];
        if (b == a) {            /* the centre flipped back: the root itself */
            dE[d] = 0.0;
            nflip[d] = 0;
            continue;
        }
        /* E(c^{a,b}) - E(c) = 2 s_a h_a + 2 s_b h_b - 4 J_ab s_a s_b */
        dE[d] = dEa + 2.0 * (double)s[b] * h[b]
              - 4.0 * coupling(c->kind, c->J, c->N, a, b) * (double)s[a] * (double)s[b];
        flips[d][0] = a;
        flips[d][1] = b;
        nflip[d] = 2;
    }
}

/*
 * Weight of slot j, proportional to exp(-beta_eff dE_j) times the root
 * factor of the slot (1 for the uniform root; the centre slot is slot 0 of
 * a centre root and slot 1 of a leaf root).  m is the minimum of dE over the
 * slots, a normalisation that cancels in the node probabilities.
 *   +-J: W[(dE_j - m)/2] from the integer table (0 past its end), then
 *        floor(W F / 2^20) with the slot's integer factor F when the root is
 *        not uniform;
 *   Gaussian: exp(-beta_eff (dE_j - m)) f in double precision.
 */
static double min_dE(const double* dE, int nslot) {
    double m = dE[0];
    for (int j = 1; j < nslot; ++j) if (dE[j] < m) m = dE[j];
    return m;
}

static int is_centre_slot(int j, int leaf_root) { return j == (leaf_root ? 1 : 0); }

static uint64_t weight_int(const sko_ctx* c, double dEj, double m, int centre) {
    long long d = (long long)llround((dEj - m) * 0.5);
    uint64_t w = (d < c->wlen) ? c->W[d] : 0u;
    if (c->p_center > 0.0) {
        uint64_t F = centre ? c->F_c : c->F_l;
        w = (uint64_t)(((unsigned __int128)w * (unsigned __int128)F) >> 20);
    }
    return w;
}

static double weight_dbl(const sko_ctx* c, double dEj, double m, int centre) {
    double w = exp(-c->beta * c->scale * (dEj - m));
    if (c->p_center > 0.0) w *= centre ? c->f_c : c->f_l;
    return w;
}

/*
 * Slot selection with probability proportional to the slot weights above.
 *   +-J: inclusive integer prefix P_j in slot order, u = floor(U * P_K /
 *        2^64), the first j with P_j > u.
 *   Gaussian: the same in double precision with u = (U>>40) 2^-24 P_K.
 */
static int select_slot(const sko_ctx* c, const double* dE, int nslot, int leaf_root, uint64_t U) {
    const double m = min_dE(dE, nslot);
    if (c->kind == SKO_PM1) {
        uint64_t P[SKO_MAXSLOT_GUARD];
        uint64_t acc = 0;
        for (int j = 0; j < nslot; ++j) {
            acc += weight_int(c, dE[j], m, is_centre_slot(j, leaf_root));
            P[j] = acc;
        }
        uint64_t u = range64(U, acc);
        for (int j = 0; j < nslot; ++j)
            if (P[j] > u) return j;
        return nslot - 1; /* unreachable: u < P_K */
    } else {
        double P[SKO_MAXSLOT_GUARD];
        double acc = 0.0;
        for (int j = 0; j < nslot; ++j) {
            acc += weight_dbl(c, dE[j], m, is_centre_slot(j, leaf_root));
            P[j] = acc;
        }
        double u = (double)(U >> 40) * ldexp(1.0, -24) * acc;
        for (int j = 0; j < nslot; ++j)
            if (P[j] > u) return j;
        for (int j = nslot - 1; j >= 0; --j)
            if (weight_dbl(c, dE[j], m, is_centre_slot(j, leaf_root)) > 0.0) return j;
        return 0;
    }
}

/* Flip spin x: h_k -= 2 s_x J_kx for every k, then s_x = -s_x. */
static void flip_spin(const sko_ctx* c, int8_t* s, double* h, int x) {
    double sx = (double)s[x];
    for (int k = 0; k < c->N; ++k) h[k] -= 2.0 * sx * coupling(c->kind, c->J, c->N, k, x);
    s[x] = (int8_t)(-s[x]);
}

/*
 * Step t of one chain.  The MCMCMC step draws Philox block 0 of domain 0
 * (U0 = w1:w0 picks the root slot, U1 = w3:w2 picks the node) and blocks
 * 1..ceil(K/4) (site_d = floor(w * N / 2^32), four per block, d = 1..K).
 * The Metropolis step draws block 0 only: site = floor(w0 N / 2^32),
 * U1 = w3:w2 decides acceptance.
 *
 * forced >= 0 replays a slot chosen elsewhere instead of the oracle's own
 * choice (used by the decision-replay check); *own returns the oracle's
 * choice, Pout and uout the prefix sums and the draw it was taken with.
 * Returns 1 when the configuration changed (the acceptance count).
 */
static int chain_step(const sko_ctx* c, uint32_t chain, uint64_t t, int8_t* s, double* h,
                      int forced, int* own, double* Pout, double* uout) {
    uint32_t w0[4];
    draw_block(c->seed, c->stream, 0u, chain, t, 0u, w0);
    uint64_t U0 = ((uint64_t)w0[1] << 32) | w0[0];
    uint64_t U1 = ((uint64_t)w0[3] << 32) | w0[2];
    if (c->rule == SKO_METROPOLIS) {
        int i = (int)range32(w0[0], (uint32_t)c->N);
        double dE = 2.0 * (double)s[i] * h[i];
        int accept;
        double pacc;
        if (c->kind == SKO_PM1) {
            long long k = llround(dE * 0.5);
            accept = (dE <= 0.0) || ((U1 >> 11) < c->M[k]);
            pacc = (dE <= 0.0) ? 1.0 : ldexp((double)c->M[k], -53);
            if (uout) *uout = ldexp((double)(U1 >> 11), -53);
        } else {
            pacc = (dE <= 0.0) ? 1.0 : exp(-c->beta * c->scale * dE);
            double u = (double)(U1 >> 40) * ldexp(1.0, -24);
            accept = (dE <= 0.0) || (u < pacc);
            if (uout) *uout = u;
        }
        if (Pout) Pout[0] = pacc;
        if (own) *own = accept;
        if (forced >= 0) accept = forced;
        if (accept) flip_spin(c, s, h, i);
        return accept;
    }

    const int K = c->K;
    /* root: slot drawn uniformly from K+1 (leaf iff the draw is not 0), or
       the centre with probability p_center */
    int leaf_root = (c->p_center > 0.0) ? (U0 >= c->root_thr)
                                        : (range64(U0, (uint64_t)K + 1u) != 0u);
    uint32_t sites[SKO_MAXSLOT_GUARD] = {0};
    for (int d = 1; d <= K; ++d) {
        uint32_t wb[4];
        draw_block(c->seed, c->stream, 0u, chain, t, (uint32_t)(1 + (d - 1) / 4), wb);
        sites[d] = range32(wb[(d - 1) % 4], (uint32_t)c->N);
    }
    double dE[SKO_MAXSLOT_GUARD];
    int flips[SKO_MAXSLOT_GUARD][2];
    int nflip[SKO_MAXSLOT_GUARD];
    star_candidates(c, s, h, leaf_root, sites, dE, flips, nflip);
    int j = select_slot(c, dE, K + 1, leaf_root, U1);
    if (own) *own = j;
    if (Pout || uout) {
        /* prefix sums in the same order as select_slot, for the replay check */
        const double m = min_dE(dE, K + 1);
        double acc = 0.0;
        for (int q = 0; q <= K; ++q) {
            const int centre = is_centre_slot(q, leaf_root);
            acc += (c->kind == SKO_PM1) ? (double)weight_int(c, dE[q], m, centre)
                                        : weight_dbl(c, dE[q], m, centre);
            if (Pout) Pout[q] = acc;
        }
        if (uout) *uout = (c->kind == SKO_PM1) ? ldexp((double)U1, -64) * acc
                                               : (double)(U1 >> 40) * ldexp(1.0, -24) * acc;
    }
    if (forced >= 0) j = forced;
    for (int f = 0; f < nflip[j]; ++f) flip_spin(c, s, h, flips[j][f]);
    return nflip[j] > 0;
}

/*
 * Node-weighted energy change of the graph that step t generates from the
 * state (s, h), without taking the step: sum_j P_node(j) dE_j over its K+1
 * slots with the probabilities the step chooses with (the same draws,
 * candidates and weights as chain_step); Metropolis: p_acc dE of its
 * proposal.
 */
static double graph_mean_dE(const sko_ctx* c, uint32_t chain, uint64_t t, const int8_t* s, const double* h) {
    uint32_t w0[4];
    draw_block(c->seed, c->stream, 0u, chain, t, 0u, w0);
    const uint64_t U0 = ((uint64_t)w0[1] << 32) | w0[0];
    if (c->rule == SKO_METROPOLIS) {
        const int i = (int)range32(w0[0], (uint32_t)c->N);
        const double dE = 2.0 * (double)s[i] * h[i];
        double pacc = 1.0;
        if (dE > 0.0)
            pacc = (c->kind == SKO_PM1) ? ldexp((double)c->M[llround(dE * 0.5)], -53)
                                        : exp(-c->beta * c->scale * dE);
        return pacc * dE;
    }
    const int K = c->K;
    const int leaf_root = (c->p_center > 0.0) ? (U0 >= c->root_thr) : (range64(U0, (uint64_t)K + 1u) != 0u);
    uint32_t sites[SKO_MAXSLOT_GUARD] = {0};
    for (int d = 1; d <= K; ++d) {
        uint32_t wb[4];
        draw_block(c->seed, c->stream, 0u, chain, t, (uint32_t)(1 + (d - 1) / 4), wb);
        sites[d] = range32(wb[(d - 1) % 4], (uint32_t)c->N);
    }
    double dE[SKO_MAXSLOT_GUARD];
    int flips[SKO_MAXSLOT_GUARD][2];
    int nflip[SKO_MAXSLOT_GUARD];
    star_candidates(c, s, h, leaf_root, sites, dE, flips, nflip);
    const double m = min_dE(dE, K + 1);
    double num = 0.0, den = 0.0;
    for (int q = 0; q <= K; ++q) {
        const int centre = is_centre_slot(q, leaf_root);
        const double w = (c->kind == SKO_PM1) ? (double)weight_int(c, dE[q], m, centre)
                                              : weight_dbl(c, dE[q], m, centre);
        num += w * dE[q];
        den += w;
    }
    return num / den;
}

/*
 * Root distribution (App. B.2, p_r free): p_center = 0 selects the uniform
 * root; 0 < p_center < 1 asks for the centre as the root with probability
 * p_center and every leaf with p_l = (1 - p_center)/K.  The slot factors are
 * the root probabilities over the larger of the two, kept as 20-bit integers
 * F = round(f 2^20) (one of them 2^20; both must be >= 1, else -1), and the
 * root probabilities actually used are the ones these integers fix exactly,
 * p~_c = F_c / (F_c + K F_l) and p~_l = F_l / (F_c + K F_l), so that the
 * factors stay proportional to the root probabilities (the condition for
 * detailed balance).  The root is the centre iff U0 < floor(p~_c 2^64).
 * The Gaussian weights take f = F / 2^20.  Metropolis ignores p_center.
 */
static int root_setup(sko_ctx* c, double p_center) {
    c->p_center = 0.0;
    c->f_c = c->f_l = 1.0;
    c->F_c = c->F_l = (uint64_t)1 << 20;
    c->root_thr = 0;
    if (c->rule != SKO_MCMCMC || p_center == 0.0) return 0;
    if (!(p_center > 0.0 && p_center < 1.0)) return -1;
    const double pl = (1.0 - p_center) / (double)c->K;
    const double pm = p_center > pl ? p_center : pl;
    c->F_c = (uint64_t)(p_center / pm * 1048576.0 + 0.5);
    c->F_l = (uint64_t)(pl / pm * 1048576.0 + 0.5);
    if (c->F_c < 1u || c->F_l < 1u) return -1;
    c->f_c = ldexp((double)c->F_c, -20);
    c->f_l = ldexp((double)c->F_l, -20);
    c->p_center = (double)c->F_c / ((double)c->F_c + (double)c->K * (double)c->F_l);
    c->root_thr = (uint64_t)ldexp(c->p_center, 64);
    return 0;
}

static int ctx_init(sko_ctx* c, int N, int kind, const void* J, double scale, int rule, int K,
                    double beta, uint64_t seed, uint32_t stream, double p_center) {
    if (N < 2 || N > 65536 || !J) return -1;
    if (kind != SKO_PM1 && kind != SKO_GAUSS) return -1;
    if (rule != SKO_MCMCMC && rule != SKO_METROPOLIS) return -1;
    if (rule == SKO_MCMCMC && (K < 1 || K > SKO_MAX_K)) return -1;
    if (!(beta >= 0.0) || !(scale > 0.0)) return -1;
    memset(c, 0, sizeof(*c));
    c->N = N; c->kind = kind; c->J = J; c->scale = scale; c->rule = rule; c->K = K;
    c->beta = beta; c->seed = seed; c->stream = stream;
    if (root_setup(c, p_center)) return -1;
    if (kind == SKO_PM1) {
        int dmax = 4 * N + 4;
        c->W = (uint64_t*)calloc((size_t)dmax + 1, sizeof(uint64_t));
        c->M = (uint64_t*)calloc((size_t)N + 1, sizeof(uint64_t));
        if (!c->W || !c->M) return -2;
        c->wlen = sko_weight_table(beta * scale, dmax, c->W);
        c->mlen = sko_metropolis_table(beta * scale, N, c->M);
    }
    return 0;
}

static void ctx_free(sko_ctx* c) {
    free(c->W);
    free(c->M);
}

/*
 * Runs chains chain0 .. chain0+nchains-1 for nsteps steps from step 0.
 *   init_spins: nchains*N spins (+-1), or NULL for the Philox random start.
 *   Every record_every steps (after step t with (t+1) % record_every == 0)
 *   record r stores: rec_E[r*nchains+i] = scale * E of chain i,
 *   rec_acc[r*nchains+i] = steps in the interval whose configuration changed,
 *   rec_q[r*(nchains/2)+m] = (1/N) sum_k s_k s'_k of the pair (2m, 2m+1)
 *   (chain0 must be even for q), rec_Enw[r*nchains+i] = scale * the
 *   node-weighted energy of the recorded state with the graph of step t+1
 *   (see the header).  Any
 *   output may be NULL.  p_center: the root distribution (root_setup).
 *   trace (nchains*nsteps, may be NULL) receives the slot chosen at each step
 *   (Metropolis: 1 accepted, 0 rejected).
 *   resync_every > 0 recomputes the fields from scratch at that period and
 *   checks them against the maintained ones (exact for +-J, 1e-9 Gaussian).
 * Returns 0, -1 on a bad argument, -2 out of memory, -3 on a field mismatch.
 */
int sko_run_p(int N, int kind, const void* J, double scale, int rule, int K, double beta,
              uint64_t seed, uint32_t stream, uint32_t chain0, uint32_t nchains,
              const int8_t* init_spins, uint64_t nsteps, uint32_t record_every,
              double* rec_E, uint32_t* rec_acc, double* rec_q,
              int8_t* final_spins, double* final_E, int32_t* trace, uint32_t resync_every,
              double p_center, double* rec_Enw) {
    sko_ctx c;
    int rc = ctx_init(&c, N, kind, J, scale, rule, K, beta, seed, stream, p_center);
    if (rc) return rc;
    if (rec_q && (chain0 % 2u) != 0u) { ctx_free(&c); return -1; }
    uint64_t nrec = record_every ? nsteps / record_every : 0;
    int8_t* s = (int8_t*)malloc((size_t)N);
    double* h = (double*)malloc(sizeof(double) * (size_t)N);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)N);
    int8_t* partner = (int8_t*)malloc((size_t)N * (nrec ? nrec : 1));
    if (!s || !h || !h2 || !partner) { rc = -2; goto done; }
    for (uint32_t ci = 0; ci < nchains; ++ci) {
        uint32_t chain = chain0 + ci;
        if (init_spins) memcpy(s, init_spins + (size_t)ci * N, (size_t)N);
        else sko_init_spins(seed, stream, 0 + chain, N, s);
        sko_fields(N, kind, J, s, h);
        uint32_t acc = 0;
        for (uint64_t t = 0; t < nsteps; ++t) {
            int own = -1;
            acc += (uint32_t)chain_step(&c, chain, t, s, h, -1, &own, NULL, NULL);
            if (trace) trace[(size_t)ci * nsteps + t] = own;
            if (resync_every && ((t + 1) % resync_every) == 0) {
                sko_fields(N, kind, J, s, h2);
                for (int k = 0; k < N; ++k) {
                    double d = fabs(h2[k] - h[k]);
                    if ((kind == SKO_PM1 && d != 0.0) || (kind == SKO_GAUSS && d > 1e-9)) {
                        rc = -3;
                        goto done;
                    }
                }
            }
            if (record_every && ((t + 1) % record_every) == 0) {
                uint64_t r = (t + 1) / record_every - 1;
                if (rec_E || rec_Enw) {
                    const double E = sko_energy(N, kind, J, scale, s);
                    if (rec_E) rec_E[r * nchains + ci] = E;
                    if (rec_Enw) rec_Enw[r * nchains + ci] = E + scale * graph_mean_dE(&c, chain, t + 1, s, h);
                }
                if (rec_acc) rec_acc[r * nchains + ci] = acc;
                acc = 0;
                if (rec_q) {
                    if ((ci % 2u) == 0u) {
                        memcpy(partner + (size_t)r * N, s, (size_t)N);
                    } else {
                        double q = 0.0;
                        for (int k = 0; k < N; ++k)
                            q += (double)s[k] * (double)partner[(size_t)r * N + k];
                        rec_q[r * (nchains / 2) + ci / 2] = q / (double)N;
                    }
                }
            }
        }
        if (final_spins) memcpy(final_spins + (size_t)ci * N, s, (size_t)N);
        if (final_E) final_E[ci] = sko_energy(N, kind, J, scale, s);
    }
done:
    free(s); free(h); free(h2); free(partner);
    ctx_free(&c);
    return rc;
}

/* sko_run_p with the uniform root. */
int sko_run(int N, int kind, const void* J, double scale, int rule, int K, double beta,
            uint64_t seed, uint32_t stream, uint32_t chain0, uint32_t nchains,
            const int8_t* init_spins, uint64_t nsteps, uint32_t record_every,
            double* rec_E, uint32_t* rec_acc, double* rec_q,
            int8_t* final_spins, double* final_E, int32_t* trace, uint32_t resync_every) {
    return sko_run_p(N, kind, J, scale, rule, K, beta, seed, stream, chain0, nchains, init_spins,
                     nsteps, record_every, rec_E, rec_acc, rec_q, final_spins, final_E, trace,
                     resync_every, 0.0, NULL);
}

/*
 * Decision replay for one chain: walks the chain with the oracle's random
 * numbers but follows the slot sequence `slots` taken elsewhere (the GPU
 * trace).  A step whose slot differs from the oracle's own choice is
 * admissible when the oracle's draw u lies within tol * P_K of the chosen
 * slot's interval [P_{j-1}, P_j) (Metropolis: within tol of the acceptance
 * threshold), i.e. when it is a near-tie that rounding may decide either way.
 * Returns the number of inadmissible steps (>= 0) or a negative error;
 * n_disagree counts all differing steps, first_bad the first inadmissible one.
 */
long long sko_replay_p(int N, int kind, const void* J, double scale, int rule, int K, double beta,
                       uint64_t seed, uint32_t stream, uint32_t chain, const int8_t* init_spins,
                       uint64_t nsteps, const int32_t* slots, double tol,
                       long long* n_disagree, long long* first_bad,
                       int8_t* final_spins, double* final_E, double p_center) {
    sko_ctx c;
    int rc = ctx_init(&c, N, kind, J, scale, rule, K, beta, seed, stream, p_center);
    if (rc) return rc;
    int8_t* s = (int8_t*)malloc((size_t)N);
    double* h = (double*)malloc(sizeof(double) * (size_t)N);
    double P[SKO_MAXSLOT_GUARD];
    long long bad = 0, dis = 0, first = -1;
    if (!s || !h) { free(s); free(h); ctx_free(&c); return -2; }
    if (init_spins) memcpy(s, init_spins, (size_t)N);
    else sko_init_spins(seed, stream, chain, N, s);
    sko_fields(N, kind, J, s, h);
    for (uint64_t t = 0; t < nsteps; ++t) {
        int g = slots[t];
        int nslot = (rule == SKO_METROPOLIS) ? 2 : K + 1;
        if (g < 0 || g >= nslot) { bad++; if (first < 0) first = (long long)t; break; }
        int own = -1;
        double u = 0.0;
        chain_step(&c, chain, t, s, h, g, &own, P, &u);
        if (own != g) {
            dis++;
            int ok;
            if (rule == SKO_METROPOLIS) {
                ok = fabs(u - P[0]) <= tol;
            } else {
                double PK = P[K];
                double lo = (g == 0) ? 0.0 : P[g - 1];
                double hi = P[g];
                ok = (u >= lo - tol * PK) && (u < hi + tol * PK);
            }
            if (!ok) { bad++; if (first < 0) first = (long long)t; }
        }
    }
    if (final_spins) memcpy(final_spins, s, (size_t)N);
    if (final_E) *final_E = sko_energy(N, kind, J, scale, s);
    if (n_disagree) *n_disagree = dis;
    if (first_bad) *first_bad = first;
    free(s); free(h);
    ctx_free(&c);
    return bad;
}

/*
 * One chain's own trajectory together with what each step's choice is taken
 * from, so that tests can place a replayed slot relative to the draw:
 * own[t] = the slot the step chose (Metropolis: 1 accepted, 0 rejected),
 * u[t] = its draw on the scale of the prefix sums, P[t * stride + j] = the
 * inclusive prefix sums of the slot weights in slot order (stride K + 1;
 * Metropolis: stride 1, P = the acceptance probability).  Returns 0 or a
 * negative error as sko_run.
 */
int sko_run_detail(int N, int kind, const void* J, double scale, int rule, int K, double beta,
                   uint64_t seed, uint32_t stream, uint32_t chain, const int8_t* init_spins,
                   uint64_t nsteps, double p_center, int32_t* own, double* u, double* P) {
    sko_ctx c;
    int rc = ctx_init(&c, N, kind, J, scale, rule, K, beta, seed, stream, p_center);
    if (rc) return rc;
    const int stride = (rule == SKO_METROPOLIS) ? 1 : K + 1;
    int8_t* s = (int8_t*)malloc((size_t)N);
    double* h = (double*)malloc(sizeof(double) * (size_t)N);
    if (!s || !h) { free(s); free(h); ctx_free(&c); return -2; }
    if (init_spins) memcpy(s, init_spins, (size_t)N);
    else sko_init_spins(seed, stream, chain, N, s);
    sko_fields(N, kind, J, s, h);
    double Pb[SKO_MAXSLOT_GUARD];
    for (uint64_t t = 0; t < nsteps; ++t) {
        int o = -1;
        double uu = 0.0;
        chain_step(&c, chain, t, s, h, -1, &o, Pb, &uu);
        own[t] = o;
        u[t] = uu;
        memcpy(P + (size_t)t * (size_t)stride, Pb, sizeof(double) * (size_t)stride);
    }
    free(s); free(h);
    ctx_free(&c);
    return 0;
}

/* sko_replay_p with the uniform root. */
long long sko_replay(int N, int kind, const void* J, double scale, int rule, int K, double beta,
                     uint64_t seed, uint32_t stream, uint32_t chain, const int8_t* init_spins,
                     uint64_t nsteps, const int32_t* slots, double tol,
                     long long* n_disagree, long long* first_bad,
                     int8_t* final_spins, double* final_E) {
    return sko_replay_p(N, kind, J, scale, rule, K, beta, seed, stream, chain, init_spins, nsteps,
                        slots, tol, n_disagree, first_bad, final_spins, final_E, 0.0);
}

/* ------------------------------------------------------------------ */
/* Exact enumeration (small N)                                         */
/* ------------------------------------------------------------------ */
static void spins_of(uint32_t x, int N, int8_t* s) {
    for (int i = 0; i < N; ++i) s[i] = ((x >> i) & 1u) ? (int8_t)-1 : (int8_t)1;
}

/* pi(x) = exp(-beta E(x)) / Z over all 2^N states, x bit i set <=> s_i = -1. */
int sko_boltzmann(int N, int kind, const void* J, double scale, double beta, double* pi) {
    if (N < 1 || N > 24) return -1;
    int8_t s[24];
    uint32_t n = 1u << N;
    double emin = INFINITY;
    for (uint32_t x = 0; x < n; ++x) {
        spins_of(x, N, s);
        pi[x] = sko_energy(N, kind, J, scale, s);
        if (pi[x] < emin) emin = pi[x];
    }
    double Z = 0.0;
    for (uint32_t x = 0; x < n; ++x) {
        pi[x] = exp(-beta * (pi[x] - emin));
        Z += pi[x];
    }
    for (uint32_t x = 0; x < n; ++x) pi[x] /= Z;
    return 0;
}

/*
 * Exact one-step transition matrix P[x*2^N + y] of the chain, by enumerating
 * the root choice and every K-tuple of sites (N^K tuples, each 1/N^K).
 *   root_mode 0: the method: uniform root over the K+1 slots, or (p_center
 *                > 0) the centre with probability p_center and the slot
 *                weights times the root probabilities;
 *   root_mode 1: the root always at the centre (an invalid variant, kept as a
 *                negative control for the detailed-balance test);
 *   root_mode 2: the centre as root with probability p_center but the slot
 *                weights left without the root factor (a second invalid
 *                variant, the negative control for the root factors).
 *   weight_mode 0: weights exp(-beta dE) in double precision;
 *   weight_mode 1: the +-J integer tables used by the trajectories.
 */
int sko_transition_matrix_p(int N, int kind, const void* J, double scale, int rule, int K,
                            double beta, int root_mode, int weight_mode, double p_center,
                            double* P) {
    if (N < 1 || N > 12) return -1;
    if (rule == SKO_MCMCMC && (K < 1 || K > 8)) return -1;
    if (root_mode == 2 && !(p_center > 0.0)) return -1;
    sko_ctx c;
    int rc = ctx_init(&c, N, kind, J, scale, rule, K < 1 ? 1 : K, beta, 0, 0,
                      root_mode == 1 ? 0.0 : p_center);
    if (rc) return rc;
    const double pc = c.p_center > 0.0 ? c.p_center : 1.0 / (double)((K < 1 ? 1 : K) + 1);
    if (root_mode == 2) {  /* drop the factors, keep the root probabilities */
        c.p_center = 0.0;
    }
    if (weight_mode == 1 && kind != SKO_PM1) { ctx_free(&c); return -1; }
    uint32_t n = 1u << N;
    memset(P, 0, sizeof(double) * (size_t)n * n);
    int8_t s[12];
    double h[12];
    const double be = beta * scale;
    for (uint32_t x = 0; x < n; ++x) {
        spins_of(x, N, s);
        sko_fields(N, kind, J, s, h);
        double* row = P + (size_t)x * n;
        if (rule == SKO_METROPOLIS) {
            for (int i = 0; i < N; ++i) {
                double dE = 2.0 * (double)s[i] * h[i];
                double a;
                if (dE <= 0.0) a = 1.0;
                else if (weight_mode == 1) a = ldexp((double)c.M[llround(dE * 0.5)], -53);
                else a = exp(-be * dE);
                row[x ^ (1u << i)] += a / (double)N;
                row[x] += (1.0 - a) / (double)N;
            }
            continue;
        }
        long long ntup = 1;
        for (int d = 0; d < K; ++d) ntup *= N;
        const double ptup = 1.0 / (double)ntup;
        for (int leaf = 0; leaf <= 1; ++leaf) {
            double proot;
            if (root_mode == 1) proot = leaf ? 0.0 : 1.0;
            else proot = leaf ? 1.0 - pc : pc;
            if (proot == 0.0) continue;
            uint32_t sites[SKO_MAXSLOT_GUARD] = {0};
            for (long long tup = 0; tup < ntup; ++tup) {
                double dE[SKO_MAXSLOT_GUARD], w[SKO_MAXSLOT_GUARD];
                int flips[SKO_MAXSLOT_GUARD][2], nflip[SKO_MAXSLOT_GUARD];
                star_candidates(&c, s, h, leaf, sites, dE, flips, nflip);
                const double m = min_dE(dE, K + 1);
                double tot = 0.0;
                for (int j = 0; j <= K; ++j) {
                    const int centre = is_centre_slot(j, leaf);
                    w[j] = (weight_mode == 1) ? (double)weight_int(&c, dE[j], m, centre)
                                              : weight_dbl(&c, dE[j], m, centre);
                    tot += w[j];
                }
                for (int j = 0; j <= K; ++j) {
                    uint32_t y = x;
                    for (int f = 0; f < nflip[j]; ++f) y ^= 1u << flips[j][f];
                    row[y] += proot * ptup * w[j] / tot;
                }
                /* odometer over the K-tuple of sites */
                for (int d = 1; d <= K; ++d) {
                    if (++sites[d] < (uint32_t)N) break;
                    sites[d] = 0;
                }
            }
        }
    }
    ctx_free(&c);
    return 0;
}

/* sko_transition_matrix_p with the uniform root (p_center = 0). */
int sko_transition_matrix(int N, int kind, const void* J, double scale, int rule, int K,
                          double beta, int root_mode, int weight_mode, double* P) {
    return sko_transition_matrix_p(N, kind, J, scale, rule, K, beta, root_mode, weight_mode, 0.0, P);
}

/* ------------------------------------------------------------------ */
/* Deeper graphs (App. B): trees populated from a root                  */
/* ------------------------------------------------------------------ */
/*
 * Templates, nodes numbered 0..V-1 with a parent for every node v >= 1:
 *   SKO_TREE: the full k-ary tree of depth D (App. B.2, populating process),
 *             V = (k^(D+1) - 1)/(k - 1), parent(v) = (v - 1)/k; uniform root.
 *   SKO_LINE: the line of L nodes (App. B.1, addition process), parent(v) =
 *             v - 1.  Adding each of the L - 1 new nodes at either end with
 *             probability 1/2 leaves the starting configuration at position v
 *             with probability binom(L-1, v)/2^(L-1) (Eq. eq_create_line_graph,
 *             read with L - 1 additions for L nodes, C13), which is the
 *             populating process of App. B.2 on the line with that root
 *             distribution.
 * With the root at position r (the current state c), every other node is
 * generated from its neighbour toward r by flipping the site drawn for the
 * edge between them, so P_gen(T|c at r) = p_r N^-(V-1) and the node rule
 * (Eq. eq_det_balance_graph_solution) weights node v by P_eq(c_v) p_v.
 *
 * Root distribution and node factors in integers: F_v = 2^20 for the tree;
 * for the line F_v = round(2^20 c_v / max_u c_u) with c_0 = 1 and
 * c_(v+1) = c_v (L-1-v)/(v+1) evaluated in double precision in this order
 * (c_v = binom(L-1, v)).  The root is the first v whose inclusive prefix
 * sum of F exceeds floor(U0 sum(F) / 2^64); node weights are
 * floor(W[(dE - m)/2] F_v / 2^20) (+-J) or exp(-beta (dE - m)) F_v / 2^20
 * (Gaussian); root probabilities and factors are then exactly proportional.
 * Nodes whose factor rounds to 0 are never the root and never chosen.
 *
 * Draws of step t: block 0 as for the star (U0 root, U1 node); the site of
 * the edge between v and parent(v) is site_v = floor(w N / 2^32), word
 * (v-1) % 4 of block 1 + (v-1)/4, v = 1..V-1.  The node chosen is the first
 * in node order whose inclusive weight prefix exceeds u, as for the star.
 */
#define SKO_TREE 1
#define SKO_LINE 2
#define SKO_MAX_V 8192

typedef struct {
    int type, V, k;
    uint64_t* F;
    uint64_t Fsum;
} sko_graph;

static int graph_setup(sko_graph* g, int type, int k, int D, int L) {
    memset(g, 0, sizeof(*g));
    if (type == SKO_TREE) {
        if (k < 2 || D < 1) return -1;
        long long V = 1, lvl = 1;
        for (int d = 1; d <= D; ++d) {
            lvl *= k;
            V += lvl;
            if (V > SKO_MAX_V) return -1;
        }
        g->V = (int)V;
    } else if (type == SKO_LINE) {
        if (L < 2 || L > SKO_MAX_V) return -1;
        g->V = L;
    } else {
        return -1;
    }
    g->type = type;
    g->k = k;
    g->F = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)g->V);
    if (!g->F) return -2;
    if (type == SKO_TREE) {
        for (int v = 0; v < g->V; ++v) g->F[v] = (uint64_t)1 << 20;
    } else {
        double* cv = (double*)malloc(sizeof(double) * (size_t)g->V);
        if (!cv) return -2;
        const int n = g->V - 1;
        double cmax = 1.0;
        cv[0] = 1.0;
        for (int v = 0; v < n; ++v) {
            cv[v + 1] = cv[v] * (double)(n - v) / (double)(v + 1);
            if (cv[v + 1] > cmax) cmax = cv[v + 1];
        }
        for (int v = 0; v < g->V; ++v) g->F[v] = (uint64_t)(cv[v] / cmax * 1048576.0 + 0.5);
        free(cv);
    }
    g->Fsum = 0;
    for (int v = 0; v < g->V; ++v) g->Fsum += g->F[v];
    return 0;
}

static void graph_free(sko_graph* g) { free(g->F); }

static int tparent(const sko_graph* g, int v) { return g->type == SKO_TREE ? (v - 1) / g->k : v - 1; }

static int tdepth(const sko_graph* g, int v) {
    int d = 0;
    while (v > 0) { v = tparent(g, v); ++d; }
    return d;
}

/* Edges (child node ids) on the template path between a and b, in the order
   a -> ... -> lca -> ... -> b, into edges[] (capacity V); down[] (capacity
   V) is scratch.  Returns their number. */
static int tpath(const sko_graph* g, int a, int b, int* edges, int* down) {
    int da = tdepth(g, a), db = tdepth(g, b);
    int n = 0, nd = 0;
    while (da > db) { edges[n++] = a; a = tparent(g, a); --da; }
    while (db > da) { down[nd++] = b; b = tparent(g, b); --db; }
    while (a != b) {
        edges[n++] = a; a = tparent(g, a);
        down[nd++] = b; b = tparent(g, b);
    }
    for (int i = nd - 1; i >= 0; --i) edges[n++] = down[i];
    return n;
}

static int graph_root(const sko_graph* g, uint64_t U0) {
    const uint64_t x = range64(U0, g->Fsum);
    uint64_t acc = 0;
    for (int v = 0; v < g->V; ++v) {
        acc += g->F[v];
        if (acc > x) return v;
    }
    return g->V - 1;
}

/* Energy change of flipping the sites x[0..n-1] in order (repeats cancel),
   from (s, h), using scratch copies s2/h2.  Fields updated as in flip_spin. */
static double flips_dE(const sko_ctx* c, const int8_t* s, const double* h, const uint32_t* x, int n,
                       int8_t* s2, double* h2) {
    memcpy(s2, s, (size_t)c->N);
    memcpy(h2, h, sizeof(double) * (size_t)c->N);
    double dE = 0.0;
    for (int i = 0; i < n; ++i) {
        const int y = (int)x[i];
        dE += 2.0 * (double)s2[y] * h2[y];
        flip_spin(c, s2, h2, y);
    }
    return dE;
}

/* Node weights; F = the node's factor (2^20 = 1). */
static uint64_t graph_weight_int(const sko_ctx* c, uint64_t F, double dE, double m) {
    long long d = (long long)llround((dE - m) * 0.5);
    uint64_t w = (d < c->wlen) ? c->W[d] : 0u;
    return (uint64_t)(((unsigned __int128)w * (unsigned __int128)F) >> 20);
}
static double graph_weight_dbl(const sko_ctx* c, uint64_t F, double dE, double m) {
    if (!F) return 0.0;
    return exp(-c->beta * c->scale * (dE - m)) * ldexp((double)F, -20);
}

/*
 * One step on a graph: root r from U0, the V-1 edge sites, every node's
 * energy change relative to the root (its path's flips), the node chosen
 * with probability ~ P_eq(c_v) F_v, and the move (the chosen path's flips).
 * forced/own/Pout/uout as for chain_step.  Returns 1 if the state changed.
 */
static int graph_step(const sko_ctx* c, const sko_graph* g, uint32_t chain, uint64_t t, int8_t* s, double* h,
                      int forced, int* own, double* Pout, double* uout, uint32_t* site, double* dE,
                      int8_t* s2, double* h2, int* edges, int* down, uint32_t* xs) {
    uint32_t w0[4];
    draw_block(c->seed, c->stream, 0u, chain, t, 0u, w0);
    const uint64_t U0 = ((uint64_t)w0[1] << 32) | w0[0];
    const uint64_t U1 = ((uint64_t)w0[3] << 32) | w0[2];
    const int V = g->V;
    const int r = graph_root(g, U0);
    for (int v = 1; v < V; ++v) {
        uint32_t wb[4];
        draw_block(c->seed, c->stream, 0u, chain, t, (uint32_t)(1 + (v - 1) / 4), wb);
        site[v] = range32(wb[(v - 1) % 4], (uint32_t)c->N);
    }
    double m = 0.0;
    for (int v = 0; v < V; ++v) {
        const int n = tpath(g, r, v, edges, down);
        for (int i = 0; i < n; ++i) xs[i] = site[edges[i]];
        dE[v] = flips_dE(c, s, h, xs, n, s2, h2);
        if (g->F[v] && dE[v] < m) m = dE[v];
    }
    /* weights in node order, first inclusive prefix above u */
    int j = -1;
    if (c->kind == SKO_PM1) {
        uint64_t tot = 0;
        for (int v = 0; v < V; ++v) tot += graph_weight_int(c, g->F[v], dE[v], m);
        const uint64_t u = range64(U1, tot);
        uint64_t acc = 0;
        for (int v = 0; v < V; ++v) {
            acc += graph_weight_int(c, g->F[v], dE[v], m);
            if (Pout) Pout[v] = (double)acc;
            if (j < 0 && acc > u) j = v;
        }
        if (uout) *uout = ldexp((double)U1, -64) * (double)tot;
    } else {
        double tot = 0.0;
        for (int v = 0; v < V; ++v) tot += graph_weight_dbl(c, g->F[v], dE[v], m);
        const double u = (double)(U1 >> 40) * ldexp(1.0, -24) * tot;
        double acc = 0.0;
        for (int v = 0; v < V; ++v) {
            acc += graph_weight_dbl(c, g->F[v], dE[v], m);
            if (Pout) Pout[v] = acc;
            if (j < 0 && acc > u) j = v;
        }
        if (j < 0)
            for (int v = V - 1; v >= 0; --v)
                if (graph_weight_dbl(c, g->F[v], dE[v], m) > 0.0) { j = v; break; }
        if (uout) *uout = u;
    }
    if (own) *own = j;
    if (forced >= 0) j = forced;
    const int n = tpath(g, r, j, edges, down);
    for (int i = 0; i < n; ++i) flip_spin(c, s, h, (int)site[edges[i]]);
    /* changed iff some site flips an odd number of times */
    int changed = 0;
    for (int i = 0; i < n && !changed; ++i) {
        int cnt = 0;
        for (int q = 0; q < n; ++q) cnt += site[edges[q]] == site[edges[i]];
        changed = cnt & 1;
    }
    return changed;
}

/*
 * Runs chains on a graph (graph_type SKO_TREE with arity/depth, or SKO_LINE
 * with `line_nodes`); outputs as sko_run (no overlap, no node-weighted
 * records).  trace receives the node chosen at each step.
 */
int sko_run_graph(int N, int kind, const void* J, double scale, int graph_type, int arity, int depth,
                  int line_nodes, double beta, uint64_t seed, uint32_t stream, uint32_t chain0,
                  uint32_t nchains, const int8_t* init_spins, uint64_t nsteps, uint32_t record_every,
                  double* rec_E, uint32_t* rec_acc, int8_t* final_spins, double* final_E, int32_t* trace) {
    sko_graph g;
    int rc = graph_setup(&g, graph_type, arity, depth, line_nodes);
    if (rc) return rc;
    sko_ctx c;
    rc = ctx_init(&c, N, kind, J, scale, SKO_MCMCMC, 1, beta, seed, stream, 0.0);
    if (rc) { graph_free(&g); return rc; }
    int8_t* s = (int8_t*)malloc((size_t)N);
    int8_t* s2 = (int8_t*)malloc((size_t)N);
    double* h = (double*)malloc(sizeof(double) * (size_t)N);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)N);
    uint32_t* site = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)g.V);
    double* dE = (double*)malloc(sizeof(double) * (size_t)g.V);
    int* edges = (int*)malloc(sizeof(int) * (size_t)g.V);
    int* down = (int*)malloc(sizeof(int) * (size_t)g.V);
    uint32_t* xs = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)g.V);
    if (!s || !s2 || !h || !h2 || !site || !dE || !edges || !down || !xs) { rc = -2; goto done; }
    for (uint32_t ci = 0; ci < nchains; ++ci) {
        const uint32_t chain = chain0 + ci;
        if (init_spins) memcpy(s, init_spins + (size_t)ci * N, (size_t)N);
        else sko_init_spins(seed, stream, chain, N, s);
        sko_fields(N, kind, J, s, h);
        uint32_t acc = 0;
        for (uint64_t t = 0; t < nsteps; ++t) {
            int own = -1;
            acc += (uint32_t)graph_step(&c, &g, chain, t, s, h, -1, &own, NULL, NULL, site, dE, s2, h2,
                                        edges, down, xs);
            if (trace) trace[(size_t)ci * nsteps + t] = own;
            if (record_every && ((t + 1) % record_every) == 0) {
                const uint64_t r = (t + 1) / record_every - 1;
                if (rec_E) rec_E[r * nchains + ci] = sko_energy(N, kind, J, scale, s);
                if (rec_acc) rec_acc[r * nchains + ci] = acc;
                acc = 0;
            }
        }
        if (final_spins) memcpy(final_spins + (size_t)ci * N, s, (size_t)N);
        if (final_E) final_E[ci] = sko_energy(N, kind, J, scale, s);
    }
done:
    free(s); free(s2); free(h); free(h2); free(site); free(dE); free(edges); free(down); free(xs);
    ctx_free(&c);
    graph_free(&g);
    return rc;
}

/* One chain's own trajectory on a graph with each step's node choice, draw
 * and inclusive prefix sums (P[t * V + v]), as sko_run_detail. */
int sko_run_graph_detail(int N, int kind, const void* J, double scale, int graph_type, int arity, int depth,
                         int line_nodes, double beta, uint64_t seed, uint32_t stream, uint32_t chain,
                         const int8_t* init_spins, uint64_t nsteps, int32_t* own, double* u, double* P) {
    sko_graph g;
    int rc = graph_setup(&g, graph_type, arity, depth, line_nodes);
    if (rc) return rc;
    sko_ctx c;
    rc = ctx_init(&c, N, kind, J, scale, SKO_MCMCMC, 1, beta, seed, stream, 0.0);
    if (rc) { graph_free(&g); return rc; }
    const int V = g.V;
    int8_t* s = (int8_t*)malloc((size_t)N);
    int8_t* s2 = (int8_t*)malloc((size_t)N);
    double* h = (double*)malloc(sizeof(double) * (size_t)N);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)N);
    uint32_t* site = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)V);
    double* dE = (double*)malloc(sizeof(double) * (size_t)V);
    int* edges = (int*)malloc(sizeof(int) * (size_t)V);
    int* down = (int*)malloc(sizeof(int) * (size_t)V);
    uint32_t* xs = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)V);
    if (!s || !s2 || !h || !h2 || !site || !dE || !edges || !down || !xs) { rc = -2; goto done; }
    if (init_spins) memcpy(s, init_spins, (size_t)N);
    else sko_init_spins(seed, stream, chain, N, s);
    sko_fields(N, kind, J, s, h);
    for (uint64_t t = 0; t < nsteps; ++t) {
        int o = -1;
        double uu = 0.0;
        graph_step(&c, &g, chain, t, s, h, -1, &o, P + (size_t)t * (size_t)V, &uu, site, dE, s2, h2, edges,
                   down, xs);
        own[t] = o;
        u[t] = uu;
    }
done:
    free(s); free(s2); free(h); free(h2); free(site); free(dE); free(edges); free(down); free(xs);
    ctx_free(&c);
    graph_free(&g);
    return rc;
}

/* Decision replay on a graph (see sko_replay). */
long long sko_replay_graph(int N, int kind, const void* J, double scale, int graph_type, int arity, int depth,
                           int line_nodes, double beta, uint64_t seed, uint32_t stream, uint32_t chain,
                           const int8_t* init_spins, uint64_t nsteps, const int32_t* slots, double tol,
                           long long* n_disagree, long long* first_bad, int8_t* final_spins, double* final_E) {
    sko_graph g;
    int rc = graph_setup(&g, graph_type, arity, depth, line_nodes);
    if (rc) return rc;
    sko_ctx c;
    rc = ctx_init(&c, N, kind, J, scale, SKO_MCMCMC, 1, beta, seed, stream, 0.0);
    if (rc) { graph_free(&g); return rc; }
    const int V = g.V;
    int8_t* s = (int8_t*)malloc((size_t)N);
    int8_t* s2 = (int8_t*)malloc((size_t)N);
    double* h = (double*)malloc(sizeof(double) * (size_t)N);
    double* h2 = (double*)malloc(sizeof(double) * (size_t)N);
    uint32_t* site = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)V);
    double* dE = (double*)malloc(sizeof(double) * (size_t)V);
    double* P = (double*)malloc(sizeof(double) * (size_t)V);
    int* edges = (int*)malloc(sizeof(int) * (size_t)V);
    int* down = (int*)malloc(sizeof(int) * (size_t)V);
    uint32_t* xs = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)V);
    long long bad = 0, dis = 0, first = -1;
    if (!s || !s2 || !h || !h2 || !site || !dE || !P || !edges || !down || !xs) { bad = -2; goto done; }
    if (init_spins) memcpy(s, init_spins, (size_t)N);
    else sko_init_spins(seed, stream, chain, N, s);
    sko_fields(N, kind, J, s, h);
    for (uint64_t t = 0; t < nsteps; ++t) {
        const int gs = slots[t];
        if (gs < 0 || gs >= V) { bad++; if (first < 0) first = (long long)t; break; }
        int own = -1;
        double u = 0.0;
        graph_step(&c, &g, chain, t, s, h, gs, &own, P, &u, site, dE, s2, h2, edges, down, xs);
        if (own != gs) {
            dis++;
            const double PK = P[V - 1];
            const double lo = gs == 0 ? 0.0 : P[gs - 1];
            const double hi = P[gs];
            if (!(u >= lo - tol * PK && u < hi + tol * PK)) { bad++; if (first < 0) first = (long long)t; }
        }
    }
    if (final_spins) memcpy(final_spins, s, (size_t)N);
    if (final_E) *final_E = sko_energy(N, kind, J, scale, s);
    if (n_disagree) *n_disagree = dis;
    if (first_bad) *first_bad = first;
done:
    free(s); free(s2); free(h); free(h2); free(site); free(dE); free(P); free(edges); free(down); free(xs);
    ctx_free(&c);
    graph_free(&g);
    return bad;
}

/*
 * Exact one-step transition matrix on a graph by enumeration (small N and
 * V: every root with probability F_r / sum F and every (V-1)-tuple of edge
 * sites).  weight_mode 0: fp64 weights; 1: the +-J integer weights.
 * root_weights 0 drops the node factors F_v from the weights while keeping
 * the root distribution (the negative control for the line).
 */
int sko_transition_matrix_graph(int N, int kind, const void* J, double scale, int graph_type, int arity,
                                int depth, int line_nodes, double beta, int weight_mode, int root_weights,
                                double* P) {
    if (N < 1 || N > 10) return -1;
    sko_graph g;
    int rc = graph_setup(&g, graph_type, arity, depth, line_nodes);
    if (rc) return rc;
    if (g.V > 8) { graph_free(&g); return -1; }
    sko_ctx c;
    rc = ctx_init(&c, N < 2 ? 2 : N, kind, J, scale, SKO_MCMCMC, 1, beta, 0, 0, 0.0);
    c.N = N;
    if (rc) { graph_free(&g); return rc; }
    if (weight_mode == 1 && kind != SKO_PM1) { ctx_free(&c); graph_free(&g); return -1; }
    const int V = g.V;
    const uint32_t n = 1u << N;
    memset(P, 0, sizeof(double) * (size_t)n * n);
    int8_t s[12], s2[12];
    double h[12], h2[12];
    uint32_t site[8], xs[8];
    double dE[8], w[8];
    int edges[8], down[8];
    long long ntup = 1;
    for (int e = 1; e < V; ++e) ntup *= N;
    for (uint32_t x = 0; x < n; ++x) {
        spins_of(x, N, s);
        sko_fields(N, kind, J, s, h);
        double* row = P + (size_t)x * n;
        for (int r = 0; r < V; ++r) {
            const double pr = (double)g.F[r] / (double)g.Fsum;
            if (pr == 0.0) continue;
            for (int e = 0; e < V; ++e) site[e] = 0;
            for (long long tup = 0; tup < ntup; ++tup) {
                double m = 0.0;
                for (int v = 0; v < V; ++v) {
                    const int ne = tpath(&g, r, v, edges, down);
                    for (int i = 0; i < ne; ++i) xs[i] = site[edges[i]];
                    dE[v] = flips_dE(&c, s, h, xs, ne, s2, h2);
                    if (g.F[v] && dE[v] < m) m = dE[v];
                }
                double tot = 0.0;
                for (int v = 0; v < V; ++v) {
                    const uint64_t F = root_weights ? g.F[v] : (g.F[v] ? ((uint64_t)1 << 20) : 0u);
                    w[v] = (weight_mode == 1) ? (double)graph_weight_int(&c, F, dE[v], m)
                                              : graph_weight_dbl(&c, F, dE[v], m);
                    tot += w[v];
                }
                for (int v = 0; v < V; ++v) {
                    if (w[v] == 0.0) continue;
                    const int ne = tpath(&g, r, v, edges, down);
                    uint32_t y = x;
                    for (int i = 0; i < ne; ++i) y ^= 1u << site[edges[i]];
                    row[y] += pr * (w[v] / tot) / (double)ntup;
                }
                for (int e = 1; e < V; ++e) {  /* odometer over the edge sites */
                    if (++site[e] < (uint32_t)N) break;
                    site[e] = 0;
                }
            }
        }
    }
    ctx_free(&c);
    graph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Set generation probabilities (App. D.1, D.2)                         */
/* ------------------------------------------------------------------ */
/*
 * The process of App. D.1: from a set T ⊊ S, repeatedly choose a parent
 * uniformly from the current set and generate a new element with
 * P_gen(e | parent), until the set is S.  For the n elements of S, with
 * P[e*n + p] = P_gen(e | p), and every M ⊆ S given as a bit mask,
 * Pt(M) = P_gen(S | S \ M) (Eq. eq_def_rec_P): the probability that the
 * additions, in any order, are exactly the elements of M.  Pt(empty) = 1;
 * Pt(S) (no starting element) is 0 by convention.
 *
 * sko_setgen_bruteforce: the sum over every order of M's elements of the
 * product of the per-addition probabilities (1/|current|) sum_{p in current}
 * P_gen(e | p) -- the definition, by enumeration (|M|! orders).
 */
static double setgen_orders(int n, const double* P, uint32_t cur, uint32_t left) {
    if (!left) return 1.0;
    const int ncur = __builtin_popcount(cur);
    double tot = 0.0;
    for (int e = 0; e < n; ++e) {
        if (!((left >> e) & 1u)) continue;
        double pe = 0.0;
        for (int p = 0; p < n; ++p)
            if ((cur >> p) & 1u) pe += P[(size_t)e * n + p];
        pe /= (double)ncur;
        tot += pe * setgen_orders(n, P, cur | (1u << e), left & ~(1u << e));
    }
    return tot;
}

double sko_setgen_bruteforce(int n, const double* P, uint32_t M) {
    if (n < 1 || n > 12) return -1.0;
    const uint32_t all = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
    if ((M & ~all) != 0u) return -1.0;
    if (M == all) return 0.0;
    return setgen_orders(n, P, all & ~M, M);
}

/*
 * sko_setgen_dp: every Pt(M) by the recursion on the first addition (App. D.2,
 * Eq. eq_rec_set_mul_el as read for the process above): the first added
 * element e' of M is generated from a parent in the current set S \ M,
 *   Pt(M) = (1/|S \ M|) sum_{e' in M} [sum_{p in S \ M} P_gen(e' | p)] Pt(M \ {e'}),
 * taken over masks in increasing order (M \ {e'} < M).  n <= 26.
 */
int sko_setgen_dp(int n, const double* P, double* out) {
    if (n < 1 || n > 26) return -1;
    const uint32_t all = (1u << n) - 1u;
    out[0] = 1.0;
    for (uint32_t M = 1; M <= all; ++M) {
        if (M == all) { out[M] = 0.0; continue; }
        const uint32_t cur = all & ~M;
        double tot = 0.0;
        for (int e = 0; e < n; ++e) {
            if (!((M >> e) & 1u)) continue;
            double a = 0.0;
            for (int p = 0; p < n; ++p)
                if ((cur >> p) & 1u) a += P[(size_t)e * n + p];
            tot += a * out[M & ~(1u << e)];
        }
        out[M] = tot / (double)__builtin_popcount(cur);
    }
    return 0;
}

/*
 * sko_setgen_cumulative: the same Pt(M) by the paper's cumulative form
 * (App. D.2, Eq. eq_rec_set_short): a table c(M, e) = sum_{p in S \ M}
 * P_gen(e | p) for every e in M, built from smaller sets --
 *   c({e}, e) = sum_{p != e} P_gen(e | p),
 *   c(M, e)   = c(M \ {f}, e) - P_gen(e | f) for an f in M, f != e (the
 *               lowest one): moving f from S \ M into M removes its term --
 * then Pt(M) = (1/|S \ M|) sum_{e in M} c(M, e) Pt(M \ {e}), O(n 2^n) work
 * (the printed definition garbles the orientation of P_gen and the sets
 * summed over; this is the reading under which it equals the recursion).
 * n <= 20 (a table of n 2^n doubles).
 */
int sko_setgen_cumulative(int n, const double* P, double* out) {
    if (n < 1 || n > 20) return -1;
    const uint32_t all = (1u << n) - 1u;
    double* c = (double*)malloc(sizeof(double) * (size_t)n << n);
    if (!c) return -2;
    out[0] = 1.0;
    for (uint32_t M = 1; M <= all; ++M) {
        if (M == all) { out[M] = 0.0; continue; }
        double tot = 0.0;
        for (int e = 0; e < n; ++e) {
            if (!((M >> e) & 1u)) continue;
            const uint32_t rest = M & ~(1u << e);
            double ce;
            if (!rest) {
                ce = 0.0;
                for (int p = 0; p < n; ++p)
                    if (p != e) ce += P[(size_t)e * n + p];
            } else {
                const int f = __builtin_ctz(rest);
                ce = c[(size_t)(M & ~(1u << f)) * n + e] - P[(size_t)e * n + f];
            }
            c[(size_t)M * n + e] = ce;
            tot += ce * out[rest];
        }
        out[M] = tot / (double)(n - __builtin_popcount(M));
    }
    free(c);
    return 0;
}
