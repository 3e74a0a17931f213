/*
 * pt_oracle.c -- plain CPU oracle for Metropolis-Hastings with Parallel Tempering on the
 * periodic two-dimensional Ising model (arXiv 2512.03825: Sec. 2.1 Eq. 1, Sec. 2.2 Eqs. 2-3,
 * Sec. 3 replica scheduling and swap rule).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct definition that the
 * CUDA library is compared against bit for bit. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it. It shares no code, header or table generator with
 * the CUDA library: Philox, the quantiser and both threshold formulas are written here again.
 *
 * State: one int8 spin (+1 / -1) per site and per replica slot, spin[r][y][x]. Replica r
 * keeps its configuration in slot r for the whole run and samples at temperature index
 * temp_of_slot[r] (inverse temperature beta[temp_of_slot[r]]); slot_of_temp[] is the inverse
 * permutation. An accepted exchange between temperatures k and k+1 swaps their slots in these
 * two maps, which is the same Markov chain as swapping the two configurations (Sec. 2.1).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = the 64-bit seed.
 *   initial spin  (site i, slot r):           ctr = {i, 0, r>>2, TAG_INIT}                word r&3, bit 31
 *   spin update   (site i, slot r, sweep t):  ctr = {i, lo32(t), r>>2, TAG_SPIN|hi32(t)<<8} word r&3
 *   exchange      (pair k, exchange e):       ctr = {k, lo32(e), 0, TAG_EXCH|hi32(e)<<8}   word 0
 *   single flip   (slot r, iteration i):      ctr = {lo32(i), r, 0, TAG_FLIP|hi32(i)<<8}
 *                 word 0 picks the site floor(u0 * L^2 / 2^32), word 1 decides acceptance
 * The paper fixes no generator; the counter layout is this framework's choice and the CUDA
 * library uses the same one. Nothing here is blocked, fused or reordered for speed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

#define TAG_SPIN 0u
#define TAG_EXCH 1u
#define TAG_INIT 2u
#define TAG_FLIP 3u

/* ---------------------------------------------------------------------------------------
 * Philox4x32-10, written from the definition in Salmon et al., "Parallel Random Numbers: As
 * Easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplications whose halves are
 * xored with the other counter words and the round key; the key is bumped by the Weyl
 * constants between rounds.
 * ------------------------------------------------------------------------------------- */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                            int word) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[word];
}

/* ---------------------------------------------------------------------------------------
 * Energy quantisation. Eq. 3 is evaluated in integers: s is the smallest integer in
 * 1..1000 for which s*J and s*h are both within 1e-9 of integers; J_int = round(s*J),
 * h_int = round(s*h), and s*E(sigma) = E_int(sigma) exactly. (The paper works in floating
 * point and says nothing about this; the integer form makes every decision exact.)
 * ------------------------------------------------------------------------------------- */
int oracle_quantise(double J, double h, int64_t* s_out, int64_t* J_int, int64_t* h_int) {
    if (!isfinite(J) || !isfinite(h)) return ORACLE_EINVAL;
    for (int64_t s = 1; s <= 1000; ++s) {
        double sj = (double)s * J, sh = (double)s * h;
        double rj = nearbyint(sj), rh = nearbyint(sh);
        if (fabs(sj - rj) <= 1e-9 && fabs(sh - rh) <= 1e-9) {
            if (fabs(rj) > 1048576.0 || fabs(rh) > 1048576.0) return ORACLE_EINVAL;
            *s_out = s;
            *J_int = (int64_t)rj;
            *h_int = (int64_t)rh;
            return ORACLE_OK;
        }
    }
    return ORACLE_EINVAL;
}

/* Metropolis acceptance threshold (Eq. 1 with the Boltzmann target of Eq. 2, k_B = 1):
 * a trial that raises the energy by dE (= dE_int / s) is accepted with probability
 * exp(-beta * dE). With a 32-bit uniform integer u the test is u < T where
 * T = floor(2^32 * exp(-(beta * dE_int) / s)). dE_int <= 0 is always accepted: T = 2^32.
 * Returned in [0, 2^32]. */
uint64_t oracle_spin_threshold(double beta, int64_t dE_int, int64_t s) {
    if (dE_int <= 0) return 4294967296ull;
    double x = (beta * (double)dE_int) / (double)s;
    return (uint64_t)floor(4294967296.0 * exp(-x));
}

/* Replica-exchange threshold (Sec. 3, the Barker-form swap probability
 * e^{x} / (1 + e^{x}) with x = (beta_lo - beta_hi)(E_lo - E_hi), which equals
 * 1 / (1 + e^{y}) with y = (beta_hi - beta_lo) * n / s, n = E_int(lo) - E_int(hi)).
 * Accept iff u < S. Products y above 44 are always rejected (S = 0) and below -44 always
 * accepted (S = 2^32); in between S = floor(2^32 / (1 + exp(y))). Returned in [0, 2^32]. */
uint64_t oracle_swap_threshold(double beta_lo, double beta_hi, int64_t n, int64_t s) {
    double y = ((beta_hi - beta_lo) * (double)n) / (double)s;
    if (y > 44.0) return 0;
    if (y < -44.0) return 4294967296ull;
    return (uint64_t)floor(4294967296.0 / (1.0 + exp(y)));
}

/* The Metropolis-form swap probability min(1, e^{x}) = min(1, e^{-y}), the option next to the
 * Barker form (the paper's rule is Barker; Metropolis is the usual alternative in the
 * parallel-tempering literature). Accept iff u < S: S = 2^32 for y <= 0, 0 for y > 44, and
 * floor(2^32 * exp(-y)) in between. Returned in [0, 2^32]. */
uint64_t oracle_swap_threshold_metropolis(double beta_lo, double beta_hi, int64_t n,
                                          int64_t s) {
    double y = ((beta_hi - beta_lo) * (double)n) / (double)s;
    if (y <= 0.0) return 4294967296ull;
    if (y > 44.0) return 0;
    return (uint64_t)floor(4294967296.0 * exp(-y));
}

#define ORACLE_SWAP_BARKER 0
#define ORACLE_SWAP_METROPOLIS 1

/* --------------------------------------------------------------------------------------- */

typedef struct oracle_pt {
    int L, R;
    int swap_rule;    /* ORACLE_SWAP_BARKER or ORACLE_SWAP_METROPOLIS */
    double* beta;     /* [R], by temperature index */
    int64_t s, J_int, h_int;
    uint64_t seed;
    int8_t* spin;     /* [R][L][L], by replica slot */
    int32_t* temp_of_slot;  /* [R] */
    int32_t* slot_of_temp;  /* [R] */
    uint64_t t, e;    /* sweeps done, exchanges done */
    uint64_t it;      /* single-spin-flip iterations done */
    uint64_t* attempted; /* [R-1] */
    uint64_t* accepted;  /* [R-1] */
} oracle_pt;

static int threads_wanted = 1;
void oracle_set_threads(int n) { threads_wanted = n < 1 ? 1 : n; }
int oracle_get_threads(void) { return threads_wanted; }

static int8_t* lattice(const oracle_pt* p, int r) { return p->spin + (size_t)r * p->L * p->L; }

void oracle_destroy(oracle_pt* p) {
    if (!p) return;
    free(p->beta); free(p->spin); free(p->temp_of_slot); free(p->slot_of_temp);
    free(p->attempted); free(p->accepted);
    free(p);
}

/* Initialisation phase (Sec. 3: build the data structures): every spin of every replica is
 * drawn uniformly from {-1, +1} with the TAG_INIT stream; slot r starts at temperature r. */
int oracle_create_ex(int L, const double* betas, int R, double J, double h, uint64_t seed,
                     int swap_rule, oracle_pt** out) {
    *out = NULL;
    if (L < 4 || L > 16384 || (L & 1) || R < 1 || R > 2048 || !betas) return ORACLE_EINVAL;
    if (swap_rule != ORACLE_SWAP_BARKER && swap_rule != ORACLE_SWAP_METROPOLIS)
        return ORACLE_EINVAL;
    for (int k = 0; k < R; ++k)
        if (!isfinite(betas[k]) || betas[k] < 0.0) return ORACLE_EINVAL;
    oracle_pt* p = (oracle_pt*)calloc(1, sizeof(oracle_pt));
    if (!p) return ORACLE_ENOMEM;
    if (oracle_quantise(J, h, &p->s, &p->J_int, &p->h_int) != ORACLE_OK) { free(p); return ORACLE_EINVAL; }
    p->L = L; p->R = R; p->seed = seed; p->swap_rule = swap_rule;
    p->beta = (double*)malloc(sizeof(double) * R);
    p->spin = (int8_t*)malloc((size_t)R * L * L);
    p->temp_of_slot = (int32_t*)malloc(sizeof(int32_t) * R);
    p->slot_of_temp = (int32_t*)malloc(sizeof(int32_t) * R);
    p->attempted = (uint64_t*)calloc(R, sizeof(uint64_t));
    p->accepted = (uint64_t*)calloc(R, sizeof(uint64_t));
    if (!p->beta || !p->spin || !p->temp_of_slot || !p->slot_of_temp || !p->attempted ||
        !p->accepted) {
        oracle_destroy(p); return ORACLE_ENOMEM;
    }
    memcpy(p->beta, betas, sizeof(double) * R);
    for (int r = 0; r < R; ++r) {
        p->temp_of_slot[r] = r;
        p->slot_of_temp[r] = r;
        int8_t* sp = lattice(p, r);
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                uint32_t i = (uint32_t)(y * L + x);
                uint32_t u = philox_word(seed, i, 0u, (uint32_t)(r >> 2), TAG_INIT, r & 3);
                sp[y * L + x] = (u >> 31) ? (int8_t)1 : (int8_t)-1;
            }
    }
    *out = p;
    return ORACLE_OK;
}

int oracle_create(int L, const double* betas, int R, double J, double h, uint64_t seed,
                  oracle_pt** out) {
    return oracle_create_ex(L, betas, R, J, h, seed, ORACLE_SWAP_BARKER, out);
}

/* Eq. 3 in integers: E_int = h_int * sum_i sigma_i - J_int * sum_<ij> sigma_i sigma_j, each of
 * the 2 L^2 nearest-neighbour bonds of the periodic lattice counted once (right and down).
 * Of the configuration held in slot r. */
static int64_t slot_energy_int(const oracle_pt* p, int r) {
    const int L = p->L;
    const int8_t* sp = lattice(p, r);
    int64_t field = 0, bonds = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int s = sp[y * L + x];
            int right = sp[y * L + (x + 1) % L];
            int down = sp[((y + 1) % L) * L + x];
            field += s;
            bonds += s * right + s * down;
        }
    return p->h_int * field - p->J_int * bonds;
}

static int64_t slot_magnetisation(const oracle_pt* p, int r) {
    const int8_t* sp = lattice(p, r);
    int64_t m = 0;
    for (size_t i = 0; i < (size_t)p->L * p->L; ++i) m += sp[i];
    return m;
}

/* Energy and magnetisation of the configuration currently at temperature index k. */
int64_t oracle_energy_int(const oracle_pt* p, int k) { return slot_energy_int(p, p->slot_of_temp[k]); }
int64_t oracle_magnetisation(const oracle_pt* p, int k) {
    return slot_magnetisation(p, p->slot_of_temp[k]);
}

/* One single-spin Metropolis trial at site (x, y) of the replica in slot r in sweep t
 * (Sec. 2.1, Eq. 1): the trial state flips sigma; Delta E from Eq. 3 is
 * 2 sigma (J * sum_nb sigma_nb - h); the trial is accepted when u < T(beta, Delta E) with beta
 * the inverse temperature the slot currently runs at. */
static void metropolis_site(oracle_pt* p, int r, int x, int y) {
    const int L = p->L;
    int8_t* sp = lattice(p, r);
    int s = sp[y * L + x];
    int nb = sp[y * L + (x + 1) % L] + sp[y * L + (x + L - 1) % L] +
             sp[((y + 1) % L) * L + x] + sp[((y + L - 1) % L) * L + x];
    int64_t dE_int = 2 * (int64_t)s * (p->J_int * nb - p->h_int);
    if (dE_int <= 0) { sp[y * L + x] = (int8_t)-s; return; }
    uint32_t i = (uint32_t)(y * L + x);
    uint32_t u = philox_word(p->seed, i, (uint32_t)p->t, (uint32_t)(r >> 2),
                             TAG_SPIN | ((uint32_t)(p->t >> 32) << 8), r & 3);
    double beta = p->beta[p->temp_of_slot[r]];
    if ((uint64_t)u < oracle_spin_threshold(beta, dE_int, p->s)) sp[y * L + x] = (int8_t)-s;
}

/* One sweep: every site gets one trial. Sites are visited colour by colour on the
 * checkerboard (colour 0 = (x + y) even, then colour 1); sites of one colour have no common
 * bond, so their trials are independent and their order does not matter. */
static void sweep_once(oracle_pt* p) {
    const int L = p->L, R = p->R;
    for (int colour = 0; colour < 2; ++colour) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads_wanted) schedule(static) collapse(2)
#endif
        for (int r = 0; r < R; ++r)
            for (int y = 0; y < L; ++y)
                for (int x = (y + colour) & 1; x < L; x += 2) metropolis_site(p, r, x, y);
    }
    p->t += 1;
}

/* One single-spin-flip Metropolis iteration of the replica in slot r (Sec. 2.1: the trial
 * state x_trial = g(x) flips one spin, chosen uniformly at random; it is accepted with
 * probability min(1, e^{-beta Delta E}), Eq. 1): iteration i draws one Philox block, word 0
 * selects site floor(u0 * L^2 / 2^32) (row-major, i = y L + x) and word 1 is the acceptance
 * draw, compared with the same threshold as a sweep's trial. */
static void metropolis_flip(oracle_pt* p, int r, uint64_t i) {
    const int L = p->L;
    const uint32_t c3 = TAG_FLIP | ((uint32_t)(i >> 32) << 8);
    const uint32_t u0 = philox_word(p->seed, (uint32_t)i, (uint32_t)r, 0u, c3, 0);
    const uint32_t u1 = philox_word(p->seed, (uint32_t)i, (uint32_t)r, 0u, c3, 1);
    const uint64_t site = ((uint64_t)u0 * (uint64_t)L * (uint64_t)L) >> 32;
    const int x = (int)(site % (uint64_t)L), y = (int)(site / (uint64_t)L);
    int8_t* sp = lattice(p, r);
    int s = sp[y * L + x];
    int nb = sp[y * L + (x + 1) % L] + sp[y * L + (x + L - 1) % L] +
             sp[((y + 1) % L) * L + x] + sp[((y + L - 1) % L) * L + x];
    int64_t dE_int = 2 * (int64_t)s * (p->J_int * nb - p->h_int);
    double beta = p->beta[p->temp_of_slot[r]];
    if (dE_int <= 0 || (uint64_t)u1 < oracle_spin_threshold(beta, dE_int, p->s))
        sp[y * L + x] = (int8_t)-s;
}

/* Exchange the configurations at temperatures k and k+1 by swapping their slots. */
static void swap_temperatures(oracle_pt* p, int k) {
    int a = p->slot_of_temp[k], b = p->slot_of_temp[k + 1];
    p->slot_of_temp[k] = b;
    p->slot_of_temp[k + 1] = a;
    p->temp_of_slot[a] = k + 1;
    p->temp_of_slot[b] = k;
}

/* Swap iteration (Sec. 3): neighbours only, each replica at most once; the first swap
 * iteration pairs temperatures (0,1),(2,3),..., the next (1,2),(3,4),..., alternating. */
static void exchange_once(oracle_pt* p) {
    const int R = p->R;
    int parity = (int)(p->e & 1);
    for (int k = parity; k + 1 < R; k += 2) {
        int64_t n = oracle_energy_int(p, k) - oracle_energy_int(p, k + 1);
        uint64_t S = p->swap_rule == ORACLE_SWAP_METROPOLIS
                         ? oracle_swap_threshold_metropolis(p->beta[k], p->beta[k + 1], n, p->s)
                         : oracle_swap_threshold(p->beta[k], p->beta[k + 1], n, p->s);
        uint32_t u = philox_word(p->seed, (uint32_t)k, (uint32_t)p->e, 0u,
                                 TAG_EXCH | ((uint32_t)(p->e >> 32) << 8), 0);
        p->attempted[k] += 1;
        if ((uint64_t)u < S) {
            p->accepted[k] += 1;
            swap_temperatures(p, k);
        }
    }
    p->e += 1;
}

/* Execution phase (Sec. 3, interval scheduling): n sweeps; with m > 0 a swap iteration follows
 * every sweep after which the total number of sweeps done since creation is a multiple of m.
 * m = 0 runs without swaps. */
int oracle_sweep(oracle_pt* p, int64_t n, int m) {
    if (!p || n < 0 || m < 0) return ORACLE_EINVAL;
    for (int64_t j = 0; j < n; ++j) {
        sweep_once(p);
        if (m > 0 && p->t % (uint64_t)m == 0) exchange_once(p);
    }
    return ORACLE_OK;
}

/* Same as oracle_sweep, recording E_int and M of every temperature after each sweep (after
 * that sweep's swap iteration, if any): E_out and M_out are [n][R]. */
int oracle_trace(oracle_pt* p, int64_t n, int m, int64_t* E_out, int64_t* M_out) {
    if (!p || n < 0 || m < 0) return ORACLE_EINVAL;
    for (int64_t j = 0; j < n; ++j) {
        sweep_once(p);
        if (m > 0 && p->t % (uint64_t)m == 0) exchange_once(p);
        for (int k = 0; k < p->R; ++k) {
            if (E_out) E_out[j * p->R + k] = oracle_energy_int(p, k);
            if (M_out) M_out[j * p->R + k] = oracle_magnetisation(p, k);
        }
    }
    return ORACLE_OK;
}

/* The paper's "iteration" read as one single-spin flip per replica: n iterations of every
 * replica; after every iteration that leaves the iteration count a
 * multiple of m (> 0), one swap iteration, the same as after sweeps and sharing their swap
 * index e). The iteration index i counts iterations since creation, independently of
 * sweeps. */
int oracle_flip(oracle_pt* p, int64_t n, int m) {
    if (!p || n < 0 || m < 0) return ORACLE_EINVAL;
    for (int64_t j = 0; j < n; ++j) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(threads_wanted) schedule(static)
#endif
        for (int r = 0; r < p->R; ++r) metropolis_flip(p, r, p->it);
        p->it += 1;
        if (m > 0 && p->it % (uint64_t)m == 0) exchange_once(p);
    }
    return ORACLE_OK;
}

uint64_t oracle_iterations(const oracle_pt* p) { return p->it; }
void oracle_set_iterations(oracle_pt* p, uint64_t it) { p->it = it; }

int64_t oracle_scale(const oracle_pt* p) { return p->s; }

/* Spins of the configuration currently at temperature k. */
int oracle_get_spins(const oracle_pt* p, int k, int8_t* out) {
    if (!p || k < 0 || k >= p->R || !out) return ORACLE_EINVAL;
    memcpy(out, lattice(p, p->slot_of_temp[k]), (size_t)p->L * p->L);
    return ORACLE_OK;
}

int oracle_set_spins(oracle_pt* p, int k, const int8_t* in) {
    if (!p || k < 0 || k >= p->R || !in) return ORACLE_EINVAL;
    for (size_t i = 0; i < (size_t)p->L * p->L; ++i)
        if (in[i] != 1 && in[i] != -1) return ORACLE_EINVAL;
    memcpy(lattice(p, p->slot_of_temp[k]), in, (size_t)p->L * p->L);
    return ORACLE_OK;
}

/* slot_of_temp: the replica slot (chain) currently at each temperature index. */
void oracle_chain_map(const oracle_pt* p, int32_t* out) {
    memcpy(out, p->slot_of_temp, sizeof(int32_t) * p->R);
}

void oracle_swap_stats(const oracle_pt* p, uint64_t* attempted, uint64_t* accepted) {
    if (p->R < 2) return;
    if (attempted) memcpy(attempted, p->attempted, sizeof(uint64_t) * (p->R - 1));
    if (accepted) memcpy(accepted, p->accepted, sizeof(uint64_t) * (p->R - 1));
}

void oracle_counters(const oracle_pt* p, uint64_t* t, uint64_t* e) { *t = p->t; *e = p->e; }

/* Replace the whole state (test support: lets a test continue the chain from a state taken
 * elsewhere). spins_by_slot is [R][L][L] (+1 / -1), slot_of_temp a permutation of 0..R-1,
 * t and e the sweep and swap-iteration counters, attempted / accepted [R-1] (may be NULL
 * when R == 1). */
int oracle_load_state(oracle_pt* p, const int8_t* spins_by_slot, const int32_t* slot_of_temp,
                      uint64_t t, uint64_t e, const uint64_t* attempted,
                      const uint64_t* accepted) {
    const int R = p->R;
    const size_t n = (size_t)p->L * p->L;
    for (size_t i = 0; i < (size_t)R * n; ++i)
        if (spins_by_slot[i] != 1 && spins_by_slot[i] != -1) return ORACLE_EINVAL;
    for (int k = 0; k < R; ++k) {
        if (slot_of_temp[k] < 0 || slot_of_temp[k] >= R) return ORACLE_EINVAL;
        for (int j = 0; j < k; ++j)
            if (slot_of_temp[j] == slot_of_temp[k]) return ORACLE_EINVAL;
    }
    memcpy(p->spin, spins_by_slot, (size_t)R * n);
    for (int k = 0; k < R; ++k) {
        p->slot_of_temp[k] = slot_of_temp[k];
        p->temp_of_slot[slot_of_temp[k]] = k;
    }
    p->t = t;
    p->e = e;
    if (R > 1) {
        memcpy(p->attempted, attempted, sizeof(uint64_t) * (R - 1));
        memcpy(p->accepted, accepted, sizeof(uint64_t) * (R - 1));
    }
    return ORACLE_OK;
}
