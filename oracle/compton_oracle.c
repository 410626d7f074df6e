/*
 * compton_oracle.c -- plain FP64 CPU oracle of the Compton pair-scatter step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path; the product path never
 * calls it.
 *
 * What it follows (arXiv 2206.02937, "Machine Learning-based models in
 * particle-in-cell codes for advanced physics extensions"):
 *   - Sec. 3.1: particles are binned into collision cells, a list of
 *     lepton-photon pairs is formed per cell, the probability of interaction
 *     of each pair is compared with a random number, and accepted pairs are
 *     collided with a momentum update.
 *   - Sec. 3.2: the probability is obtained by boosting the photon to the
 *     lepton rest frame, evaluating the Klein-Nishina cross section there and
 *     boosting the result back to the simulation frame; momenta are in units
 *     of m_e c.
 * The paper prints no formula for these steps (they live in its cited
 * Compton-module paper), so every formula below is the textbook one, and each
 * reading of a point the paper leaves open is stated where it is used.
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, high-precision evaluation, quadrature, conservation, brute force,
 * chi-square).  Philox4x32-10 is pinned by the generator's published
 * known-answer vectors (Salmon et al., SC'11) and by statistics on the CPU,
 * and on a GPU by agreement with cuRAND's device Philox4_32_10.
 *
 * Everything is FP64, single-threaded, in the order the method states it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror and   */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds,  */
/* each a pair of 32x32->64 multiplies by the two round multipliers, an xor */
/* with the other two counter words and the key, and a word permutation;    */
/* the key is bumped by the two Weyl constants between rounds.              */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Counter layout used by the whole method: (id, step low word, stream, step
 * high word) under key (seed low word, seed high word).  Streams:
 *   1  electron pairing key   (id = particle id, word 0)
 *   2  photon pairing key     (id = particle id, word 0)
 *   3  Bernoulli trial        (id = pair index / 4, word = pair index mod 4:
 *                              one block serves four consecutive pairs)
 *   4  scattering angles      (id = pair index, words 0 and 1) */
static void draw(uint64_t seed, uint64_t step, uint32_t stream, uint32_t id, uint32_t out[4])
{
    uint32_t ctr[4] = {id, (uint32_t)step, stream, (uint32_t)(step >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* Uniform on [0,1) from the top 24 bits of a word (exact in FP32 and FP64). */
static double unif_closed0(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }
/* Uniform on (0,1), the same 24 bits offset by half a step. */
static double unif_open(uint32_t r) { return ((double)(r >> 8) + 0.5) * (1.0 / 16777216.0); }

/* ------------------------------------------------------------------------ */
/* Klein-Nishina total cross section in units of the Thomson cross section, */
/* as a function of the photon energy x in the electron rest frame (m_e c^2).*/
/* Textbook closed form, with L = ln(1+2x):                                  */
/*   s(x) = 3/4 { (1+x)/x^3 [2x(1+x)/(1+2x) - L] + L/(2x) - (1+3x)/(1+2x)^2 } */
/* The closed form cancels for small x, so below x = 1/4 its Taylor series  */
/* is summed instead.  The n-th coefficient follows from expanding the three */
/* terms: with d_m = (-1)^m 2^(m-1) (2-m)/m (the x^m coefficient of the      */
/* bracket), a_n = 3/4 [ d_(n+3) + d_(n+2) + (-2)^n/(n+1)                    */
/*                        - (n+1)(-2)^n - 3n(-2)^(n-1) ].                    */
/* ------------------------------------------------------------------------ */
static double kn_bracket_coef(int m)
{
    if (m < 3) return 0.0;
    double sgn = (m % 2 == 0) ? 1.0 : -1.0;
    return sgn * ldexp(1.0, m - 1) * (double)(2 - m) / (double)m;
}

double or_kn_series_coef(int n)
{
    double t1 = kn_bracket_coef(n + 3) + kn_bracket_coef(n + 2);
    double m2n = (n % 2 == 0) ? ldexp(1.0, n) : -ldexp(1.0, n); /* (-2)^n */
    double t2 = m2n / (double)(n + 1);
    double t3 = (double)(n + 1) * m2n + (n >= 1 ? 3.0 * (double)n * (m2n / -2.0) : 0.0);
    return 3.0 * (t1 + (t2 - t3)) / 4.0;
}

double or_kn_sigma(double x)
{
    if (x < 0.25) {
        double sum = 0.0, xn = 1.0;
        for (int n = 0; n < 120; ++n) {
            double term = or_kn_series_coef(n) * xn;
            sum += term;
            if (n > 4 && fabs(term) < 1e-19 * fabs(sum)) break;
            xn *= x;
        }
        return sum;
    }
    double L = log1p(2.0 * x);
    double a = (1.0 + x) / (x * x * x) * (2.0 * x * (1.0 + x) / (1.0 + 2.0 * x) - L);
    double b = L / (2.0 * x);
    double c = (1.0 + 3.0 * x) / ((1.0 + 2.0 * x) * (1.0 + 2.0 * x));
    return 0.75 * (a + b - c);
}

/* Differential cross section in the rest frame per unit t = 1 - cos(theta'),
 * integrated over azimuth, in units of sigma_T.  With xi = 1/(1+x t) (the
 * Compton ratio eps1'/eps'), the Klein-Nishina formula
 *   dsigma/dOmega = r_e^2/2 xi^2 (xi + 1/xi - sin^2 theta')
 * gives dsigma/dt = 3/8 (xi^3 + xi - xi^2 t (2 - t)). */
double or_kn_dsigma_dt(double x, double t)
{
    double xi = 1.0 / (1.0 + x * t);
    return 0.375 * (xi * xi * xi + xi - xi * xi * t * (2.0 - t));
}

/* Cumulative cross section: integral of or_kn_dsigma_dt from 0 to t, from the
 * antiderivatives of its three terms (w = x t):
 *   int xi^3        = t (2 + w) / (2 (1+w)^2)
 *   int xi          = ln(1+w) / x
 *   int xi^2 t(2-t) = [(2x+2) ln(1+w) - w - (2x+1) w/(1+w)] / x^3
 * The last one cancels like 1/x^3; for x t < 1/2 it is summed as the series
 *   sum_k (k+1) (-x)^k [2 t^(k+2)/(k+2) - t^(k+3)/(k+3)]. */
double or_kn_cdf(double x, double t)
{
    double w = x * t;
    double a = t * (2.0 + w) / (2.0 * (1.0 + w) * (1.0 + w));
    double b = (w == 0.0) ? t : log1p(w) / x;
    double c;
    if (w < 0.5) {
        c = 0.0;
        double mx = 1.0; /* (-x)^k */
        for (int k = 0; k < 400; ++k) {
            double tk2 = pow(t, k + 2);
            double term = (double)(k + 1) * mx * (2.0 * tk2 / (double)(k + 2) - tk2 * t / (double)(k + 3));
            c += term;
            if (k > 3 && fabs(term) <= 1e-19 * fabs(c)) break;
            mx *= -x;
        }
    } else {
        double L = log1p(w);
        c = ((2.0 * x + 2.0) * L - w - (2.0 * x + 1.0) * w / (1.0 + w)) / (x * x * x);
    }
    return 0.375 * (a + b - c);
}

/* Inverse of the cumulative cross section: the t in [0,2] with
 * cdf(t) = u cdf(2).  Bisection to the last representable midpoint; slow and
 * plainly correct (the cumulative is strictly increasing). */
double or_kn_sample_t(double x, double u)
{
    double target = u * or_kn_cdf(x, 2.0);
    double lo = 0.0, hi = 2.0;
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (or_kn_cdf(x, mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Kinematics.  Electron u = p_e/(m_e c), gamma = sqrt(1+u^2); photon k =    */
/* p_gamma/(m_e c), energy eps = |k|.                                        */
/* ------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* Invariants of a pair: x = gamma eps - u.k, the photon energy in the
 * electron rest frame, and v = 1 - beta cos(psi), the flux (Moller) factor
 * that carries the rest-frame rate back to the simulation frame.  Both are
 * formed without cancellation:
 *   1 - beta      = 1 / (gamma (gamma + |u|))
 *   1 - cos(psi)  = |u x k|^2 / (|u|^2 |k|^2 (1 + cos psi))   for cos psi > 0
 *   v             = (1 - beta) + beta (1 - cos psi),   x = gamma eps v.
 * An electron at rest has v = 1.  out = {x, v}. */
void or_invariants(const double u[3], const double k[3], double out[2])
{
    double uu = dot3(u, u), un = sqrt(uu);
    double gamma = sqrt(1.0 + uu);
    double eps = norm3(k);
    double v;
    if (un == 0.0 || eps == 0.0) {
        v = 1.0;
    } else {
        double beta = un / gamma;
        double one_m_beta = 1.0 / (gamma * (gamma + un));
        double cosp = dot3(u, k) / (un * eps);
        double one_m_cos;
        if (cosp > 0.0) {
            double cx = u[1] * k[2] - u[2] * k[1];
            double cy = u[2] * k[0] - u[0] * k[2];
            double cz = u[0] * k[1] - u[1] * k[0];
            double sin2 = (cx * cx + cy * cy + cz * cz) / (uu * eps * eps);
            one_m_cos = sin2 / (1.0 + cosp);
        } else {
            one_m_cos = 1.0 - cosp;
        }
        v = one_m_beta + beta * one_m_cos;
    }
    out[0] = gamma * eps * v;
    out[1] = v;
}

/* Lorentz boost of a photon (eps, k) into the rest frame of an electron of
 * four-velocity (gamma, u):  eps' = gamma eps - u.k,
 *   k' = k + u [ (u.k)/(gamma+1) - eps ]. */
void or_boost_to_rest(const double u[3], double eps, const double k[3], double* eps_r, double kr[3])
{
    double gamma = sqrt(1.0 + dot3(u, u));
    double uk = dot3(u, k);
    double f = uk / (gamma + 1.0) - eps;
    *eps_r = gamma * eps - uk;
    for (int i = 0; i < 3; ++i) kr[i] = k[i] + u[i] * f;
}

/* The inverse boost:  eps = gamma eps' + u.k',
 *   k = k' + u [ (u.k')/(gamma+1) + eps' ]. */
void or_boost_to_lab(const double u[3], double eps_r, const double kr[3], double* eps, double k[3])
{
    double gamma = sqrt(1.0 + dot3(u, u));
    double uk = dot3(u, kr);
    double f = uk / (gamma + 1.0) + eps_r;
    *eps = gamma * eps_r + uk;
    for (int i = 0; i < 3; ++i) k[i] = kr[i] + u[i] * f;
}

/* Orthonormal basis (b1, b2) completing a unit vector n, by the branchless
 * construction of Duff, Burgess, Christensen, Hery, Kensler, Liani and
 * Villemin, "Building an Orthonormal Basis, Revisited" (JCGT 6(1), 2017). */
void or_onb(const double n[3], double b1[3], double b2[3])
{
    double sgn = copysign(1.0, n[2]);
    double a = -1.0 / (sgn + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sgn * n[0] * n[0] * a;
    b1[1] = sgn * b;
    b1[2] = -sgn * n[0];
    b2[0] = b;
    b2[1] = sgn + n[1] * n[1] * a;
    b2[2] = -n[1];
}

/* The uniform of the Bernoulli trial of pair p (Sec. 3.1: the probability
 * is compared against a random number): word p mod 4 of the stream-3 block
 * at counter p / 4. */
double or_bernoulli_u0(uint64_t seed, uint64_t step, uint32_t p)
{
    uint32_t r[4];
    draw(seed, step, 3u, p >> 2, r);
    return unif_closed0(r[p & 3u]);
}

/* The collision of one pair with its own draws (Sec. 3.1, "the kinetic
 * collision is resolved"): t from the inverse cumulative cross section with
 * word 0 of the stream-4 draw, phi = 2 pi u2 from word 1, the scattered
 * photon built in the rest frame (energy x/(1 + x t), polar angle from the
 * incoming rest-frame direction, azimuth about it in the Duff et al. basis),
 * boosted back, and the electron given the momentum the photon lost:
 * u <- u + k - k1. */
static void collide_words(const double u[3], const double k[3], uint32_t w_angle, uint32_t w_phi,
                          double u_out[3], double k_out[3])
{
    double inv[2];
    or_invariants(u, k, inv);
    double x = inv[0];
    double eps = norm3(k);
    double u1 = unif_open(w_angle);
    double u2 = unif_closed0(w_phi);
    double t = or_kn_sample_t(x, u1);
    double phi = 2.0 * OR_PI * u2;
    double eps_r, kr[3];
    or_boost_to_rest(u, eps, k, &eps_r, kr);
    /* the rest-frame energy is the invariant x; its direction is kr/|kr| */
    double krn = norm3(kr);
    double n[3] = {kr[0] / krn, kr[1] / krn, kr[2] / krn};
    double b1[3], b2[3];
    or_onb(n, b1, b2);
    double cth = 1.0 - t;
    double sth = sqrt(t * (2.0 - t));
    double cph = cos(phi), sph = sin(phi);
    double e1r = x / (1.0 + x * t);
    double k1r[3];
    for (int i = 0; i < 3; ++i)
        k1r[i] = e1r * (cth * n[i] + sth * (cph * b1[i] + sph * b2[i]));
    double e1, k1[3];
    or_boost_to_lab(u, e1r, k1r, &e1, k1);
    for (int i = 0; i < 3; ++i) {
        u_out[i] = u[i] + k[i] - k1[i];
        k_out[i] = k1[i];
    }
}

void or_collide(const double u[3], const double k[3], uint64_t seed, uint64_t step, uint32_t ctr_id,
                double u_out[3], double k_out[3])
{
    uint32_t r[4];
    draw(seed, step, 4u, ctr_id, r);
    collide_words(u, k, r[0], r[1], u_out, k_out);
}

/* One pair event (Sec. 3.1, Sec. 3.2).
 *   a = n dt s(x) v,  P = 1 - exp(-a)   (evaluated as -expm1(-a));
 *   scatter iff u0 < P, u0 = or_bernoulli_u0;
 *   if scattered: or_collide.
 * n_dens is the pair density (normalised units), dt the time step.
 * Outputs: u_out, k_out (unchanged when not scattered), P, flag, x. */
void or_scatter_event(const double u[3], const double k[3], double n_dens, double dt,
                      uint64_t seed, uint64_t step, uint32_t ctr_id,
                      double u_out[3], double k_out[3], double* P_out, int* flag_out, double* x_out)
{
    double inv[2];
    or_invariants(u, k, inv);
    double x = inv[0], v = inv[1];
    double eps = norm3(k);
    double P = 0.0;
    if (eps > 0.0) {
        double s = or_kn_sigma(x);
        double a = n_dens * dt * s * v;
        P = -expm1(-a);
    }
    double u0 = or_bernoulli_u0(seed, step, ctr_id);
    int flag = (u0 < P) ? 1 : 0;
    for (int i = 0; i < 3; ++i) { u_out[i] = u[i]; k_out[i] = k[i]; }
    if (flag) or_collide(u, k, seed, step, ctr_id, u_out, k_out);
    *P_out = P;
    *flag_out = flag;
    *x_out = x;
}

/* ------------------------------------------------------------------------ */
/* Binning and random in-cell pairing (Sec. 3.1, first step).               */
/* Each particle gets the key word 0 of draw(seed, step, stream, id); within */
/* a cell particles are ordered by (key, id, input index), i.e. a stable    */
/* sort by (cell, key, id).  Cells are in increasing order.                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t cell;
    uint32_t key;
    uint32_t id;
    int64_t idx;
} sort_rec;

static int rec_cmp(const void* pa, const void* pb)
{
    const sort_rec* a = (const sort_rec*)pa;
    const sort_rec* b = (const sort_rec*)pb;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

uint32_t or_pair_key(uint64_t seed, uint64_t step, uint32_t stream, uint32_t id)
{
    uint32_t r[4];
    draw(seed, step, stream, id, r);
    return r[0];
}

/* perm[j] = input index of the j-th particle in sorted order;
 * off[c] = first sorted position of cell c, off[n_cells] = n.
 * Returns 0, or -1 when a cell index is out of range or memory runs out. */
int or_sort_species(int64_t n, const int32_t* cell, const uint32_t* id, int64_t n_cells,
                    uint64_t seed, uint64_t step, uint32_t stream, int64_t* perm, int64_t* off)
{
    sort_rec* recs = (sort_rec*)malloc((size_t)(n > 0 ? n : 1) * sizeof(sort_rec));
    if (!recs) return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (cell[i] < 0 || (int64_t)cell[i] >= n_cells) { free(recs); return -1; }
        recs[i].cell = cell[i];
        recs[i].key = or_pair_key(seed, step, stream, id[i]);
        recs[i].id = id[i];
        recs[i].idx = i;
    }
    qsort(recs, (size_t)n, sizeof(sort_rec), rec_cmp);
    for (int64_t c = 0; c <= n_cells; ++c) off[c] = 0;
    for (int64_t j = 0; j < n; ++j) {
        perm[j] = recs[j].idx;
        off[recs[j].cell + 1] += 1;
    }
    for (int64_t c = 0; c < n_cells; ++c) off[c + 1] += off[c];
    free(recs);
    return 0;
}

/* One whole step (Sec. 3.1): bin and order both species, pair rank k of the
 * electrons with rank k of the photons in every cell for
 * k < M_c = min(N_e,c, N_g,c), and resolve every pair.  Pairs are numbered
 * in cell order; pair number p is the counter id of its scattering draw.
 *
 * Reading of a point the paper leaves open: with unequal counts the pair
 * density is n = max(N_e,c, N_g,c) * w_over_v, so that M_c pairs with this
 * density give the expected event count N_e N_g w_over_v sigma v dt of the
 * cell, and no particle sits in two pairs.
 *
 * Outputs, all in sorted order: e_out/g_out (3 x n, FP64 momenta after the
 * step, row-major by component), e_perm/g_perm (input index), e_off/g_off
 * (n_cells+1), pair_off (n_cells+1) and per pair P, flag, x.  The pair arrays
 * must hold min(n_e, n_g) entries.  Returns the number of pairs, or -1. */
int64_t or_step(int64_t n_cells, double w_over_v, double dt, uint64_t seed, uint64_t step,
                int64_t n_e, const float* eux, const float* euy, const float* euz,
                const int32_t* ecell, const uint32_t* eid,
                int64_t n_g, const float* gkx, const float* gky, const float* gkz,
                const int32_t* gcell, const uint32_t* gid,
                double* e_out, double* g_out, int64_t* e_perm, int64_t* g_perm,
                int64_t* e_off, int64_t* g_off, int64_t* pair_off,
                double* P, int32_t* flag, double* x)
{
    if (or_sort_species(n_e, ecell, eid, n_cells, seed, step, 1u, e_perm, e_off)) return -1;
    if (or_sort_species(n_g, gcell, gid, n_cells, seed, step, 2u, g_perm, g_off)) return -1;
    for (int64_t j = 0; j < n_e; ++j) {
        int64_t i = e_perm[j];
        e_out[j] = eux[i]; e_out[n_e + j] = euy[i]; e_out[2 * n_e + j] = euz[i];
    }
    for (int64_t j = 0; j < n_g; ++j) {
        int64_t i = g_perm[j];
        g_out[j] = gkx[i]; g_out[n_g + j] = gky[i]; g_out[2 * n_g + j] = gkz[i];
    }
    int64_t np = 0;
    pair_off[0] = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t ne = e_off[c + 1] - e_off[c];
        int64_t ng = g_off[c + 1] - g_off[c];
        int64_t m = ne < ng ? ne : ng;
        double n_dens = (double)(ne > ng ? ne : ng) * w_over_v;
        for (int64_t q = 0; q < m; ++q) {
            int64_t je = e_off[c] + q, jg = g_off[c] + q;
            double u[3] = {e_out[je], e_out[n_e + je], e_out[2 * n_e + je]};
            double k[3] = {g_out[jg], g_out[n_g + jg], g_out[2 * n_g + jg]};
            double uo[3], ko[3];
            int f;
            or_scatter_event(u, k, n_dens, dt, seed, step, (uint32_t)np, uo, ko, &P[np], &f, &x[np]);
            flag[np] = f;
            e_out[je] = uo[0]; e_out[n_e + je] = uo[1]; e_out[2 * n_e + je] = uo[2];
            g_out[jg] = ko[0]; g_out[n_g + jg] = ko[1]; g_out[2 * n_g + jg] = ko[2];
            ++np;
        }
        pair_off[c + 1] = np;
    }
    return np;
}

/* ------------------------------------------------------------------------ */
/* Unequal macro-particle weights (Sec. 3.2 gives P_max = 2 sigma_T c dt     */
/* max[w_e, w_g]: the probability bound of a pair takes the heavier of the   */
/* two weights).  Reading built here:                                       */
/*   - w is a macro-particle's weight over the cell volume (the density it  */
/*     adds); binning and pairing are those of or_step;                     */
/*   - pair density n_p = max(N_e, N_g) max(w_e, w_g), so that the expected  */
/*     number of real events of a cell, sum over pairs of P min(w_e, w_g) V, */
/*     is n_e n_g sigma v dt V in the small-probability limit, as with      */
/*     equal weights;                                                       */
/*   - a colliding pair is resolved as in or_collide; the lighter partner   */
/*     takes its new momentum, the heavier one only if u w_heavy < w_light, */
/*     u = (r2 >> 8) 2^-24 with r2 word 2 of draw(seed, step, 4, p) (weight  */
/*     rejection; equal weights update both).                               */
/* ew or gw NULL: every particle of that species has weight w_over_v.       */
/* Outputs as or_step, plus the sorted weights (e_w_out, g_w_out; FP64) and */
/* upd[p] = (electron updated) | (photon updated) << 1 for every pair.      */
/* ------------------------------------------------------------------------ */
int64_t or_step_weighted(int64_t n_cells, double w_over_v, double dt, uint64_t seed, uint64_t step,
                         int64_t n_e, const float* eux, const float* euy, const float* euz,
                         const int32_t* ecell, const uint32_t* eid, const float* ew,
                         int64_t n_g, const float* gkx, const float* gky, const float* gkz,
                         const int32_t* gcell, const uint32_t* gid, const float* gw,
                         double* e_out, double* g_out, double* e_w_out, double* g_w_out,
                         int64_t* e_perm, int64_t* g_perm, int64_t* e_off, int64_t* g_off, int64_t* pair_off,
                         double* P, int32_t* flag, int32_t* upd)
{
    if (or_sort_species(n_e, ecell, eid, n_cells, seed, step, 1u, e_perm, e_off)) return -1;
    if (or_sort_species(n_g, gcell, gid, n_cells, seed, step, 2u, g_perm, g_off)) return -1;
    for (int64_t j = 0; j < n_e; ++j) {
        int64_t i = e_perm[j];
        e_out[j] = eux[i]; e_out[n_e + j] = euy[i]; e_out[2 * n_e + j] = euz[i];
        e_w_out[j] = ew ? (double)ew[i] : w_over_v;
    }
    for (int64_t j = 0; j < n_g; ++j) {
        int64_t i = g_perm[j];
        g_out[j] = gkx[i]; g_out[n_g + j] = gky[i]; g_out[2 * n_g + j] = gkz[i];
        g_w_out[j] = gw ? (double)gw[i] : w_over_v;
    }
    int64_t np = 0;
    pair_off[0] = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t ne = e_off[c + 1] - e_off[c];
        int64_t ng = g_off[c + 1] - g_off[c];
        int64_t m = ne < ng ? ne : ng;
        double n_max = (double)(ne > ng ? ne : ng);
        for (int64_t q = 0; q < m; ++q) {
            int64_t je = e_off[c] + q, jg = g_off[c] + q;
            double we = e_w_out[je], wg = g_w_out[jg];
            double n_pair = n_max * (we > wg ? we : wg);
            double u[3] = {e_out[je], e_out[n_e + je], e_out[2 * n_e + je]};
            double k[3] = {g_out[jg], g_out[n_g + jg], g_out[2 * n_g + jg]};
            double uo[3], ko[3], xx;
            int f;
            or_scatter_event(u, k, n_pair, dt, seed, step, (uint32_t)np, uo, ko, &P[np], &f, &xx);
            flag[np] = f;
            int up_e = 0, up_g = 0;
            if (f) {
                uint32_t r[4];
                draw(seed, step, 4u, (uint32_t)np, r);
                double uw = unif_closed0(r[2]);
                up_e = (we <= wg) || (uw * we < wg);
                up_g = (wg <= we) || (uw * wg < we);
            }
            upd[np] = up_e | (up_g << 1);
            if (up_e) { e_out[je] = uo[0]; e_out[n_e + je] = uo[1]; e_out[2 * n_e + je] = uo[2]; }
            if (up_g) { g_out[jg] = ko[0]; g_out[n_g + jg] = ko[1]; g_out[2 * n_g + jg] = ko[2]; }
            ++np;
        }
        pair_off[c + 1] = np;
    }
    return np;
}

/* Pre-paired events (the serving form): pair i uses counter id i under the
 * given seed and step, with its own density n[i].  Outputs 3 x n FP64
 * momenta (row-major by component), P and flag per pair. */
void or_pairs(int64_t n, const float* ux, const float* uy, const float* uz,
              const float* kx, const float* ky, const float* kz, const float* n_dens,
              double dt, uint64_t seed, uint64_t step,
              double* u_out, double* k_out, double* P, int32_t* flag)
{
    for (int64_t i = 0; i < n; ++i) {
        double u[3] = {ux[i], uy[i], uz[i]};
        double k[3] = {kx[i], ky[i], kz[i]};
        double uo[3], ko[3], xx;
        int f;
        or_scatter_event(u, k, n_dens[i], dt, seed, step, (uint32_t)i, uo, ko, &P[i], &f, &xx);
        flag[i] = f;
        for (int c = 0; c < 3; ++c) { u_out[c * n + i] = uo[c]; k_out[c * n + i] = ko[c]; }
    }
}

/* The ratio r = s(x) v / 2 per pair: the quantity the surrogate network
 * predicts (the probability normalised by its cell maximum of Sec. 3.2,
 * P_max = 2 sigma_T c dt max w, in the small-probability limit). */
void or_ratio(int64_t n, const float* ux, const float* uy, const float* uz,
              const float* kx, const float* ky, const float* kz, double* r)
{
    for (int64_t i = 0; i < n; ++i) {
        double u[3] = {ux[i], uy[i], uz[i]};
        double k[3] = {kx[i], ky[i], kz[i]};
        double inv[2];
        or_invariants(u, k, inv);
        double eps = norm3(k);
        r[i] = eps > 0.0 ? 0.5 * or_kn_sigma(inv[0]) * inv[1] : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* No-Time-Counter candidate selection (Sec. 3.1, second step; Bird 1989).   */
/* The paper gives no formula (its module paper is not available); the      */
/* reading built here:                                                      */
/*   - the particles are binned and ordered as or_step does;                */
/*   - cell c draws N = floor(E + U) candidate pairs, E = N_e N_g (w/V)      */
/*     sigma_max v_max dt with sigma_max v_max = 2 sigma_T c (sigma <=       */
/*     sigma_T, v <= 2), U = word 0 of draw(seed, step, 5, c);              */
/*   - candidate j takes the block draw(seed, step, 6 | j << 8, c): word 0   */
/*     picks the electron (e_off + floor(w0 N_e / 2^32)), word 1 the photon, */
/*     and the pair collides iff the uniform of word 2 is below              */
/*     r = sigma_KN(x) v / (2 sigma_T), the acceptance ratio of the method;  */
/*   - an accepted candidate collides at once (angle from word 3, azimuth   */
/*     from word 0 of draw(seed, step, 7 | j << 8, c)) and later candidates */
/*     of the cell see the updated momenta.                                 */
/* Outputs e_out, g_out as or_step; per cell the candidate and collision    */
/* counts and near[c] = 1 if some candidate's uniform lay within 1e-6 of its */
/* ratio (a decision FP32 arithmetic may take the other way).               */
/* ------------------------------------------------------------------------ */
static int64_t pick(uint32_t w, int64_t n) { return (int64_t)(((uint64_t)w * (uint64_t)n) >> 32); }

int64_t or_ntc_step(int64_t n_cells, double w_over_v, double dt, uint64_t seed, uint64_t step,
                    int64_t n_e, const float* eux, const float* euy, const float* euz,
                    const int32_t* ecell, const uint32_t* eid,
                    int64_t n_g, const float* gkx, const float* gky, const float* gkz,
                    const int32_t* gcell, const uint32_t* gid,
                    double* e_out, double* g_out, int64_t* e_perm, int64_t* g_perm,
                    int64_t* e_off, int64_t* g_off, int64_t* n_cand, int64_t* n_coll, int32_t* near)
{
    if (or_sort_species(n_e, ecell, eid, n_cells, seed, step, 1u, e_perm, e_off)) return -1;
    if (or_sort_species(n_g, gcell, gid, n_cells, seed, step, 2u, g_perm, g_off)) return -1;
    for (int64_t j = 0; j < n_e; ++j) {
        int64_t i = e_perm[j];
        e_out[j] = eux[i]; e_out[n_e + j] = euy[i]; e_out[2 * n_e + j] = euz[i];
    }
    for (int64_t j = 0; j < n_g; ++j) {
        int64_t i = g_perm[j];
        g_out[j] = gkx[i]; g_out[n_g + j] = gky[i]; g_out[2 * n_g + j] = gkz[i];
    }
    int64_t total = 0;
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t ne = e_off[c + 1] - e_off[c];
        int64_t ng = g_off[c + 1] - g_off[c];
        n_cand[c] = 0;
        n_coll[c] = 0;
        near[c] = 0;
        if (ne == 0 || ng == 0) continue;
        uint32_t r[4];
        draw(seed, step, 5u, (uint32_t)c, r);
        double expect = (double)ne * (double)ng * w_over_v * 2.0 * dt;
        int64_t nc = (int64_t)floor(expect + unif_closed0(r[0]));
        n_cand[c] = nc;
        for (int64_t j = 0; j < nc; ++j) {
            uint32_t q[4];
            draw(seed, step, 6u | ((uint32_t)j << 8), (uint32_t)c, q);
            int64_t je = e_off[c] + pick(q[0], ne);
            int64_t jg = g_off[c] + pick(q[1], ng);
            double u[3] = {e_out[je], e_out[n_e + je], e_out[2 * n_e + je]};
            double k[3] = {g_out[jg], g_out[n_g + jg], g_out[2 * n_g + jg]};
            double ratio = 0.0;
            if (norm3(k) > 0.0) {
                double inv[2];
                or_invariants(u, k, inv);
                ratio = 0.5 * or_kn_sigma(inv[0]) * inv[1];
            }
            double ua = unif_closed0(q[2]);
            if (fabs(ua - ratio) < 1e-6) near[c] = 1;
            if (ua < ratio) {
                uint32_t z[4];
                draw(seed, step, 7u | ((uint32_t)j << 8), (uint32_t)c, z);
                double uo[3], ko[3];
                collide_words(u, k, q[3], z[0], uo, ko);
                e_out[je] = uo[0]; e_out[n_e + je] = uo[1]; e_out[2 * n_e + je] = uo[2];
                g_out[jg] = ko[0]; g_out[n_g + jg] = ko[1]; g_out[2 * n_g + jg] = ko[2];
                ++n_coll[c];
            }
        }
        total += nc;
    }
    return total;
}
