/*
 * Plain FP64 CPU oracle for the wildfire cellular automaton of arXiv 2502.18738
 * (PyTorchFire). TEST INFRASTRUCTURE ONLY: it exists to check the CUDA library,
 * and only the tests, the package's smoke entry and the benchmark's CPU-baseline
 * leg may load it. It shares no code, header or constant with the CUDA path.
 *
 * Every function is a direct, unblocked transcription of the equations it cites:
 *   orc_philox4x32_10   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel
 *                        random numbers: as easy as 1, 2, 3"), the counter RNG that
 *                        supplies the two uniform matrices of the step (Sec. 2.2, data flow).
 *   orc_prep            Eq. 1 (slope), Eq. 3 (wind), Eq. 4 (slope factor), Eq. 2
 *                        (propagation probability) and Eq. 5/8 (f_p = tanh(c x)).
 *   orc_step_discrete   Sec. 2.2 transition rules with Eq. 9 (ignition probability).
 *   orc_step_diff       the differentiable (mean-field) step: Eq. 9 with the burning
 *                        indicator replaced by the burning probability b.
 *   orc_adjoint_step    the exact transpose (reverse-mode chain rule) of orc_step_diff.
 *   orc_prep_adjoint    the chain rule of orc_prep to (p_h, c1, c2, a, p_veg, p_den).
 *
 * Conventions (readings of the paper where it is silent or ambiguous):
 *   grid H x W row-major, row r grows southward, column c grows eastward;
 *   direction d = 0..7 is the offset (dr, dc) from the receiving cell j to its burning
 *   neighbour i = j + (dr, dc), in the order (-1,-1) (-1,0) (-1,1) (0,-1) (0,1) (1,-1) (1,0) (1,1);
 *   slope theta_s = atan((E_j - E_i) / (k l)) in degrees (uphill spread is positive);
 *   wind: theta = theta_w,j - phi_d, phi_d = atan2(dr, -dc) in degrees is the direction
 *   of travel from i to j, measured from East counter-clockwise;
 *   the receiving cell's fields are used; neighbours outside the grid never burn.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_C_FP 1.1486328125 /* Eq. 8: the paper's value of c */

static const int ORC_DR[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
static const int ORC_DC[8] = {-1, 0, 1, -1, 1, -1, 0, 1};

/* ---------------------------------------------------------------- Philox */

static void orc_mulhilo(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: each round multiplies words 0 and 2 by the two Philox
 * multipliers, swaps and xors the halves with the key; the key is advanced by the two
 * Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        orc_mulhilo(0xD2511F53u, c0, &hi0, &lo0);
        orc_mulhilo(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in [0,1) from the top 24 bits of a 32-bit draw (exact in FP32 and FP64). */
static double orc_uniform(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* The two uniform draws of one cell at one step: counter (cell, run, step, fire),
 * key (seed low word, seed high word); lane 0 = ignition draw, lane 1 = continue draw. */
void orc_cell_draws(uint64_t seed, uint32_t run, uint32_t step, uint32_t fire, uint32_t cell,
                    double* u0, double* u1) {
    uint32_t ctr[4] = {cell, run, step, fire};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    *u0 = orc_uniform(x[0]);
    *u1 = orc_uniform(x[1]);
}

/* ------------------------------------------------------------------ prep */

static double orc_deg(double rad) { return rad * (180.0 / M_PI); }
static double orc_rad(double deg) { return deg * (M_PI / 180.0); }

/* Per-direction factors of one (j, d) pair, following Eq. 1-4. Returns 0 when the
 * neighbour i is outside the grid. */
/* slope: the H x W x 3 x 3 input of Sec. 2.1 (degrees, [r][c][dr+1][dc+1], Eq. 1 with E
 * the cell and E-hat its neighbour) when given, else Eq. 1 from the altitude map E */
static int orc_factors(int H, int W, int r, int c, int d, const float* E, const float* slope, const float* V,
                       const float* th, double c1, double c2, double a, double l,
                       double* pw, double* ps, double* theta_s, double* cos_m1, double* Vj) {
    int ri = r + ORC_DR[d], ci = c + ORC_DC[d];
    if (ri < 0 || ri >= H || ci < 0 || ci >= W) return 0;
    size_t j = (size_t)r * W + c, i = (size_t)ri * W + ci;
    double ts;
    if (slope) {
        ts = (double)slope[j * 9 + (size_t)(ORC_DR[d] + 1) * 3 + (size_t)(ORC_DC[d] + 1)];
    } else {
        double k = (ORC_DR[d] != 0 && ORC_DC[d] != 0) ? sqrt(2.0) : 1.0;   /* Eq. 1 */
        double dE = E ? ((double)E[j] - (double)E[i]) : 0.0;
        ts = orc_deg(atan(dE / (k * l)));                                   /* Eq. 1, degrees */
    }
    double v = V ? (double)V[j] : 0.0;
    double phi = orc_deg(atan2((double)ORC_DR[d], (double)(-ORC_DC[d])));
    double theta = (th ? (double)th[j] : 0.0) - phi;
    double cm1 = cos(orc_rad(theta)) - 1.0;
    *pw = exp(c1 * v) * exp(c2 * v * cm1);                                /* Eq. 3 */
    *ps = exp(a * ts);                                                    /* Eq. 4 */
    *theta_s = ts;
    *cos_m1 = cm1;
    *Vj = v;
    return 1;
}

/* q[d][j] = f_p(p_propagate) for the burning neighbour in direction d of cell j. */
void orc_prep(int H, int W, const float* E, const float* slope, const float* p_veg, const float* p_den,
              const float* V, const float* th, const uint8_t* burnable, double p_h, double c1,
              double c2, double a, double l, double* q) {
    size_t HW = (size_t)H * W;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            size_t j = (size_t)r * W + c;
            double pv = p_veg ? (double)p_veg[j] : 0.0;
            double pd = p_den ? (double)p_den[j] : 0.0;
            for (int d = 0; d < 8; ++d) {
                double pw, ps, ts, cm1, v;
                double qq = 0.0;
                if (orc_factors(H, W, r, c, d, E, slope, V, th, c1, c2, a, l, &pw, &ps, &ts, &cm1, &v)) {
                    double pp = p_h * (1.0 + pv) * (1.0 + pd) * pw * ps;          /* Eq. 2 */
                    qq = tanh(ORC_C_FP * pp);                                      /* Eq. 5 */
                }
                if (burnable && burnable[j] == 0) qq = 0.0;
                q[(size_t)d * HW + j] = qq;
            }
        }
    }
}

/* ---------------------------------------------------------- discrete step */

/* Eq. 9, p_ignite = 1 - prod_i (1 - p_i), is evaluated as -expm1(sum_i log1p(-p_i)):
 * the same quantity, without the cancellation of 1 - prod in floating point, which
 * would round every contribution below ~1e-16 to zero (those tiny probabilities at the
 * leading edge of the fire are what later grows into the front). */
static double orc_one_minus_exp(double logprod) { return -expm1(logprod); }

/* One synchronous step of R realisations (Sec. 2.2 rules, Eq. 9). States:
 * 0 non-burnable, 1 unburned, 2 burning, 3 burned. Realisation r uses Philox run
 * index run0 + r. P_out (nullable, R*H*W) receives the FP64 ignition probability of
 * every unburned cell (0 elsewhere); u_out (nullable) receives the draw that decided
 * the cell (u0 for unburned, u1 for burning, -1 otherwise). The ignition comparison is
 * taken in FP32: the FP64 probability is rounded to float first, as the kernel's is. */
void orc_step_discrete(int H, int W, int R, const uint8_t* S, uint8_t* S_next, const double* q,
                       float p_continue, uint64_t seed, uint32_t run0, uint32_t step, uint32_t fire,
                       double* P_out, double* u_out) {
    size_t HW = (size_t)H * W;
    for (int rr = 0; rr < R; ++rr) {
        const uint8_t* s = S + (size_t)rr * HW;
        uint8_t* sn = S_next + (size_t)rr * HW;
#pragma omp parallel for schedule(static)
        for (int r = 0; r < H; ++r) {
            for (int c = 0; c < W; ++c) {
                size_t j = (size_t)r * W + c;
                uint8_t st = s[j], out = st;
                double P = 0.0, u = -1.0;
                if (st == 1) {
                    double logprod = 0.0;   /* log of prod (1 - q) over burning neighbours */
                    for (int d = 0; d < 8; ++d) {
                        int ri = r + ORC_DR[d], ci = c + ORC_DC[d];
                        if (ri < 0 || ri >= H || ci < 0 || ci >= W) continue;
                        if (s[(size_t)ri * W + ci] == 2) logprod += log1p(-q[(size_t)d * HW + j]);
                    }
                    P = orc_one_minus_exp(logprod);                              /* Eq. 9 */
                    double u0, u1;
                    orc_cell_draws(seed, run0 + (uint32_t)rr, step, fire, (uint32_t)j, &u0, &u1);
                    u = u0;
                    if ((float)u0 < (float)P) out = 2;
                } else if (st == 2) {
                    double u0, u1;
                    orc_cell_draws(seed, run0 + (uint32_t)rr, step, fire, (uint32_t)j, &u0, &u1);
                    u = u1;
                    out = ((float)u1 < p_continue) ? 2 : 3;
                }
                sn[j] = out;
                if (P_out) P_out[(size_t)rr * HW + j] = P;
                if (u_out) u_out[(size_t)rr * HW + j] = u;
            }
        }
    }
}

/* T steps starting at global step index step0; S0 and S_out are R*H*W. */
void orc_forward_discrete(int H, int W, int R, const uint8_t* S0, uint8_t* S_out, const double* q,
                          float p_continue, uint64_t seed, uint32_t run0, uint32_t step0,
                          uint32_t fire, int T) {
    size_t n = (size_t)R * H * W;
    uint8_t* cur = (uint8_t*)malloc(n);
    uint8_t* nxt = (uint8_t*)malloc(n);
    memcpy(cur, S0, n);
    for (int t = 0; t < T; ++t) {
        orc_step_discrete(H, W, R, cur, nxt, q, p_continue, seed, run0, step0 + (uint32_t)t, fire,
                          NULL, NULL);
        uint8_t* tmp = cur; cur = nxt; nxt = tmp;
    }
    memcpy(S_out, cur, n);
    free(cur);
    free(nxt);
}

/* ------------------------------------------------------ differentiable step */

/* Mean-field step: state (a, b) = (P[ever ignited], P[burning]).
 *   P_j = 1 - prod_d (1 - b_i q_dj)          (Eq. 9 with the indicator replaced by b_i)
 *   n_j = (1 - a_j) P_j,  a'_j = a_j + n_j,  b'_j = n_j + p_continue b_j
 * P_out (nullable) receives P. */
void orc_step_diff(int H, int W, const double* a, const double* b, const double* q, double p_continue,
                   double* a_next, double* b_next, double* P_out) {
    size_t HW = (size_t)H * W;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            size_t j = (size_t)r * W + c;
            double logprod = 0.0;
            for (int d = 0; d < 8; ++d) {
                int ri = r + ORC_DR[d], ci = c + ORC_DC[d];
                if (ri < 0 || ri >= H || ci < 0 || ci >= W) continue;
                logprod += log1p(-b[(size_t)ri * W + ci] * q[(size_t)d * HW + j]);
            }
            double P = orc_one_minus_exp(logprod);                               /* Eq. 9 */
            double n = (1.0 - a[j]) * P;
            a_next[j] = a[j] + n;
            b_next[j] = n + p_continue * b[j];
            if (P_out) P_out[j] = P;
        }
    }
}

/* Reverse-mode transpose of orc_step_diff. Inputs: state (a, b) at t, adjoints
 * (la1, lb1) of (a', b') at t+1. Outputs (overwritten): adjoints (la0, lb0) of (a, b).
 * Gq (8*H*W) is ACCUMULATED with dL/dq_dj of this step. Written as a plain scatter
 * over the receiving cells j, one leave-one-out product per (j, d). */
void orc_adjoint_step(int H, int W, const double* a, const double* b, const double* q, double p_continue,
                      const double* la1, const double* lb1, double* la0, double* lb0, double* Gq) {
    size_t HW = (size_t)H * W;
    for (size_t j = 0; j < HW; ++j) { la0[j] = 0.0; lb0[j] = 0.0; }
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            size_t j = (size_t)r * W + c;
            int inside[8];
            size_t src[8];
            double logprod = 0.0;
            for (int d = 0; d < 8; ++d) {
                int ri = r + ORC_DR[d], ci = c + ORC_DC[d];
                inside[d] = !(ri < 0 || ri >= H || ci < 0 || ci >= W);
                src[d] = inside[d] ? (size_t)ri * W + ci : 0;
                if (inside[d]) logprod += log1p(-b[src[d]] * q[(size_t)d * HW + j]);
            }
            double P = orc_one_minus_exp(logprod);
            double ln = la1[j] + lb1[j];                 /* n feeds both a' and b' */
            la0[j] += la1[j] - ln * P;                   /* a' = a + (1-a) P */
            lb0[j] += p_continue * lb1[j];               /* b' = n + p_c b */
            double lP = ln * (1.0 - a[j]);
            for (int d = 0; d < 8; ++d) {
                if (!inside[d]) continue;
                double loo = 1.0;                        /* prod over d' != d */
                for (int e = 0; e < 8; ++e) {
                    if (e == d || !inside[e]) continue;
                    loo *= 1.0 - b[src[e]] * q[(size_t)e * HW + j];
                }
                lb0[src[d]] += lP * q[(size_t)d * HW + j] * loo;   /* dP/db_i */
                Gq[(size_t)d * HW + j] += lP * b[src[d]] * loo;    /* dP/dq_dj */
            }
        }
    }
}

/* Chain rule of orc_prep. Gq = dL/dq (8*H*W). grad4 (accumulated) = dL/d(p_h, c1, c2, a);
 * g_pveg, g_pden (nullable, H*W, accumulated) = per-cell gradients. */
void orc_prep_adjoint(int H, int W, const float* E, const float* slope, const float* p_veg, const float* p_den,
                      const float* V, const float* th, const uint8_t* burnable, double p_h, double c1,
                      double c2, double a, double l, const double* Gq, double grad4[4], double* g_pveg,
                      double* g_pden) {
    size_t HW = (size_t)H * W;
    double gh = 0.0, g1 = 0.0, g2 = 0.0, ga = 0.0;
    for (int r = 0; r < H; ++r) {
        for (int c = 0; c < W; ++c) {
            size_t j = (size_t)r * W + c;
            if (burnable && burnable[j] == 0) continue;
            double pv = p_veg ? (double)p_veg[j] : 0.0;
            double pd = p_den ? (double)p_den[j] : 0.0;
            for (int d = 0; d < 8; ++d) {
                double pw, ps, ts, cm1, v;
                if (!orc_factors(H, W, r, c, d, E, slope, V, th, c1, c2, a, l, &pw, &ps, &ts, &cm1, &v)) continue;
                double pp = p_h * (1.0 + pv) * (1.0 + pd) * pw * ps;
                double qq = tanh(ORC_C_FP * pp);
                double gpp = Gq[(size_t)d * HW + j] * ORC_C_FP * (1.0 - qq * qq);  /* tanh' */
                gh += gpp * (1.0 + pv) * (1.0 + pd) * pw * ps;
                g1 += gpp * pp * v;
                g2 += gpp * pp * v * cm1;
                ga += gpp * pp * ts;
                if (g_pveg) g_pveg[j] += gpp * p_h * (1.0 + pd) * pw * ps;
                if (g_pden) g_pden[j] += gpp * p_h * (1.0 + pv) * pw * ps;
            }
        }
    }
    grad4[0] += gh; grad4[1] += g1; grad4[2] += g2; grad4[3] += ga;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
