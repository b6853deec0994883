/*
 * FP64 CPU oracle for the GB / constant-(pH,E) / E-REMD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA path: no headers, no tables, no helpers.
 *
 * Every function is the plain definition written out in double precision:
 * O(N^2) double loops, no tiling, no fixed point, no series, no reordering.
 *
 * Sources of the mathematics
 *   - Generalized Born model of Onufriev, Bashford and Case ("igb=2" in AMBER),
 *     used for MD and for every state-change energy (Sec. III.D).  The paper
 *     only names the model; its pieces are the Hawkins-Cramer-Truhlar pairwise
 *     descreening integral and the OBC rescaling of the integral into an
 *     effective Born radius, both restated below from their definitions.
 *   - Redox Monte Carlo criterion, Eq. 8 (Sec. II.A); protonation criterion,
 *     Eq. 9 (Sec. II.B); proposal and residue choice (Sec. III.A, III.A.1);
 *     one attempt per residue in random order (Sec. III.A.2).
 *   - E-REMD exchange, Eq. 14-15 (Sec. II.C) and the neighbour schedule of
 *     Sec. III.B; pH exchange by analogy with Eq. 12 for protons.
 *   - Philox4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     SC'11), from its published definition.
 *   - Optional cutoffs (the paper's GB runs use none; its explicit-solvent
 *     runs use an 8 A direct-space cutoff, Sec. III.D): a Born-radius cutoff
 *     that restricts the HCT integral to a ball of radius rgbmax about the
 *     descreened atom, and truncation of the GB and Coulomb pair sums at
 *     distance `cut`.  Both default to 0 = off.
 *   - BAOAB Langevin splitting (Leimkuhler and Matthews, 2013) for the MD
 *     driver; the paper only says "Langevin dynamics" (Sec. III.D).
 *
 * Parity status: every function below is pinned by tests that do not re-use
 * it (quadrature, closed forms, finite differences, numpy's Philox).
 *
 * Units: kcal/mol, Angstrom, e, ps, amu, V, K.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GBO_KE 332.0522173          /* Coulomb constant, kcal*A/(mol*e^2) */
#define GBO_FARADAY 23.0605478      /* kcal/(mol*V) */
#define GBO_LN10 2.302585092994045684
#define GBO_ACCEL 418.4             /* (kcal/mol/A)/amu -> A/ps^2 */
#define GBO_PI 3.14159265358979323846

typedef struct {
    double alpha, beta, gamma;      /* OBC rescaling */
    double offset;                  /* dielectric offset subtracted from rho */
    double eps_in, eps_out;
    double bond_k, bond_r0;         /* E = k (r - r0)^2 over (i, i+1) */
    double rep_k, rep_sigma;        /* E = k (sigma - r)^2, r < sigma, |i-j|>1 */
    double dt, friction, mass, kT;  /* Langevin driver */
    double kappa;                   /* inverse Debye length of the salt (1/A); 0 = no salt */
    double rgbmax;                  /* Born-radius cutoff (A); 0 = none */
    double cut;                     /* pair cutoff of E_GB and E_Coul (A); 0 = none */
} gbo_params;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10                                                             */
/* ------------------------------------------------------------------------ */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

/* One 4x64 block: counter c, key k -> out.  Round multipliers and Weyl key
 * increments are the published Philox4x64 constants. */
void gbo_philox4x64(const uint64_t c_in[4], const uint64_t k_in[2], uint64_t out[4]) {
    uint64_t c0 = c_in[0], c1 = c_in[1], c2 = c_in[2], c3 = c_in[3];
    uint64_t k0 = k_in[0], k1 = k_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint64_t a, uint64_t b, uint64_t tag, uint64_t blk, uint64_t w[4]) {
    uint64_t c[4] = {a, b, tag, blk};
    uint64_t k[2] = {seed, 0};
    gbo_philox4x64(c, k, w);
}

/* uniform on [0,1) from the top 53 bits */
static double unif53(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }
/* integer in [0, n) from the top 32 bits */
static int32_t pick(uint64_t w, int32_t n) { return (int32_t)(((w >> 32) * (uint64_t)n) >> 32); }

/* ------------------------------------------------------------------------ */
/* Generalized Born: HCT descreening integral and OBC radii                  */
/* ------------------------------------------------------------------------ */

/* H(r; a, s) = (1/4pi) * integral of |y - x_i|^-4 over the part of the ball of
 * radius s centred at x_j (distance r from x_i) that lies outside the ball of
 * radius a centred at x_i.  Closed form from integrating over spherical shells
 * around x_i between L = max(a, |r - s|) and U = r + s; when x_i is engulfed
 * (a < s - r) the complete shells between a and s - r add 1/a - 1/L. */
double gbo_hct_pair(double r, double a, double s) {
    if (a >= r + s) return 0.0;
    double U = r + s;
    double L = fmax(a, fabs(r - s));
    double b = 1.0 / L - 1.0 / U
             + 0.25 * r * (1.0 / (U * U) - 1.0 / (L * L))
             + (0.5 / r) * log(L / U)
             + (0.25 * s * s / r) * (1.0 / (L * L) - 1.0 / (U * U));
    if (a < s - r) b += 2.0 * (1.0 / a - 1.0 / L);
    return 0.5 * b;
}

/* dH/dr of the expression above (L depends on r only when L = |r - s|). */
double gbo_hct_pair_dr(double r, double a, double s) {
    if (a >= r + s) return 0.0;
    double U = r + s;
    double L, dL;
    if (a > fabs(r - s)) { L = a; dL = 0.0; }
    else { L = fabs(r - s); dL = (r > s) ? 1.0 : -1.0; }
    double L2 = L * L, U2 = U * U;
    double db = -dL / L2 + 1.0 / U2
              + 0.25 * (1.0 / U2 - 1.0 / L2)
              + 0.25 * r * (-2.0 / (U2 * U) + 2.0 * dL / (L2 * L))
              - (0.5 / (r * r)) * log(L / U)
              + (0.5 / r) * (dL / L - 1.0 / U)
              - (0.25 * s * s / (r * r)) * (1.0 / L2 - 1.0 / U2)
              + (0.25 * s * s / r) * (-2.0 * dL / (L2 * L) + 2.0 / (U2 * U));
    if (a < s - r) db += 2.0 * dL / L2;
    return 0.5 * db;
}

/* The same integral restricted to the ball |y - x_i| < rc (a Born-radius
 * cutoff: only the part of sphere j within rc of atom i descreens it); rc <= 0
 * means no cutoff.  Written from the shell integral
 *   H = int_L^U' f(t) / t^2 dt + int_a^{min(L, rc)} dt / t^2   (engulfed only),
 * f(t) = (s^2 - (r - t)^2) / (4 r t) the fraction of the shell of radius t
 * about x_i inside sphere j, U' = min(r + s, rc), whose antiderivative is
 *   F(t) = -(s^2 - r^2) / (8 r t^2) - 1 / (2 t) - ln(t) / (4 r). */
static double hct_F(double t, double r, double s) {
    return -(s * s - r * r) / (8.0 * r * t * t) - 0.5 / t - log(t) / (4.0 * r);
}
double gbo_hct_pair_cut(double r, double a, double s, double rc) {
    if (!(rc > 0.0)) return gbo_hct_pair(r, a, s);
    if (a >= r + s) return 0.0;
    double L = fmax(a, fabs(r - s));
    double Up = fmin(r + s, rc);
    double H = (Up > L) ? hct_F(Up, r, s) - hct_F(L, r, s) : 0.0;
    if (a < s - r && a < rc) H += 1.0 / a - 1.0 / fmin(L, rc);
    return H;
}

/* dH/dr of gbo_hct_pair_cut: with dF/dt = f(t)/t^2 and
 * dF/dr = (r^2 + s^2) / (8 r^2 t^2) + ln(t) / (4 r^2) at fixed t. */
double gbo_hct_pair_dr_cut(double r, double a, double s, double rc) {
    if (!(rc > 0.0)) return gbo_hct_pair_dr(r, a, s);
    if (a >= r + s) return 0.0;
    double L, dL;
    if (a > fabs(r - s)) { L = a; dL = 0.0; }
    else { L = fabs(r - s); dL = (r > s) ? 1.0 : -1.0; }
    double U = r + s, Up = fmin(U, rc), dUp = (U < rc) ? 1.0 : 0.0;
    double d = 0.0;
    if (Up > L) {
        double fU = (s * s - (r - Up) * (r - Up)) / (4.0 * r * Up * Up * Up);
        double fL = (s * s - (r - L) * (r - L)) / (4.0 * r * L * L * L);
        double gU = (r * r + s * s) / (8.0 * r * r * Up * Up) + log(Up) / (4.0 * r * r);
        double gL = (r * r + s * s) / (8.0 * r * r * L * L) + log(L) / (4.0 * r * r);
        d = (fU * dUp + gU) - (fL * dL + gL);
    }
    if (a < s - r && a < rc && L < rc) d += dL / (L * L);
    return d;
}

/* Pair cutoff of the GB and Coulomb sums: a pair farther apart than `cut`
 * (exact distance, double precision) contributes nothing; cut <= 0 means no
 * cutoff. */
static int beyond_cut(double r, const gbo_params* p) {
    return p->cut > 0.0 && r > p->cut;
}

static double dist(const double* x, int64_t i, int64_t j, double d[3]) {
    d[0] = x[3 * j] - x[3 * i];
    d[1] = x[3 * j + 1] - x[3 * i + 1];
    d[2] = x[3 * j + 2] - x[3 * i + 2];
    return sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/* Effective Born radii of one molecule of n atoms.
 *   a_i   = rho_i - offset
 *   s_j   = screen_j * a_j
 *   I_i   = sum_{j != i} H(r_ij; a_i, s_j)   (H restricted to the ball of
 *           radius rgbmax about x_i when rgbmax > 0, gbo_hct_pair_cut)
 *   psi_i = a_i I_i
 *   R_i   = 1 / (1/a_i - tanh(alpha psi - beta psi^2 + gamma psi^3) / rho_i)
 *   dR_i/dpsi_i = R_i^2 (1 - tanh^2) (alpha - 2 beta psi + 3 gamma psi^2) / rho_i
 * Any output pointer may be NULL. */
static double born_integral(int64_t n, const double* x, const double* rho, const double* screen,
                            const gbo_params* p, int64_t i) {
    double a_i = rho[i] - p->offset;
    double I = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double d[3];
        double r = dist(x, i, j, d);
        double s_j = screen[j] * (rho[j] - p->offset);
        I += gbo_hct_pair_cut(r, a_i, s_j, p->rgbmax);
    }
    return I;
}

void gbo_born_radii(int64_t n, const double* x, const double* rho, const double* screen,
                    const gbo_params* p, double* I_out, double* psi_out, double* R_out,
                    double* dRdpsi_out) {
    for (int64_t i = 0; i < n; ++i) {
        double a_i = rho[i] - p->offset;
        double I = born_integral(n, x, rho, screen, p, i);
        double psi = a_i * I;
        double phi = p->alpha * psi - p->beta * psi * psi + p->gamma * psi * psi * psi;
        double th = tanh(phi);
        double R = 1.0 / (1.0 / a_i - th / rho[i]);
        if (I_out) I_out[i] = I;
        if (psi_out) psi_out[i] = psi;
        if (R_out) R_out[i] = R;
        if (dRdpsi_out)
            dRdpsi_out[i] = R * R * (1.0 - th * th) *
                            (p->alpha - 2.0 * p->beta * psi + 3.0 * p->gamma * psi * psi) / rho[i];
    }
}

/* Born radii of the m atoms listed in idx only (same definition as above),
 * for spot checks of large molecules: R_out[k] is the radius of atom idx[k]. */
void gbo_born_radii_subset(int64_t n, const double* x, const double* rho, const double* screen,
                           const gbo_params* p, const int64_t* idx, int64_t m, double* R_out) {
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx[k];
        double a_i = rho[i] - p->offset;
        double psi = a_i * born_integral(n, x, rho, screen, p, i);
        double phi = p->alpha * psi - p->beta * psi * psi + p->gamma * psi * psi * psi;
        R_out[k] = 1.0 / (1.0 / a_i - tanh(phi) / rho[i]);
    }
}

/* GB function f_ij = sqrt(r^2 + R_i R_j exp(-r^2 / (4 R_i R_j))). */
static double f_gb(double r, double Ri, double Rj) {
    return sqrt(r * r + Ri * Rj * exp(-r * r / (4.0 * Ri * Rj)));
}

/* Solvent term of the GB kernel with Debye-Hueckel screening by salt (inverse
 * Debye length kappa; kappa = 0 gives the plain form):
 *   g(f) = (1/eps_in - exp(-kappa f) / eps_out) / f,
 * so that E_GB = -1/2 k_e sum_i sum_j q_i q_j g(f_ij) with f_ii = R_i, and its
 * derivative g'(f) = -(1/eps_in - exp(-kappa f)/eps_out) / f^2
 *                    + kappa exp(-kappa f) / (eps_out f). */
static double gb_g(double f, const gbo_params* p) {
    return (1.0 / p->eps_in - exp(-p->kappa * f) / p->eps_out) / f;
}
static double gb_dg(double f, const gbo_params* p) {
    double e = exp(-p->kappa * f);
    return -(1.0 / p->eps_in - e / p->eps_out) / (f * f) + p->kappa * e / (p->eps_out * f);
}

/* Electrostatic energy at fixed Born radii:
 *   E_GB   = -1/2 k_e sum_i sum_j q_i q_j g(f_ij)   (f_ii = R_i; g above: 
 *            (1/eps_in - 1/eps_out) / f without salt)
 *   E_Coul = (k_e / eps_in) sum_{i<j} q_i q_j / r_ij
 * pairs with r_ij > cut are left out when cut > 0 (truncation); self terms
 * are kept.  E[0] = E_GB, E[1] = E_Coul. */
void gbo_energy_fixed_radii(int64_t n, const double* x, const double* q, const double* R,
                            const gbo_params* p, double E[2]) {
    double egb = 0.0, ecoul = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) {
                egb += -0.5 * GBO_KE * q[i] * q[i] * gb_g(R[i], p);
                continue;
            }
            double d[3];
            double r = dist(x, i, j, d);
            if (beyond_cut(r, p)) continue;                /* pair cutoff: truncated */
            egb += -0.5 * GBO_KE * q[i] * q[j] * gb_g(f_gb(r, R[i], R[j]), p);
            if (j > i) ecoul += (GBO_KE / p->eps_in) * q[i] * q[j] / r;
        }
    }
    E[0] = egb;
    E[1] = ecoul;
}

/* Energy, forces F = -dE/dx (3n), charge derivative phi = dE/dq (n), and the
 * Born radii / dE/dR used on the way.  E[0] = E_GB, E[1] = E_Coul.
 * Any of F, phi, R_out, dEdR_out may be NULL. */
void gbo_energy_forces(int64_t n, const double* x, const double* q, const double* rho,
                       const double* screen, const gbo_params* p, double E[2], double* F,
                       double* phi, double* R_out, double* dEdR_out) {
    double* R = (double*)malloc(sizeof(double) * (size_t)n);
    double* dRdpsi = (double*)malloc(sizeof(double) * (size_t)n);
    double* dEdR = (double*)calloc((size_t)n, sizeof(double));
    gbo_born_radii(n, x, rho, screen, p, NULL, NULL, R, dRdpsi);
    double kc = GBO_KE / p->eps_in;
    double egb = 0.0, ecoul = 0.0;
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)n);
    if (phi) memset(phi, 0, sizeof(double) * (size_t)n);

    /* direct part: ordered pairs (i, j), each carrying -1/2 k_e q_i q_j g(f_ij) */
    for (int64_t i = 0; i < n; ++i) {
        egb += -0.5 * GBO_KE * q[i] * q[i] * gb_g(R[i], p);
        dEdR[i] += -0.5 * GBO_KE * q[i] * q[i] * gb_dg(R[i], p);
        if (phi) phi[i] += -GBO_KE * q[i] * gb_g(R[i], p);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            double r = dist(x, i, j, d);
            if (beyond_cut(r, p)) continue;                /* pair cutoff: truncated */
            double RR = R[i] * R[j];
            double D = r * r / (4.0 * RR);
            double e = exp(-D);
            double f = sqrt(r * r + RR * e);
            double c = -0.5 * GBO_KE * q[i] * q[j];
            egb += c * gb_g(f, p);
            /* d(c g(f)) = c g'(f) df, with df/dr = r (1 - e/4) / f,
             * df/dR_i = R_j e (1 + D) / (2 f), df/dR_j = R_i e (1 + D) / (2 f) */
            double dEdf = c * gb_dg(f, p);
            double dEdr = dEdf * r * (1.0 - 0.25 * e) / f;
            dEdR[i] += dEdf * R[j] * e * (1.0 + D) / (2.0 * f);
            dEdR[j] += dEdf * R[i] * e * (1.0 + D) / (2.0 * f);
            if (phi) phi[i] += -GBO_KE * q[j] * gb_g(f, p) + kc * q[j] / r;
            if (j > i) {
                ecoul += kc * q[i] * q[j] / r;
                dEdr += -kc * q[i] * q[j] / (r * r);
            }
            if (F) {
                /* E term depends on r_ij; d r_ij / d x_j = d / r, d x_i = -d / r */
                for (int k = 0; k < 3; ++k) {
                    F[3 * j + k] -= dEdr * d[k] / r;
                    F[3 * i + k] += dEdr * d[k] / r;
                }
            }
        }
    }
    /* Born-radius chain rule: E depends on R_i(psi_i), psi_i = a_i sum_j H(r_ij; a_i, s_j) */
    if (F) {
        for (int64_t i = 0; i < n; ++i) {
            double a_i = rho[i] - p->offset;
            double ci = dEdR[i] * dRdpsi[i] * a_i;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double d[3];
                double r = dist(x, i, j, d);
                double s_j = screen[j] * (rho[j] - p->offset);
                double dEdr = ci * gbo_hct_pair_dr_cut(r, a_i, s_j, p->rgbmax);
                for (int k = 0; k < 3; ++k) {
                    F[3 * j + k] -= dEdr * d[k] / r;
                    F[3 * i + k] += dEdr * d[k] / r;
                }
            }
        }
    }
    E[0] = egb;
    E[1] = ecoul;
    if (R_out) memcpy(R_out, R, sizeof(double) * (size_t)n);
    if (dEdR_out) memcpy(dEdR_out, dEdR, sizeof(double) * (size_t)n);
    free(R);
    free(dRdpsi);
    free(dEdR);
}

/* Chain restraints of the MD driver: bonds (i, i+1) and soft repulsion between
 * non-bonded pairs.  E[0] = bonds, E[1] = repulsion.  Forces are ADDED to F. */
void gbo_restraints(int64_t n, const double* x, const gbo_params* p, double E[2], double* F) {
    double eb = 0.0, er = 0.0;
    for (int64_t i = 0; i + 1 < n; ++i) {
        double d[3];
        double r = dist(x, i, i + 1, d);
        eb += p->bond_k * (r - p->bond_r0) * (r - p->bond_r0);
        double dEdr = 2.0 * p->bond_k * (r - p->bond_r0);
        if (F)
            for (int k = 0; k < 3; ++k) {
                F[3 * (i + 1) + k] -= dEdr * d[k] / r;
                F[3 * i + k] += dEdr * d[k] / r;
            }
    }
    if (p->rep_k != 0.0) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = i + 2; j < n; ++j) {
                double d[3];
                double r = dist(x, i, j, d);
                if (r >= p->rep_sigma) continue;
                er += p->rep_k * (p->rep_sigma - r) * (p->rep_sigma - r);
                double dEdr = -2.0 * p->rep_k * (p->rep_sigma - r);
                if (F)
                    for (int k = 0; k < 3; ++k) {
                        F[3 * j + k] -= dEdr * d[k] / r;
                        F[3 * i + k] += dEdr * d[k] / r;
                    }
            }
    }
    E[0] = eb;
    E[1] = er;
}

/* ------------------------------------------------------------------------ */
/* Monte Carlo state change at fixed Born radii (Eq. 8, Eq. 9)               */
/* ------------------------------------------------------------------------ */

/* One attempt per replica for sites of the given kind (0 = protonation,
 * 1 = redox).  Per replica r:
 *   w = Philox(counter = (r, step, 1 + kind, 0), key = (seed, 0))
 *   site  = the floor((w0>>32) * n_kind / 2^32)-th site of this kind   (Sec. III.A.1)
 *   state = uniform over the site's other states from w1                (Sec. III.A)
 *   dE_elec = E_elec(q') - E_elec(q) by two full evaluations at the same R
 *   dG = dE_elec - (G_ref(s') - G_ref(s))
 *        + F (E - E0_ref) (n_e(s') - n_e(s))             (Eq. 8)
 *        + kT ln10 (pH - pKa_ref) (n_H(s') - n_H(s))     (Eq. 9)
 *   accept iff dG <= 0 or u < exp(-dG / kT), u from w2.
 * On acceptance the site's charges in q and its state are replaced.
 * thresh_out[r] = -kT ln u (the dG at which the decision flips).
 * Replicas without a site of this kind report site_out = -1 and no change. */
void gbo_mc_step(int32_t n_rep, const int64_t* atom_off, const double* x, double* q,
                 const double* R, const int32_t* site_off, const int32_t* site_kind,
                 const int32_t* site_nstates, const int32_t* site_atom_off,
                 const int32_t* site_atom_idx, const int32_t* site_state_off,
                 const int32_t* site_q_off, const float* q_state, const double* G_ref,
                 const int32_t* n_H, const int32_t* n_e, const double* pKa_ref,
                 const double* E0_ref, const double* pH, const double* Epot, double kT,
                 uint64_t seed, uint64_t step, int32_t kind, const gbo_params* p,
                 int32_t* state, double* dG_out, uint8_t* acc_out, double* thresh_out,
                 int32_t* site_out, int32_t* new_state_out) {
    for (int32_t r = 0; r < n_rep; ++r) {
        uint64_t w[4];
        draw(seed, (uint64_t)r, step, 1 + (uint64_t)kind, 0, w);
        int32_t n_kind = 0;
        for (int32_t s = site_off[r]; s < site_off[r + 1]; ++s) n_kind += (site_kind[s] == kind);
        dG_out[r] = 0.0;
        acc_out[r] = 0;
        thresh_out[r] = 0.0;
        site_out[r] = -1;
        new_state_out[r] = -1;
        if (n_kind == 0) continue;
        int32_t want = pick(w[0], n_kind), site = -1;
        for (int32_t s = site_off[r], c = 0; s < site_off[r + 1]; ++s)
            if (site_kind[s] == kind) {
                if (c == want) { site = s; break; }
                ++c;
            }
        int32_t cur = state[site];
        int32_t ns = site_nstates[site];
        int32_t k = pick(w[1], ns - 1);
        int32_t nxt = (k < cur) ? k : k + 1;

        int64_t n = atom_off[r + 1] - atom_off[r];
        const double* xr = x + 3 * atom_off[r];
        double* qr = q + atom_off[r];
        const double* Rr = R + atom_off[r];
        int32_t na = site_atom_off[site + 1] - site_atom_off[site];
        double* q_new = (double*)malloc(sizeof(double) * (size_t)n);
        memcpy(q_new, qr, sizeof(double) * (size_t)n);
        for (int32_t a = 0; a < na; ++a)
            q_new[site_atom_idx[site_atom_off[site] + a]] =
                (double)q_state[site_q_off[site] + nxt * na + a];
        double E0[2], E1[2];
        gbo_energy_fixed_radii(n, xr, qr, Rr, p, E0);
        gbo_energy_fixed_radii(n, xr, q_new, Rr, p, E1);
        double dE = (E1[0] + E1[1]) - (E0[0] + E0[1]);
        int32_t so = site_state_off[site];
        double dG = dE - (G_ref[so + nxt] - G_ref[so + cur]);
        dG += GBO_FARADAY * (Epot[r] - E0_ref[site]) * (double)(n_e[so + nxt] - n_e[so + cur]);
        dG += kT * GBO_LN10 * (pH[r] - pKa_ref[site]) * (double)(n_H[so + nxt] - n_H[so + cur]);
        double u = unif53(w[2]);
        int acc = (dG <= 0.0) || (u < exp(-dG / kT));
        dG_out[r] = dG;
        acc_out[r] = (uint8_t)acc;
        thresh_out[r] = (u > 0.0) ? -kT * log(u) : INFINITY;
        site_out[r] = site;
        new_state_out[r] = nxt;
        if (acc) {
            memcpy(qr, q_new, sizeof(double) * (size_t)n);
            state[site] = nxt;
        }
        free(q_new);
    }
}

/* ------------------------------------------------------------------------ */
/* Per-residue sweep (Sec. III.A.2): one attempt for every site of the kind   */
/* ------------------------------------------------------------------------ */

/* Every site of the requested kind in replica r gets one state-change
 * attempt, the sites taken in a uniformly random order (Sec. III.A.2); each
 * attempt is the one of gbo_mc_step (new state uniform over the other states,
 * dG of Eq. 8 / 9 from two energy evaluations at fixed R, Metropolis) with
 * the charges left by the attempts before it.  Visit i (0-based) draws
 * Philox(key (seed, 0), counter (r, step, 5 + kind, i)): word 0 picks the
 * site among those not yet visited (a Fisher-Yates step over the sites of
 * the kind in index order), word 1 the new state, word 2 gives u.  Per-site
 * outputs (index = global site): dG, threshold -kT ln u, accepted flag,
 * visit position; sites of the other kind get acc = 2 and visit = -1. */
void gbo_mc_sweep(int32_t n_rep, const int64_t* atom_off, const double* x, double* q,
                  const double* R, const int32_t* site_off, const int32_t* site_kind,
                  const int32_t* site_nstates, const int32_t* site_atom_off,
                  const int32_t* site_atom_idx, const int32_t* site_state_off,
                  const int32_t* site_q_off, const float* q_state, const double* G_ref,
                  const int32_t* n_H, const int32_t* n_e, const double* pKa_ref,
                  const double* E0_ref, const double* pH, const double* Epot, double kT,
                  uint64_t seed, uint64_t step, int32_t kind, const gbo_params* p,
                  int32_t* state, double* dG_out, uint8_t* acc_out, double* thresh_out,
                  int32_t* visit_out) {
    for (int32_t r = 0; r < n_rep; ++r) {
        for (int32_t s = site_off[r]; s < site_off[r + 1]; ++s) {
            dG_out[s] = 0.0;
            acc_out[s] = 2;
            thresh_out[s] = 0.0;
            visit_out[s] = -1;
        }
        int32_t n_kind = 0;
        for (int32_t s = site_off[r]; s < site_off[r + 1]; ++s) n_kind += (site_kind[s] == kind);
        if (n_kind == 0) continue;
        int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_kind);
        for (int32_t s = site_off[r], c = 0; s < site_off[r + 1]; ++s)
            if (site_kind[s] == kind) order[c++] = s;
        int64_t n = atom_off[r + 1] - atom_off[r];
        const double* xr = x + 3 * atom_off[r];
        double* qr = q + atom_off[r];
        const double* Rr = R + atom_off[r];
        double* q_new = (double*)malloc(sizeof(double) * (size_t)n);
        for (int32_t i = 0; i < n_kind; ++i) {
            uint64_t w[4];
            draw(seed, (uint64_t)r, step, 5 + (uint64_t)kind, (uint64_t)i, w);
            int32_t j = i + pick(w[0], n_kind - i);
            int32_t tmp = order[i];
            order[i] = order[j];
            order[j] = tmp;
            int32_t site = order[i];
            int32_t cur = state[site];
            int32_t k = pick(w[1], site_nstates[site] - 1);
            int32_t nxt = (k < cur) ? k : k + 1;
            int32_t na = site_atom_off[site + 1] - site_atom_off[site];
            memcpy(q_new, qr, sizeof(double) * (size_t)n);
            for (int32_t a = 0; a < na; ++a)
                q_new[site_atom_idx[site_atom_off[site] + a]] =
                    (double)q_state[site_q_off[site] + nxt * na + a];
            double E0[2], E1[2];
            gbo_energy_fixed_radii(n, xr, qr, Rr, p, E0);
            gbo_energy_fixed_radii(n, xr, q_new, Rr, p, E1);
            double dE = (E1[0] + E1[1]) - (E0[0] + E0[1]);
            int32_t so = site_state_off[site];
            double dG = dE - (G_ref[so + nxt] - G_ref[so + cur]);
            dG += GBO_FARADAY * (Epot[r] - E0_ref[site]) * (double)(n_e[so + nxt] - n_e[so + cur]);
            dG += kT * GBO_LN10 * (pH[r] - pKa_ref[site]) * (double)(n_H[so + nxt] - n_H[so + cur]);
            double u = unif53(w[2]);
            int acc = (dG <= 0.0) || (u < exp(-dG / kT));
            dG_out[site] = dG;
            acc_out[site] = (uint8_t)acc;
            thresh_out[site] = (u > 0.0) ? -kT * log(u) : INFINITY;
            visit_out[site] = i;
            if (acc) {
                memcpy(qr, q_new, sizeof(double) * (size_t)n);
                state[site] = nxt;
            }
        }
        free(q_new);
        free(order);
    }
}

/* ------------------------------------------------------------------------ */
/* Replica exchange along E (Eq. 14-15) or pH                                */
/* ------------------------------------------------------------------------ */

/* Ladders: n_ladders independent ladders of ladder_len slots; slot k of
 * ladder l holds replica rep_at_slot[l*ladder_stride + k*slot_stride] at value
 * values[k].  Attempt number `attempt` pairs neighbours (Sec. III.B):
 * even attempts (0,1),(2,3),...; odd attempts (1,2),(3,4),... and, when `wrap`
 * is set and ladder_len is even, the pair (ladder_len-1, 0).
 * For replica i at value v_a and j at v_b:
 *   Delta = c (v_b - v_a)(N_i - N_j),  c = F/kT (dim 0, E in V) or ln 10 (dim 1, pH)
 * accept iff Delta <= 0 or u < exp(-Delta); u from Philox(l*len + a, attempt, 3, 0).
 * Outputs are written at the pair's first slot index l*len + a; entries of
 * unpaired slots are set to NaN / 0. */
void gbo_exchange(int32_t n_ladders, int32_t ladder_len, int32_t ladder_stride,
                  int32_t slot_stride, const double* values, int32_t* rep_at_slot,
                  const int32_t* n_count, int32_t dim, uint64_t attempt, uint64_t seed,
                  double kT, int32_t wrap, double* delta_out, uint8_t* acc_out) {
    double c = (dim == 0) ? GBO_FARADAY / kT : GBO_LN10;
    for (int32_t l = 0; l < n_ladders; ++l) {
        for (int32_t k = 0; k < ladder_len; ++k) {
            delta_out[l * ladder_len + k] = NAN;
            acc_out[l * ladder_len + k] = 0;
        }
        for (int32_t a = (int32_t)(attempt & 1); a < ladder_len; a += 2) {
            int32_t b = a + 1;
            if (b == ladder_len) {
                if (!(wrap && (attempt & 1) && (ladder_len % 2 == 0))) continue;
                b = 0;
            }
            int32_t* pa = &rep_at_slot[l * ladder_stride + a * slot_stride];
            int32_t* pb = &rep_at_slot[l * ladder_stride + b * slot_stride];
            int32_t i = *pa, j = *pb;
            double delta = c * (values[b] - values[a]) * (double)(n_count[i] - n_count[j]);
            uint64_t w[4];
            draw(seed, (uint64_t)(l * ladder_len + a), attempt, 3, 0, w);
            double u = unif53(w[0]);
            int acc = (delta <= 0.0) || (u < exp(-delta));
            delta_out[l * ladder_len + a] = delta;
            acc_out[l * ladder_len + a] = (uint8_t)acc;
            if (acc) { *pa = j; *pb = i; }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Langevin MD step (BAOAB)                                                  */
/* ------------------------------------------------------------------------ */

/* Standard normals for atom `atom` of replica r at step `step`:
 * w = Philox((r, step, 4, atom), (seed, 0)); Box-Muller on (u1, u2) and (u3, u4)
 * with u1, u3 in (0, 1] and u2, u4 in [0, 1).  Three of the four are used. */
void gbo_normals(uint64_t seed, uint64_t r, uint64_t step, uint64_t atom, double z[4]) {
    uint64_t w[4];
    draw(seed, r, step, 4, atom, w);
    double u1 = ((double)(w[0] >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    double u2 = unif53(w[1]);
    double u3 = ((double)(w[2] >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    double u4 = unif53(w[3]);
    double m1 = sqrt(-2.0 * log(u1)), m2 = sqrt(-2.0 * log(u3));
    z[0] = m1 * cos(2.0 * GBO_PI * u2);
    z[1] = m1 * sin(2.0 * GBO_PI * u2);
    z[2] = m2 * cos(2.0 * GBO_PI * u4);
    z[3] = m2 * sin(2.0 * GBO_PI * u4);
}

/* Total forces (GB + Coulomb + bonds + repulsion) of every replica. */
void gbo_forces_all(int32_t n_rep, const int64_t* atom_off, const double* x, const double* q,
                    const double* rho, const double* screen, const gbo_params* p, double* F,
                    double* E_out /* n_rep x 4: GB, Coul, bond, rep */) {
    for (int32_t r = 0; r < n_rep; ++r) {
        int64_t o = atom_off[r], n = atom_off[r + 1] - atom_off[r];
        double E[2], Er[2];
        gbo_energy_forces(n, x + 3 * o, q + o, rho + o, screen + o, p, E, F + 3 * o, NULL,
                          NULL, NULL);
        gbo_restraints(n, x + 3 * o, p, Er, F + 3 * o);
        if (E_out) {
            E_out[4 * r + 0] = E[0];
            E_out[4 * r + 1] = E[1];
            E_out[4 * r + 2] = Er[0];
            E_out[4 * r + 3] = Er[1];
        }
    }
}

/* One BAOAB step for every replica (mass m, friction gamma, temperature kT):
 *   B: v += dt/2 F/m ; A: x += dt/2 v ; O: v = c1 v + c2 z ; A: x += dt/2 v ;
 *   F = F(x) ; B: v += dt/2 F/m
 * with c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT / m).  F holds the forces
 * at the incoming x and is replaced by those at the outgoing x. */
void gbo_md_step(int32_t n_rep, const int64_t* atom_off, double* x, double* v, const double* q,
                 const double* rho, const double* screen, const gbo_params* p, double* F,
                 uint64_t seed, uint64_t step, double* E_out) {
    int64_t ntot = atom_off[n_rep];
    double inv_m = GBO_ACCEL / p->mass;
    double c1 = exp(-p->friction * p->dt);
    double c2 = sqrt((1.0 - c1 * c1) * p->kT * GBO_ACCEL / p->mass);
    double h = 0.5 * p->dt;
    for (int32_t r = 0; r < n_rep; ++r) {
        for (int64_t i = atom_off[r]; i < atom_off[r + 1]; ++i) {
            double z[4];
            gbo_normals(seed, (uint64_t)r, step, (uint64_t)(i - atom_off[r]), z);
            for (int k = 0; k < 3; ++k) {
                double vv = v[3 * i + k] + h * F[3 * i + k] * inv_m;
                double xx = x[3 * i + k] + h * vv;
                vv = c1 * vv + c2 * z[k];
                xx += h * vv;
                v[3 * i + k] = vv;
                x[3 * i + k] = xx;
            }
        }
    }
    gbo_forces_all(n_rep, atom_off, x, q, rho, screen, p, F, E_out);
    for (int64_t i = 0; i < ntot; ++i)
        for (int k = 0; k < 3; ++k) v[3 * i + k] += h * F[3 * i + k] * inv_m;
}
