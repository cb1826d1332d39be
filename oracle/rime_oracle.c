/*
 * rime_oracle.c -- plain FP64 CPU oracle for the RIME predict + weighted chi^2
 * (Montblanc, arXiv 1501.07719).
 *
 * TEST INFRASTRUCTURE. Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg load this library; the product path never does.
 *
 * It evaluates the definition term by term, with no blocking, factoring or
 * reordering:
 *   Eq. 1   V_tpq = G_tp ( sum_s E_tps K_tps B_s K_tqs^H E_tqs^H ) G_tq^H
 *           (the \RGqAll macro of the paper prints G_tp^H; the text says the
 *           Hermitian transpose is applied to the antenna-q terms: G_tq^H)
 *   Eq. 2   B_s = (lambda_ref / lambda)^alpha [[I+Q, U+iV], [U-iV, I-Q]]
 *   Eq. 3   K_tps = exp(2 pi i (u l + v m + w (n - 1)) / lambda), n = sqrt(1-l^2-m^2)
 *   Eq. 4   E_ps = cos^3(C lambda |l_s - dl_p|), read as cos^3(C nu_GHz rho)
 *           with C in rad^-1 GHz^-1, the argument clamped at pi/2 (E = 0 past
 *           the first null). Sec. 2.1 names a Jinc function for the VLA beam
 *           in its place; beam_model 1 takes E = 2 J1(x) / x with the same
 *           x = C nu_GHz rho (the Airy pattern of a uniformly illuminated
 *           dish, unclamped: its sidelobes change sign).
 *   Eqs. 5-6 source coherency E_p K_p B K_q^H E_q^H, summed over sources
 *   Eq. 7   chi^2 = sum w (V - D)^2, read as w times the sum over the four
 *           correlations of |V_c - D_c|^2; the ln(2 pi / w) term separately.
 * Gaussian sources (Sec. 2.1 names point and Gaussian morphologies, Table 2
 * lists "gaussian shapes", no formula is given): the brightness B is scaled by
 * the Fourier transform of a unit-flux elliptical Gaussian with FWHM axes
 * (major, minor) and position angle pa measured from +m towards +l, evaluated
 * at the baseline (u_p - u_q, v_p - v_q) / lambda:
 *   g = exp(-pi^2 (major^2 u_maj^2 + minor^2 u_min^2) / (4 ln 2)),
 *   u_maj = u sin pa + v cos pa,  u_min = u cos pa - v sin pa.
 * Sec. 1 names further morphologies (Sersic profiles among them) without a
 * formula; kind 1 is the Sersic profile of index 1, an elliptical exponential
 * disk exp(-r) in the coordinates (x_maj / major, x_min / minor) (major,
 * minor the scale lengths, pa as above), whose unit-flux Fourier transform is
 *   g = (1 + 4 pi^2 (major^2 u_maj^2 + minor^2 u_min^2))^(-3/2).
 * chi^2 uses Neumaier-compensated summation in the order (t, bl, k, c).
 *
 * Pinned by tests/test_oracle_pins.py (closed forms, invariants, an image-plane
 * quadrature of the Gaussian, a matrix formulation, finite differences).
 */
/* j0 / j1 (Bessel functions of the first kind) are X/Open math functions */
#define _XOPEN_SOURCE 700
#include "rime_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#undef I /* complex.h's imaginary unit macro; Stokes I is spelled sI below */
#define IMAG _Complex_I

typedef double complex cplx;

static const double C_LIGHT = 299792458.0;
static const double PI = 3.14159265358979323846;

/* ---------------- Neumaier (improved Kahan) summation ------------------- */
typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

/* ---------------- 2x2 complex matrices, row-major (00, 01, 10, 11) ------ */
static void mat_mul(const cplx a[4], const cplx b[4], cplx out[4]) {
    cplx r[4];
    r[0] = a[0] * b[0] + a[1] * b[2];
    r[1] = a[0] * b[1] + a[1] * b[3];
    r[2] = a[2] * b[0] + a[3] * b[2];
    r[3] = a[2] * b[1] + a[3] * b[3];
    memcpy(out, r, sizeof r);
}
static void mat_herm(const cplx a[4], cplx out[4]) {
    cplx r[4] = {conj(a[0]), conj(a[2]), conj(a[1]), conj(a[3])};
    memcpy(out, r, sizeof r);
}
/* G_p X G_q^H (the outer products of eq. 1) */
static void sandwich(const cplx gp[4], const cplx x[4], const cplx gq[4], cplx out[4]) {
    cplx gqh[4], t[4];
    mat_herm(gq, gqh);
    mat_mul(gp, x, t);
    mat_mul(t, gqh, out);
}

static long nbl_of(int na) { return (long)na * (na - 1) / 2; }

static long bl_index(int na, int p, int q) { /* p < q */
    return (long)p * na - (long)p * (p + 1) / 2 + (q - p - 1);
}

static void load_gain(const rime_oracle_problem *P, int t, int a, int k, cplx g[4]) {
    if (!P->gains) {
        g[0] = 1; g[1] = 0; g[2] = 0; g[3] = 1;
        return;
    }
    const double *x = P->gains + 8 * (((long)t * P->na + a) * P->nchan + k);
    for (int c = 0; c < 4; c++) g[c] = x[2 * c] + IMAG * x[2 * c + 1];
}

static const double *stokes_of(const rime_oracle_problem *P, int t, int s) {
    if (P->stokes_time_varying) return P->stokes + 4 * ((long)t * P->nsrc + s);
    return P->stokes + 4 * (long)s;
}

/* n - 1 = (n^2 - 1) / (n + 1) = -(l^2 + m^2) / (1 + n): same value, no cancellation. */
static double n_minus_1(double l, double m) {
    double r2 = l * l + m * m;
    return -r2 / (1.0 + sqrt(1.0 - r2));
}

/* ---------------- per-antenna and per-source factors -------------------- */
typedef struct {
    double E;          /* eq. 4 */
    double dE_dl, dE_dm;
    cplx K;            /* eq. 3 */
    cplx dK_dl, dK_dm;
} antenna_term;

/* The beam of eq. 4 as a function of x = C nu_GHz rho, and (dE/dx) / x.
 *   model 0: E = cos^3 x for x < pi/2, 0 past it;
 *            dE/dx = -3 cos^2 x sin x, so (dE/dx)/x = -3 cos^2 x (sin x / x).
 *   model 1: E = 2 J1(x) / x; with J1' = J0 - J1/x, dE/dx = 2 (J0 - 2 J1/x) / x
 *            = -2 J2(x) / x, so (dE/dx)/x = -2 (2 J1(x)/x - J0(x)) / x^2.
 *            Near x = 0 the power series of 2 J1(x)/x,
 *            sum_k (-1)^k (x/2)^(2k) / (k! (k+1)!) = 1 - x^2/8 + x^4/192 - ...,
 *            and of its derivative over x, -1/4 + x^2/48 - x^4/1536 + ...,
 *            avoid the cancellation of 2 J1/x - J0 (J0, J1: libm's j0, j1). */
static void beam_factor(int model, double x, double *E, double *dEx) {
    if (model == 1) {
        if (x < 0.05) {
            double x2 = x * x;
            *E = 1.0 - x2 / 8.0 + x2 * x2 / 192.0 - x2 * x2 * x2 / 9216.0;
            *dEx = -0.25 + x2 / 48.0 - x2 * x2 / 1536.0 + x2 * x2 * x2 / 92160.0;
        } else {
            double j1x = j1(x), j0x = j0(x);
            *E = 2.0 * j1x / x;
            *dEx = -2.0 * (2.0 * j1x / x - j0x) / (x * x);
        }
        return;
    }
    if (x >= PI / 2) {
        *E = 0.0;
        *dEx = 0.0;
        return;
    }
    double c = cos(x);
    double sinc = (x < 1e-8) ? 1.0 : sin(x) / x;
    *E = c * c * c;
    *dEx = -3.0 * c * c * sinc;
}

/* Eq. 3 and eq. 4 for antenna a, with the derivatives the gradient needs. */
static antenna_term antenna_factor(const rime_oracle_problem *P, int t, int a,
                                   double l, double m, double nu, double lambda) {
    antenna_term r;
    const double *uvw = P->uvw + 3 * ((long)t * P->na + a);
    double n1 = n_minus_1(l, m);
    double n = sqrt(1.0 - l * l - m * m);
    double phi = 2.0 * PI * (uvw[0] * l + uvw[1] * m + uvw[2] * n1) / lambda;
    r.K = cos(phi) + IMAG * sin(phi);
    /* d(n - 1)/dl = -l / n */
    r.dK_dl = r.K * IMAG * (2.0 * PI / lambda) * (uvw[0] + uvw[2] * (-l / n));
    r.dK_dm = r.K * IMAG * (2.0 * PI / lambda) * (uvw[1] + uvw[2] * (-m / n));

    double dl = 0.0, dm = 0.0;
    if (P->pointing) {
        dl = P->pointing[2 * ((long)t * P->na + a)];
        dm = P->pointing[2 * ((long)t * P->na + a) + 1];
    }
    double rho = hypot(l - dl, m - dm);
    double cnu = P->beam_c * (nu * 1e-9);
    double x = cnu * rho;
    double E, dEx;   /* E(x) and (dE/dx) / x */
    beam_factor(P->beam_model, x, &E, &dEx);
    r.E = E;
    /* dE/dl = dE/dx * cnu * (l - dl) / rho = (dE/dx / x) cnu^2 (l - dl), finite at rho = 0 */
    r.dE_dl = dEx * cnu * cnu * (l - dl);
    r.dE_dm = dEx * cnu * cnu * (m - dm);
    return r;
}

typedef struct {
    double g;          /* Gaussian shape factor (1 for points) */
    double dg_dmaj, dg_dmin, dg_dpa;
} shape_term;

static shape_term shape_factor(const rime_oracle_problem *P, int s, double du,
                               double dv, double lambda) {
    shape_term r = {1.0, 0.0, 0.0, 0.0};
    if (!P->shape) return r;
    const double *sh = P->shape + 3 * (long)s;
    double maj = sh[0], mn = sh[1], pa = sh[2];
    if (maj == 0.0 && mn == 0.0) return r;
    double u = du / lambda, v = dv / lambda;
    double umaj = u * sin(pa) + v * cos(pa);
    double umin = u * cos(pa) - v * sin(pa);
    if (P->kind && P->kind[s] == 1) {
        /* exponential disk: g = (1 + q)^(-3/2), q = 4 pi^2 (major^2 u_maj^2 + minor^2 u_min^2),
         * dg/dtheta = -3/2 (1 + q)^(-5/2) dq/dtheta */
        double kd = 4.0 * PI * PI;
        double q = kd * (maj * maj * umaj * umaj + mn * mn * umin * umin);
        r.g = pow(1.0 + q, -1.5);
        double dgdq = -1.5 * r.g / (1.0 + q);
        r.dg_dmaj = dgdq * kd * 2.0 * maj * umaj * umaj;
        r.dg_dmin = dgdq * kd * 2.0 * mn * umin * umin;
        r.dg_dpa = dgdq * kd * (2.0 * maj * maj * umaj * umin - 2.0 * mn * mn * umin * umaj);
        return r;
    }
    double k = PI * PI / (4.0 * log(2.0));
    r.g = exp(-k * (maj * maj * umaj * umaj + mn * mn * umin * umin));
    r.dg_dmaj = r.g * (-k) * 2.0 * maj * umaj * umaj;
    r.dg_dmin = r.g * (-k) * 2.0 * mn * umin * umin;
    /* d umaj / d pa = umin, d umin / d pa = -umaj */
    r.dg_dpa = r.g * (-k) * (2.0 * maj * maj * umaj * umin - 2.0 * mn * mn * umin * umaj);
    return r;
}

/* Eq. 2 brightness without its spectral factor. */
static void brightness(const double *st, cplx B[4]) {
    double sI = st[0], sQ = st[1], sU = st[2], sV = st[3];
    B[0] = sI + sQ;
    B[1] = sU + IMAG * sV;
    B[2] = sU - IMAG * sV;
    B[3] = sI - sQ;
}

/* Source coherency sum S = sum_s E_p K_p B_s K_q^H E_q^H (eqs. 5-6). */
static void coherency_sum(const rime_oracle_problem *P, int t, int p, int q, int k,
                          cplx S[4]) {
    double nu = P->freq_hz[k];
    double lambda = C_LIGHT / nu;
    double lambda_ref = C_LIGHT / P->ref_freq_hz;
    const double *up = P->uvw + 3 * ((long)t * P->na + p);
    const double *uq = P->uvw + 3 * ((long)t * P->na + q);
    for (int c = 0; c < 4; c++) S[c] = 0;
    for (int s = 0; s < P->nsrc; s++) {
        double l = P->lm[2 * s], m = P->lm[2 * s + 1];
        antenna_term ap = antenna_factor(P, t, p, l, m, nu, lambda);
        antenna_term aq = antenna_factor(P, t, q, l, m, nu, lambda);
        double spec = pow(lambda_ref / lambda, P->alpha[s]);
        shape_term sh = shape_factor(P, s, up[0] - uq[0], up[1] - uq[1], lambda);
        cplx B[4];
        brightness(stokes_of(P, t, s), B);
        cplx z = (ap.E * ap.K) * conj(aq.E * aq.K);
        for (int c = 0; c < 4; c++) S[c] += z * (spec * sh.g * B[c]);
    }
}

void rime_oracle_vis(const rime_oracle_problem *P, int t, int p, int q, int k,
                     double *out8) {
    cplx S[4], gp[4], gq[4], V[4];
    coherency_sum(P, t, p, q, k, S);
    load_gain(P, t, p, k, gp);
    load_gain(P, t, q, k, gq);
    sandwich(gp, S, gq, V); /* eq. 1 */
    for (int c = 0; c < 4; c++) {
        out8[2 * c] = creal(V[c]);
        out8[2 * c + 1] = cimag(V[c]);
    }
}

void rime_oracle_vis_list(const rime_oracle_problem *P, long n, const int *t,
                          const int *p, const int *q, const int *k, double *out8n) {
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < n; i++)
        rime_oracle_vis(P, t[i], p[i], q[i], k[i], out8n + 8 * i);
}

void rime_oracle_predict(const rime_oracle_problem *P, int t0, int t1, double *vis) {
    long nbl = nbl_of(P->na);
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = t0; t < t1; t++)
        for (int p = 0; p < P->na; p++)
            for (int q = p + 1; q < P->na; q++)
                for (int k = 0; k < P->nchan; k++) {
                    long row = (((long)(t - t0) * nbl + bl_index(P->na, p, q)) * P->nchan + k);
                    rime_oracle_vis(P, t, p, q, k, vis + 8 * row);
                }
}

/* w * sum_c |V_c - D_c|^2 for one visibility (eq. 7). */
static double chi2_term(const rime_oracle_problem *P, int t, int p, int q, int k,
                        const double V8[8]) {
    long nbl = nbl_of(P->na);
    long row = ((long)t * nbl + bl_index(P->na, p, q)) * P->nchan + k;
    const double *D = P->data + 8 * row;
    double w = P->weight[row];
    double acc = 0.0;
    for (int c = 0; c < 4; c++) {
        double dr = V8[2 * c] - D[2 * c];
        double di = V8[2 * c + 1] - D[2 * c + 1];
        acc += dr * dr + di * di;
    }
    return w * acc;
}

double rime_oracle_chi2(const rime_oracle_problem *P, int t0, int t1) {
    if (t1 <= t0) return 0.0;
    double *part = (double *)calloc((size_t)(t1 - t0), 2 * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = t0; t < t1; t++) {
        nsum acc = {0.0, 0.0};
        for (int p = 0; p < P->na; p++)
            for (int q = p + 1; q < P->na; q++)
                for (int k = 0; k < P->nchan; k++) {
                    double V8[8];
                    rime_oracle_vis(P, t, p, q, k, V8);
                    nsum_add(&acc, chi2_term(P, t, p, q, k, V8));
                }
        part[2 * (t - t0)] = acc.s;
        part[2 * (t - t0) + 1] = acc.c;
    }
    nsum tot = {0.0, 0.0};
    for (int t = t0; t < t1; t++) {
        nsum_add(&tot, part[2 * (t - t0)]);
        nsum_add(&tot, part[2 * (t - t0) + 1]);
    }
    free(part);
    return nsum_get(&tot);
}

double rime_oracle_ln_norm(const rime_oracle_problem *P) {
    long n = (long)P->ntime * nbl_of(P->na) * P->nchan;
    nsum acc = {0.0, 0.0};
    for (long i = 0; i < n; i++) nsum_add(&acc, log(2.0 * PI / P->weight[i]));
    return nsum_get(&acc);
}

/* 2 w Re sum_c conj(R_c) dV_c : the derivative of w sum_c |V_c - D_c|^2
 * along dV (product rule on eq. 7). */
static double contract(double w, const cplx R[4], const cplx dV[4]) {
    double acc = 0.0;
    for (int c = 0; c < 4; c++) acc += creal(conj(R[c]) * dV[c]);
    return 2.0 * w * acc;
}

double rime_oracle_chi2_grad(const rime_oracle_problem *P, double *grad_src,
                             double *grad_gains) {
    const int NP = 10;
    int nsrc = P->nsrc;
    long nbl = nbl_of(P->na);
    double lambda_ref = C_LIGHT / P->ref_freq_hz;
    /* per-timestep partials, summed in t order afterwards */
    nsum *gpart = (nsum *)calloc((size_t)P->ntime * nsrc * NP + 1, sizeof(nsum));
    nsum *cpart = (nsum *)calloc((size_t)P->ntime, sizeof(nsum));
    nsum *ggain = NULL;
    if (grad_gains)
        ggain = (nsum *)calloc((size_t)P->ntime * P->na * P->nchan * 8, sizeof(nsum));

#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < P->ntime; t++) {
        nsum *gs = gpart + (size_t)t * nsrc * NP;
        for (int p = 0; p < P->na; p++)
            for (int q = p + 1; q < P->na; q++)
                for (int k = 0; k < P->nchan; k++) {
                    long row = ((long)t * nbl + bl_index(P->na, p, q)) * P->nchan + k;
                    double nu = P->freq_hz[k];
                    double lambda = C_LIGHT / nu;
                    const double *up = P->uvw + 3 * ((long)t * P->na + p);
                    const double *uq = P->uvw + 3 * ((long)t * P->na + q);
                    cplx S[4], gp[4], gq[4], V[4], R[4];
                    coherency_sum(P, t, p, q, k, S);
                    load_gain(P, t, p, k, gp);
                    load_gain(P, t, q, k, gq);
                    sandwich(gp, S, gq, V);
                    const double *D = P->data + 8 * row;
                    double w = P->weight[row];
                    double chi = 0.0;
                    for (int c = 0; c < 4; c++) {
                        R[c] = V[c] - (D[2 * c] + IMAG * D[2 * c + 1]);
                        chi += creal(R[c]) * creal(R[c]) + cimag(R[c]) * cimag(R[c]);
                    }
                    nsum_add(&cpart[t], w * chi);

                    /* source parameters: dV = G_p dS G_q^H */
                    for (int s = 0; s < nsrc; s++) {
                        double l = P->lm[2 * s], m = P->lm[2 * s + 1];
                        antenna_term ap = antenna_factor(P, t, p, l, m, nu, lambda);
                        antenna_term aq = antenna_factor(P, t, q, l, m, nu, lambda);
                        double spec = pow(lambda_ref / lambda, P->alpha[s]);
                        shape_term sh = shape_factor(P, s, up[0] - uq[0], up[1] - uq[1], lambda);
                        cplx B[4];
                        brightness(stokes_of(P, t, s), B);
                        cplx Ap = ap.E * ap.K, Aq = aq.E * aq.K;
                        cplx z = Ap * conj(Aq);
                        cplx dAp_dl = ap.dE_dl * ap.K + ap.E * ap.dK_dl;
                        cplx dAq_dl = aq.dE_dl * aq.K + aq.E * aq.dK_dl;
                        cplx dAp_dm = ap.dE_dm * ap.K + ap.E * ap.dK_dm;
                        cplx dAq_dm = aq.dE_dm * aq.K + aq.E * aq.dK_dm;
                        cplx dz_dl = dAp_dl * conj(Aq) + Ap * conj(dAq_dl);
                        cplx dz_dm = dAp_dm * conj(Aq) + Ap * conj(dAq_dm);
                        double fg = spec * sh.g;
                        cplx dS[10][4];
                        for (int c = 0; c < 4; c++) {
                            dS[0][c] = dz_dl * fg * B[c];
                            dS[1][c] = dz_dm * fg * B[c];
                            dS[6][c] = z * fg * B[c] * log(lambda_ref / lambda);
                            dS[7][c] = z * spec * sh.dg_dmaj * B[c];
                            dS[8][c] = z * spec * sh.dg_dmin * B[c];
                            dS[9][c] = z * spec * sh.dg_dpa * B[c];
                        }
                        cplx zf = z * fg;
                        /* dB/dI, dB/dQ, dB/dU, dB/dV from eq. 2 */
                        dS[2][0] = zf;  dS[2][1] = 0;          dS[2][2] = 0;          dS[2][3] = zf;
                        dS[3][0] = zf;  dS[3][1] = 0;          dS[3][2] = 0;          dS[3][3] = -zf;
                        dS[4][0] = 0;   dS[4][1] = zf;         dS[4][2] = zf;         dS[4][3] = 0;
                        dS[5][0] = 0;   dS[5][1] = IMAG * zf;  dS[5][2] = -IMAG * zf; dS[5][3] = 0;
                        for (int j = 0; j < NP; j++) {
                            cplx dV[4];
                            sandwich(gp, dS[j], gq, dV);
                            nsum_add(&gs[s * NP + j], contract(w, R, dV));
                        }
                    }

                    /* gains: V = G_p S G_q^H */
                    if (ggain) {
                        cplx SGqh[4], GpS[4], gqh[4];
                        mat_herm(gq, gqh);
                        mat_mul(S, gqh, SGqh);
                        mat_mul(gp, S, GpS);
                        for (int ij = 0; ij < 4; ij++) {
                            int i = ij / 2, j = ij % 2;
                            cplx Eij[4] = {0, 0, 0, 0}, Eji[4] = {0, 0, 0, 0};
                            Eij[ij] = 1;
                            Eji[j * 2 + i] = 1;
                            cplx dVr[4], dVi[4];
                            /* d/dRe (G_p)_ij : E_ij S G_q^H ; d/dIm : i E_ij S G_q^H */
                            mat_mul(Eij, SGqh, dVr);
                            for (int c = 0; c < 4; c++) dVi[c] = IMAG * dVr[c];
                            nsum *gpij = ggain + 8 * (((long)t * P->na + p) * P->nchan + k) + 2 * ij;
                            nsum_add(&gpij[0], contract(w, R, dVr));
                            nsum_add(&gpij[1], contract(w, R, dVi));
                            /* d/dRe (G_q)_ij : G_p S E_ji ; d/dIm : -i G_p S E_ji */
                            mat_mul(GpS, Eji, dVr);
                            for (int c = 0; c < 4; c++) dVi[c] = -IMAG * dVr[c];
                            nsum *gqij = ggain + 8 * (((long)t * P->na + q) * P->nchan + k) + 2 * ij;
                            nsum_add(&gqij[0], contract(w, R, dVr));
                            nsum_add(&gqij[1], contract(w, R, dVi));
                        }
                    }
                }
    }
    nsum chi = {0.0, 0.0};
    for (int t = 0; t < P->ntime; t++) {
        nsum_add(&chi, cpart[t].s);
        nsum_add(&chi, cpart[t].c);
    }
    for (int s = 0; s < nsrc; s++)
        for (int j = 0; j < NP; j++) {
            nsum acc = {0.0, 0.0};
            for (int t = 0; t < P->ntime; t++) {
                nsum_add(&acc, gpart[((size_t)t * nsrc + s) * NP + j].s);
                nsum_add(&acc, gpart[((size_t)t * nsrc + s) * NP + j].c);
            }
            grad_src[s * NP + j] = nsum_get(&acc);
        }
    if (ggain) {
        long n = (long)P->ntime * P->na * P->nchan * 8;
        for (long i = 0; i < n; i++) grad_gains[i] = nsum_get(&ggain[i]);
        free(ggain);
    }
    free(gpart);
    free(cpart);
    return nsum_get(&chi);
}

/* eq. 3: K = exp(2 pi i nu tau) depends on nu tau only through its
 * remainder modulo whole turns; this is that remainder, nearest integer
 * removed (the definition, in FP64). */
void rime_oracle_reduced_phase(long n, const double *nu, const double *tau, double *out) {
    for (long i = 0; i < n; i++) {
        const double x = nu[i] * tau[i];
        out[i] = x - nearbyint(x);
    }
}

int rime_oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
