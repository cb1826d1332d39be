/*
 * rime_oracle.h -- plain FP64 CPU oracle for the RIME predict + weighted chi^2.
 *
 * TEST INFRASTRUCTURE. Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code, header,
 * table or helper with the CUDA library; the product path never calls it.
 *
 * Conventions (shared with the library's public API by definition, not code):
 *   baselines: pairs (p, q), p < q, canonical row-major upper-triangle order;
 *   correlations: the 2x2 matrix in row-major order (00, 01, 10, 11);
 *   complex numbers: interleaved (re, im) doubles.
 */
#ifndef RIME_ORACLE_H
#define RIME_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int na, ntime, nchan, nsrc;
    int stokes_time_varying;   /* 1: stokes is [ntime][nsrc][4] */
    double ref_freq_hz;        /* nu_ref of eq. 2 */
    double beam_c;             /* C of eq. 4, rad^-1 GHz^-1 */
    int beam_model;            /* 0: cos^3 (eq. 4); 1: 2 J1(x)/x (Sec. 2.1's Jinc) */
    const double *uvw;         /* [ntime][na][3] metres */
    const double *freq_hz;     /* [nchan] */
    const double *lm;          /* [nsrc][2] radians */
    const double *stokes;      /* [nsrc][4] or [ntime][nsrc][4]: I, Q, U, V */
    const double *alpha;       /* [nsrc] spectral index */
    const double *shape;       /* [nsrc][3] major, minor, pa; NULL = points */
    const int *kind;           /* [nsrc] morphology of a source with a shape: 0 Gaussian
                                  (major, minor = FWHM), 1 exponential disk (major, minor =
                                  scale lengths); NULL = all Gaussian */
    const double *pointing;    /* [ntime][na][2] (dl, dm) or NULL */
    const double *gains;       /* [ntime][na][nchan][4] complex or NULL (identity) */
    const double *data;        /* [ntime][nbl][nchan][4] complex */
    const double *weight;      /* [ntime][nbl][nchan] */
} rime_oracle_problem;

/* One visibility V_tpqk (2x2 complex, 8 doubles). Any p != q is accepted. */
void rime_oracle_vis(const rime_oracle_problem *P, int t, int p, int q, int k,
                     double *out8);

/* Visibilities at a list of n (t, p, q, k) points. */
void rime_oracle_vis_list(const rime_oracle_problem *P, long n, const int *t,
                          const int *p, const int *q, const int *k, double *out8n);

/* All model visibilities [t0..t1)[nbl][nchan][4] complex. */
void rime_oracle_predict(const rime_oracle_problem *P, int t0, int t1, double *vis);

/* chi^2 over timesteps [t0, t1) (eq. 7 without the ln term). */
double rime_oracle_chi2(const rime_oracle_problem *P, int t0, int t1);

/* chi^2 and its gradient.
 *   grad_src   [nsrc][10]: d/d(l, m, I, Q, U, V, alpha, major, minor, pa)
 *   grad_gains [ntime][na][nchan][4] complex: dchi2/dRe G + i dchi2/dIm G,
 *              may be NULL.  Static brightness only. */
double rime_oracle_chi2_grad(const rime_oracle_problem *P, double *grad_src,
                             double *grad_gains);

/* The likelihood constant sum ln(2 pi / w) over all visibilities (eq. 7). */
double rime_oracle_ln_norm(const rime_oracle_problem *P);

/* The phase of eq. 3 in turns, nu tau, reduced to nu tau - round(nu tau)
 * (nearest integer, ties to even), for n pairs. */
void rime_oracle_reduced_phase(long n, const double *nu, const double *tau, double *out);

/* Number of threads the parallel loops use. */
int rime_oracle_threads(void);

#ifdef __cplusplus
}
#endif
#endif
