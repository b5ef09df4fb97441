/*
 * spstd_oracle.h -- plain, slow, FP64 CPU oracle for the SPSTD method
 * (Shen, Sha, Kuang, Hu, Huang, Wu, "Symplectic Pseudospectral Time-Domain
 * Scheme for Solving Time-Dependent Schroedinger Equation", arXiv 1805.03155).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library in paper_1805_03155_gb300/;
 * the two are checked against each other, never built from each other.
 *
 * Everything is FP64, single threaded, unblocked: every function follows the
 * paper's definition step by step so that it can be read against the paper.
 *
 * Grid convention: field arrays are [n[2]][n[1]][n[0]] with x (axis 0)
 * fastest; x_j = lo + j*(hi-lo)/n (periodic box, right end excluded).
 */
#ifndef SPSTD_ORACLE_H
#define SPSTD_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dims;            /* 1, 2 or 3 */
    int64_t n[3];        /* points per axis (unused axes = 1) */
    double lo[3], hi[3]; /* periodic box per axis */
    double hbar, mass;   /* hbar and effective mass m* */
    int nyquist_zero;    /* 0: keep k_Nyq^2 = (pi/dx)^2, 1: zero the Nyquist mode */
    int bc[3];           /* per axis: ORC_PERIODIC, ORC_DIRICHLET or ORC_NEUMANN */
} orc_grid;

/* Boundary conditions (Section 2.2): the DFT for periodic or decaying fields,
 * the DST for Dirichlet walls (infinite well), the DCT for Neumann walls.
 *  ORC_PERIODIC  n points x_j = lo + j L/n, right end excluded;
 *  ORC_DIRICHLET n interior points x_j = lo + (j+1) L/(n+1), psi = 0 at lo, hi;
 *  ORC_NEUMANN   n points x_j = lo + j L/(n-1) including both walls, where
 *                d psi/dx = 0. */
enum { ORC_PERIODIC = 0, ORC_DIRICHLET = 1, ORC_NEUMANN = 2 };

/* Integrator presets (ids shared by value only with the CUDA library). */
enum { ORC_LEAPFROG = 0, ORC_STRANG = 1, ORC_PAPER3 = 2, ORC_FR4 = 3, ORC_SUZUKI6 = 4 };

int    orc_preset(int id, double *c, double *d, int *m);
int    orc_fft(double *re, double *im, int64_t n, int sign);
int    orc_laplacian_axis(const double *f, double *out, const orc_grid *g, int axis);
int    orc_apply_K(const double *src, const double *V, double *out, const orc_grid *g);
int    orc_run(double *psiR, double *psiI, const double *V, const orc_grid *g,
               const double *c, const double *d, int m, double dt, int64_t nsteps,
               int n_probe, const int64_t *probe_idx, double *probe_re, double *probe_im);
double orc_trace(const double *c, const double *d, int m, double s);
void   orc_evolution_matrix(const double *c, const double *d, int m, double s, double *M4);
double orc_stability_limit(const double *c, const double *d, int m);
int    orc_spectrum(const double *re, const double *im, int64_t M, int64_t nfft, int max_peaks,
                    double thresh, double dt, double hbar,
                    double *theta, double *E, double *amp);
double orc_phase_correct(double theta, const double *c, const double *d, int m);
int    orc_norm_energy(const double *psiR, const double *psiI, const double *V,
                       const orc_grid *g, double *norm, double *energy);
int    orc_run_rk4(double *psiR, double *psiI, const double *V, const orc_grid *g, double dt, int64_t nsteps,
                   int n_probe, const int64_t *probe_idx, double *probe_re, double *probe_im);
int    orc_run_eigen(double *psiR, double *psiI, const double *V, const orc_grid *g,
                     const double *c, const double *d, int m, double dt, int64_t nsteps,
                     int n_target, const double *E, double *acc_re, double *acc_im);

#ifdef __cplusplus
}
#endif
#endif
