/*
 * CPU oracle for sign(H_W(mu)) b by restarted LR-deflated multishift FOM.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow FP64 C written from the paper
 * (Bloch et al., "Krylov subspace methods and the sign function: multishifts
 * and deflation in the non-Hermitian case", Lattice 2009).  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header or table with the CUDA library.
 *
 * Complex numbers are C99 `double complex`.  Layouts:
 *   field  psi[site][spin 4][colour 3]         site = x + Lx*(y + Ly*(z + Lz*t))
 *   links  U[site][dir 4][3][3] (row-major)     dir = x, y, z, t
 *   deflation blocks R, L: n x m column-major (column j = vector j)
 */
#ifndef SGN_ORACLE_H
#define SGN_ORACLE_H

#include <complex.h>
#include <stdint.h>

typedef double complex orc_c;

typedef struct {
    int dims[4];          /* Lx, Ly, Lz, Lt */
    int antiperiodic[4];  /* 1: antiperiodic boundary in that direction */
    double mu;            /* quark chemical potential (time hops carry e^{+-mu}) */
    double mass;          /* Wilson kernel mass m_W (the configurations use -1.6) */
} orc_lattice;

typedef struct {
    int cycles;           /* restart cycles run */
    int matvecs;          /* applications of H_W */
    int converged;        /* 1 if every shifted system met the tolerance */
    int breakdown;        /* 1 if an Arnoldi cycle ended early on an invariant subspace */
    double res_est;       /* max_i |rho_i| * ||r|| / ||b~|| after the last cycle */
} orc_report;

/* Wilson kernel H_W(mu) = gamma5 D_W(mu) applied to one field. */
void orc_hw(const orc_lattice* lat, const orc_c* U, const orc_c* in, orc_c* out);

/* Same, restricted to the listed sites (out is written only there). */
void orc_hw_sites(const orc_lattice* lat, const orc_c* U, const orc_c* in, orc_c* out,
                  const int64_t* sites, int64_t nsites);

/* Kenney-Laub partial fractions, eq. (6.2), with the scaling c folded in. */
int orc_kenney_laub(int s, double c, double* sigma, double* omega);

/* Restarted FOM-LR(m,k), Algorithm 1, on A = H_W(mu) with the A^2 reading. */
int orc_fom_lr(const orc_lattice* lat, const orc_c* U,
               int s, const double* sigma, const double* omega,
               int k, double tol, int max_cycles, int project_each_cycle,
               int m, const orc_c* R, const orc_c* L, const orc_c* lambda,
               const orc_c* b, orc_c* x, orc_c* x_shift, orc_report* rep);

int orc_num_threads(void);
int orc_set_num_threads(int n);

#endif
