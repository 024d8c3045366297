/*
 * Oracle: the Wilson kernel H_W(mu) = gamma5 D_W(mu).  TEST INFRASTRUCTURE ONLY.
 *
 * The paper takes H_W = gamma5 D_W as its kernel (Sec. 1) and defines D_W(mu)
 * only by citation.  The reading used here (stated in the design notes):
 *
 *   D_W(mu) psi(x) = (4 + m_W) psi(x)
 *       - 1/2 sum_nu [ (1 - gamma_nu) e^{+mu delta_{nu,t}} U_nu(x)           psi(x + nu)
 *                    + (1 + gamma_nu) e^{-mu delta_{nu,t}} U_nu(x - nu)^dag  psi(x - nu) ]
 *
 * with Euclidean Hermitian chiral-basis gamma matrices
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = x, y, z),
 *   gamma_t = [[0, 1], [1, 0]],  gamma5 = gamma_x gamma_y gamma_z gamma_t,
 * and a sign flip on hops that cross an antiperiodic boundary.
 *
 * Deliberately plain: the spin structure is a general 4x4 matrix product and
 * the colour structure a general 3x3 product, so the code can be read against
 * the formula above term by term.
 */
#include "oracle.h"

#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* gamma[nu][alpha][beta], filled once from the definition above. */
static orc_c GAMMA[4][4][4];
static orc_c GAMMA5[4][4];
static int gamma_ready = 0;

static void init_gamma(void) {
    if (gamma_ready) return;
    /* Pauli matrices */
    orc_c sig[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(GAMMA, 0, sizeof(GAMMA));
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                GAMMA[k][a][2 + b] = -I * sig[k][a][b];
                GAMMA[k][2 + a][b] = I * sig[k][a][b];
            }
    for (int a = 0; a < 2; ++a) {
        GAMMA[3][a][2 + a] = 1;
        GAMMA[3][2 + a][a] = 1;
    }
    /* gamma5 = gamma_x gamma_y gamma_z gamma_t */
    orc_c t1[4][4], t2[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            orc_c acc = 0;
            for (int l = 0; l < 4; ++l) acc += GAMMA[0][i][l] * GAMMA[1][l][j];
            t1[i][j] = acc;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            orc_c acc = 0;
            for (int l = 0; l < 4; ++l) acc += t1[i][l] * GAMMA[2][l][j];
            t2[i][j] = acc;
        }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            orc_c acc = 0;
            for (int l = 0; l < 4; ++l) acc += t2[i][l] * GAMMA[3][l][j];
            GAMMA5[i][j] = acc;
        }
    gamma_ready = 1;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the later parallel regions (n >= 1); returns the count now in force. */
int orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Neighbour of site (coordinates c) one step in direction nu, forward (+1) or
 * backward (-1); *phase becomes -1 when the hop wraps an antiperiodic edge. */
static int64_t hop(const orc_lattice* lat, const int c[4], int nu, int dir, double* phase) {
    int d[4] = {c[0], c[1], c[2], c[3]};
    int L = lat->dims[nu];
    d[nu] += dir;
    *phase = 1.0;
    if (d[nu] == L) {
        d[nu] = 0;
        if (lat->antiperiodic[nu]) *phase = -1.0;
    } else if (d[nu] < 0) {
        d[nu] = L - 1;
        if (lat->antiperiodic[nu]) *phase = -1.0;
    }
    return (int64_t)d[0] + (int64_t)lat->dims[0] *
           ((int64_t)d[1] + (int64_t)lat->dims[1] * ((int64_t)d[2] + (int64_t)lat->dims[2] * d[3]));
}

static void site_hw(const orc_lattice* lat, const orc_c* U, const orc_c* in, orc_c* out, int64_t x) {
    int c[4];
    int64_t rem = x;
    for (int nu = 0; nu < 4; ++nu) {
        c[nu] = (int)(rem % lat->dims[nu]);
        rem /= lat->dims[nu];
    }
    orc_c d[4][3];
    for (int a = 0; a < 4; ++a)
        for (int col = 0; col < 3; ++col) d[a][col] = (4.0 + lat->mass) * in[(x * 4 + a) * 3 + col];

    for (int nu = 0; nu < 4; ++nu) {
        for (int dir = +1; dir >= -1; dir -= 2) {
            double phase;
            int64_t y = hop(lat, c, nu, dir, &phase);
            double emu = (nu == 3) ? exp(dir * lat->mu) : 1.0;
            /* colour part: forward U_nu(x) psi(x+nu); backward U_nu(x-nu)^dag psi(x-nu) */
            orc_c up[4][3];
            for (int a = 0; a < 4; ++a)
                for (int i = 0; i < 3; ++i) {
                    orc_c acc = 0;
                    for (int j = 0; j < 3; ++j) {
                        orc_c u = (dir > 0) ? U[((x * 4 + nu) * 3 + i) * 3 + j]
                                            : conj(U[((y * 4 + nu) * 3 + j) * 3 + i]);
                        acc += u * in[(y * 4 + a) * 3 + j];
                    }
                    up[a][i] = acc;
                }
            /* spin part: (1 - gamma) forward, (1 + gamma) backward */
            double sgn = (dir > 0) ? -1.0 : 1.0;
            for (int a = 0; a < 4; ++a)
                for (int i = 0; i < 3; ++i) {
                    orc_c acc = 0;
                    for (int b = 0; b < 4; ++b) {
                        orc_c p = ((a == b) ? 1.0 : 0.0) + sgn * GAMMA[nu][a][b];
                        acc += p * up[b][i];
                    }
                    d[a][i] -= 0.5 * emu * phase * acc;
                }
        }
    }
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) {
            orc_c acc = 0;
            for (int b = 0; b < 4; ++b) acc += GAMMA5[a][b] * d[b][i];
            out[(x * 4 + a) * 3 + i] = acc;
        }
}

void orc_hw(const orc_lattice* lat, const orc_c* U, const orc_c* in, orc_c* out) {
    init_gamma();
    int64_t vol = (int64_t)lat->dims[0] * lat->dims[1] * lat->dims[2] * lat->dims[3];
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < vol; ++x) site_hw(lat, U, in, out, x);
}

void orc_hw_sites(const orc_lattice* lat, const orc_c* U, const orc_c* in, orc_c* out,
                  const int64_t* sites, int64_t nsites) {
    init_gamma();
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nsites; ++i) site_hw(lat, U, in, out, sites[i]);
}
