/*
 * Plain CPU oracle for many-orbit Euler-Maruyama integration of Ito SDEs.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * statement of what the GPU path must compute.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header, table or constant with the CUDA library, and it
 * never includes or links anything from it.
 *
 * Everything is FP64 and single-threaded per orbit.  Each function names the
 * passage of the SODECL paper (Avramidis, Lalik, Akman, arXiv 1908.03869) it
 * follows, or the published definition it restates.
 *
 * Parity status: every function here is pinned by a CPU test (Philox against
 * two independent library implementations, the integrator against closed
 * forms / invariants / brute force, the adjoint against finite differences
 * and an analytic OU gradient).  Nothing is "parity unpinned".
 */
#ifndef SDE_ORACLE_H
#define SDE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Model identifiers (the oracle's own numbering). */
enum {
    ORACLE_KURAMOTO = 1,       /* p = (K, sigma, omega_1..omega_n), d = n + 2, m = n   */
    ORACLE_KURAMOTO_PAPER = 2, /* p = (K, omega_1..omega_n, p_1..p_n), d = 2n + 1, m = n (Eq. 5) */
    ORACLE_FHN_NET = 3,        /* x = (v_1..v_u, w_1..w_u), n = 2u, m = u, p = (a, b, eps, I, c, sigma) */
    ORACLE_OU = 4,             /* dX = -theta X dt + sigma dW, m = n, p = (theta, sigma) */
    ORACLE_GBM = 5,            /* dX = mu X dt + sigma X dW, m = n, p = (mu, sigma) */
    ORACLE_LINEAR_ODE = 6      /* dx = -theta x dt (g = 0), m = 0, p = (theta) */
};

typedef struct {
    int32_t model;
    int32_t n, m, d;
    double t0, dt;
    int64_t steps, stride;   /* K steps; a frame every `stride` steps, frame 0 = initial state */
    uint64_t seed;           /* Philox key for the Wiener increments */
    int32_t shared_params;   /* 1: params is a single vector [d] used by every orbit */
    int32_t mean_field;      /* Kuramoto only: 1 = drift via (C, S) sums, 0 = pairwise definition */
    int32_t milstein;        /* 1: Milstein step instead of Euler-Maruyama (diagonal noise) */
    int32_t rk4;             /* 1: classical fourth-order Runge-Kutta on the drift alone (ODE path) */
    int32_t implicit;        /* ODE path, drift alone: 1 implicit Euler, 2 implicit midpoint */
} oracle_problem;

/* Newton iterations per implicit step (a fixed count, started from the old
 * state). */
#define ORACLE_NEWTON_ITERS 4

/* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel
 * random numbers: as easy as 1, 2, 3").  ctr[4] counter, key[2] key. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* The Wiener-increment draw of step k, noise block b, orbit o:
 * key = (seed lo32, seed hi32), counter = (k, b, o, stream). */
void oracle_philox_block(uint64_t seed, uint32_t k, uint32_t b, uint32_t orbit,
                         uint32_t stream, uint32_t out[4]);

/* Bulk forms for tests: out[k][b][o][4] over k in [k0, k0+nk), b in
 * [b0, b0+nb), o in [o0, o0+no); and normals out[k][o][m]. */
void oracle_philox_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t b0, int64_t nb,
                        uint32_t o0, int64_t no, uint32_t stream, uint32_t *out);
void oracle_normals_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t o0, int64_t no,
                         int32_t m, double *out);

/* u = (w + 1/2) * 2^-32, strictly inside (0, 1). */
double oracle_uniform(uint32_t w);

/* Eq. 3 on one pair of Philox words: out[0] = sqrt(-2 ln U1) cos(2 pi U2),
 * out[1] = sqrt(-2 ln U1) sin(2 pi U2), U1 from w_first, U2 from w_second. */
void oracle_box_muller(uint32_t w_first, uint32_t w_second, double out[2]);

/* The m standard normals N_0..N_{m-1} of step k, orbit o (Eq. 3, blocks of
 * four per Philox call; words past m are discarded). */
void oracle_normals(uint64_t seed, uint32_t k, uint32_t orbit, int32_t m, double *out);

/* Drift f(t, x, p) (length n) and dense diffusion g(t, x, p) (n x m, row
 * major) of Eq. 1.  Return 0, or -1 for an unknown model. */
int oracle_drift(const oracle_problem *pb, double t, const double *x, const double *p, double *f);
int oracle_diffusion(const oracle_problem *pb, double t, const double *x, const double *p, double *g);

/* Milstein scheme support (the paper names the Milstein method as the next
 * integration scheme to add, Sec. 2.1 and Sec. 3; the scheme is Kloeden and
 * Platen's, "Numerical Solution of Stochastic Differential Equations",
 * Sec. 10.3).  Every model here has diagonal noise whose channel j drives
 * state component j alone with g_jj a function of x_j only; dg[j] is
 * d g_jj / d x_j for j < m.  The Milstein step adds, to component j,
 *   1/2 g_jj dg_jj/dx_j (dW_j^2 - dt),   dW_j = sqrt(dt) N_j. */
int oracle_diffusion_diag_derivative(const oracle_problem *pb, double t, const double *x, const double *p,
                                     double *dg);

/* The drift's Jacobian J[i * n + j] = d f_i / d x_j, written out from each
 * model's drift (the implicit ODE schemes' Newton iterations use it). */
int oracle_drift_jacobian(const oracle_problem *pb, double t, const double *x, const double *p, double *J);

/* Check n, m, d against the model; 0 = consistent. */
int oracle_check_problem(const oracle_problem *pb);

/* Integrate orbits [orbit_begin, orbit_begin + count) from step k_begin to
 * k_end with Eq. 2.  x_in/x_out: [count][n] (may alias).  params: [count][d]
 * or [d] when shared_params.  frames (may be NULL): [F][count][n] with
 * F = steps/stride + 1; frame f holds the state at step f*stride and only the
 * frames inside [k_begin, k_end] are written.  nthreads > 1 splits the orbits
 * over POSIX threads (the per-orbit code is the same).  Returns 0 or -1. */
int oracle_integrate(const oracle_problem *pb, const double *params, const double *x_in,
                     int64_t orbit_begin, int64_t count, int64_t k_begin, int64_t k_end,
                     double *frames, double *x_out, int32_t nthreads);

/* Discrete adjoint of the whole horizon 0..steps: given dL/dX^K, return
 * dL/dp ([count][d], per orbit, even when params are shared) and dL/dX^0
 * ([count][n], may be NULL).  Dense Jacobians, all states stored. */
int oracle_adjoint(const oracle_problem *pb, const double *params, const double *x0,
                   int64_t orbit_begin, int64_t count, const double *dL_dxK,
                   double *dL_dp, double *dL_dx0);

/* Kuramoto order parameter (Eq. 7): r = |(1/n) sum_j exp(i theta_j)| and
 * dr/dtheta (length n, may be NULL; zero where r == 0). */
void oracle_order_param(int32_t n, const double *theta, double *r, double *dr_dtheta);

#ifdef __cplusplus
}
#endif

#endif
