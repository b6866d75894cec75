/*
 * Plain CPU oracle for many-orbit Euler-Maruyama integration (FP64).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg, never by the product path.  It shares
 * no code with the CUDA library.
 *
 * Section / equation references are to the SODECL paper (arXiv 1908.03869):
 *   Eq. 1  Ito SDE system dX_i = f_i dt + sum_j g_ij dW_j          (Sec. 1.1)
 *   Eq. 2  Euler-Maruyama recursion                                (Sec. 2.1.1)
 *   Eq. 3  Box-Muller transform of two uniforms                    (Sec. 2.1.2)
 *   Eq. 5  stochastic Kuramoto model, footnote: n = m = N,
 *          f_i = omega_i + K/N sum_j sin(theta_j - theta_i), g_ij = p_i delta_ij
 *   Eq. 7  complex order parameter                                 (Sec. 2.3.1)
 * Readings of passages the paper leaves open are listed where they are used.
 */
#define _POSIX_C_SOURCE 200809L
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon et al. (SC'11):              */
/* each round multiplies counter words 0 and 2 by two fixed odd constants,   */
/* keeps the 64-bit products' halves, and mixes the high halves with the     */
/* other two counter words and the round key; the key is bumped by two Weyl  */
/* constants (golden ratio and sqrt(3)-1, as 32-bit fractions) between        */
/* rounds.                                                                    */
/* ------------------------------------------------------------------------ */

static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += PHILOX_W0;
            k[1] += PHILOX_W1;
        }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Reading of Sec. 2.1.2 ("Random123", no generator or layout named): the
 * generator is Philox4x32-10, keyed by the seed, with the counter holding the
 * step, the noise block (4 normals per call), the global orbit index and a
 * stream id (0 = Wiener increments).  Nothing is stored between steps. */
void oracle_philox_block(uint64_t seed, uint32_t k, uint32_t b, uint32_t orbit,
                         uint32_t stream, uint32_t out[4])
{
    uint32_t ctr[4] = {k, b, orbit, stream};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

void oracle_philox_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t b0, int64_t nb,
                        uint32_t o0, int64_t no, uint32_t stream, uint32_t *out)
{
    for (int64_t k = 0; k < nk; ++k)
        for (int64_t b = 0; b < nb; ++b)
            for (int64_t o = 0; o < no; ++o)
                oracle_philox_block(seed, (uint32_t)(k0 + k), (uint32_t)(b0 + b),
                                    (uint32_t)(o0 + o), stream,
                                    out + ((k * nb + b) * no + o) * 4);
}

/* Reading of Eq. 3's "uniform over [0,1]": u = (w + 1/2) 2^-32, so ln u is
 * always finite and u is never 1. */
double oracle_uniform(uint32_t w)
{
    return ((double)w + 0.5) * ldexp(1.0, -32);
}

/* Eq. 3 for one pair of words: the first word sets the radius
 * sqrt(-2 ln U1), the second the angle 2 pi U2; out[0] takes the cos branch
 * and out[1] the sin branch. */
void oracle_box_muller(uint32_t w_first, uint32_t w_second, double out[2])
{
    const double two_pi = 2.0 * acos(-1.0);   /* 2 pi, rounded to double */
    double u1 = oracle_uniform(w_first);
    double u2 = oracle_uniform(w_second);
    double radius = sqrt(-2.0 * log(u1));
    out[0] = radius * cos(two_pi * u2);
    out[1] = radius * sin(two_pi * u2);
}

/* Eq. 3 applied block by block ("called multiple times" for more than two
 * noise terms): words (w0, w1) give N_{4b}, N_{4b+1}, words (w2, w3) give
 * N_{4b+2}, N_{4b+3}; words past m are discarded. */
void oracle_normals(uint64_t seed, uint32_t k, uint32_t orbit, int32_t m, double *out)
{
    for (int32_t b = 0; 4 * b < m; ++b) {
        uint32_t w[4];
        double z[4];
        oracle_philox_block(seed, k, (uint32_t)b, orbit, 0u, w);
        oracle_box_muller(w[0], w[1], z);
        oracle_box_muller(w[2], w[3], z + 2);
        for (int q = 0; q < 4 && 4 * b + q < m; ++q)
            out[4 * b + q] = z[q];
    }
}

void oracle_normals_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t o0, int64_t no,
                         int32_t m, double *out)
{
    for (int64_t k = 0; k < nk; ++k)
        for (int64_t o = 0; o < no; ++o)
            oracle_normals(seed, (uint32_t)(k0 + k), (uint32_t)(o0 + o), m,
                           out + (k * no + o) * m);
}

/* ------------------------------------------------------------------------ */
/* Models: drift f and dense diffusion g of Eq. 1.                           */
/* ------------------------------------------------------------------------ */

int oracle_check_problem(const oracle_problem *pb)
{
    int n = pb->n, m = pb->m, d = pb->d;
    if (n <= 0 || m < 0 || d <= 0) return -1;
    if (pb->milstein != 0 && pb->milstein != 1) return -1;
    if (pb->rk4 != 0 && pb->rk4 != 1) return -1;
    if (pb->milstein && pb->rk4) return -1;
    if (pb->implicit < 0 || pb->implicit > 2) return -1;
    if (pb->implicit && (pb->milstein || pb->rk4)) return -1;
    switch (pb->model) {
    case ORACLE_KURAMOTO:       return (m == n && d == n + 2) ? 0 : -1;
    case ORACLE_KURAMOTO_PAPER: return (m == n && d == 2 * n + 1) ? 0 : -1;
    case ORACLE_FHN_NET:        return (n % 2 == 0 && m == n / 2 && d == 6) ? 0 : -1;
    case ORACLE_OU:             return (m == n && d == 2) ? 0 : -1;
    case ORACLE_GBM:            return (m == n && d == 2) ? 0 : -1;
    case ORACLE_LINEAR_ODE:     return (m == 0 && d == 1) ? 0 : -1;
    default:                    return -1;
    }
}

/* Kuramoto drift of Eq. 5/6.  Pairwise: the sum over j as written, with the
 * j = i term included (it is sin 0).  Mean field: the same sum rewritten as
 * S cos(theta_i) - C sin(theta_i) with C = sum cos theta_j, S = sum sin theta_j
 * (sin(a - b) = sin a cos b - cos a sin b). */
static void kuramoto_drift(int n, double K, const double *omega, const double *th,
                           int mean_field, double *f)
{
    if (mean_field) {
        double C = 0.0, S = 0.0;
        for (int j = 0; j < n; ++j) {
            C += cos(th[j]);
            S += sin(th[j]);
        }
        for (int i = 0; i < n; ++i)
            f[i] = omega[i] + (K / n) * (S * cos(th[i]) - C * sin(th[i]));
    } else {
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j)
                acc += sin(th[j] - th[i]);
            f[i] = omega[i] + (K / n) * acc;
        }
    }
}

int oracle_drift(const oracle_problem *pb, double t, const double *x, const double *p, double *f)
{
    (void)t; /* every model here is autonomous */
    int n = pb->n;
    switch (pb->model) {
    case ORACLE_KURAMOTO:
        kuramoto_drift(n, p[0], p + 2, x, pb->mean_field, f);
        return 0;
    case ORACLE_KURAMOTO_PAPER:
        kuramoto_drift(n, p[0], p + 1, x, pb->mean_field, f);
        return 0;
    case ORACLE_FHN_NET: {
        /* dv_i = (v_i - v_i^3/3 - w_i + I + c mean(v) - c v_i) dt + sigma v_i dW_i
         * dw_i = eps (v_i + a - b w_i) dt; mean(v) includes unit i. */
        int u = n / 2;
        double a = p[0], b = p[1], eps = p[2], I = p[3], c = p[4];
        const double *v = x, *w = x + u;
        double mean_v = 0.0;
        for (int j = 0; j < u; ++j) mean_v += v[j];
        mean_v /= u;
        for (int i = 0; i < u; ++i) {
            f[i] = v[i] - v[i] * v[i] * v[i] / 3.0 - w[i] + I + c * mean_v - c * v[i];
            f[u + i] = eps * (v[i] + a - b * w[i]);
        }
        return 0;
    }
    case ORACLE_OU:
    case ORACLE_LINEAR_ODE:
        for (int i = 0; i < n; ++i) f[i] = -p[0] * x[i];
        return 0;
    case ORACLE_GBM:
        for (int i = 0; i < n; ++i) f[i] = p[0] * x[i];
        return 0;
    default:
        return -1;
    }
}

int oracle_diffusion(const oracle_problem *pb, double t, const double *x, const double *p, double *g)
{
    (void)t;
    int n = pb->n, m = pb->m;
    for (int i = 0; i < n * m; ++i) g[i] = 0.0;
    switch (pb->model) {
    case ORACLE_KURAMOTO:        /* g_ij = sigma delta_ij (scalar-sigma variant) */
        for (int i = 0; i < n; ++i) g[i * m + i] = p[1];
        return 0;
    case ORACLE_KURAMOTO_PAPER:  /* g_ij = p_i delta_ij, Eq. 5 footnote */
        for (int i = 0; i < n; ++i) g[i * m + i] = p[1 + n + i];
        return 0;
    case ORACLE_FHN_NET: {       /* multiplicative noise on v only */
        int u = n / 2;
        for (int i = 0; i < u; ++i) g[i * m + i] = p[5] * x[i];
        return 0;
    }
    case ORACLE_OU:
        for (int i = 0; i < n; ++i) g[i * m + i] = p[1];
        return 0;
    case ORACLE_GBM:
        for (int i = 0; i < n; ++i) g[i * m + i] = p[1] * x[i];
        return 0;
    case ORACLE_LINEAR_ODE:
        return 0;
    default:
        return -1;
    }
}

/* d g_jj / d x_j of each model's diagonal noise (see oracle.h), written out
 * from the diffusion above. */
int oracle_diffusion_diag_derivative(const oracle_problem *pb, double t, const double *x, const double *p,
                                     double *dg)
{
    (void)t;
    (void)x;
    int m = pb->m;
    for (int j = 0; j < m; ++j) dg[j] = 0.0;
    switch (pb->model) {
    case ORACLE_KURAMOTO:        /* additive: g_jj = sigma */
    case ORACLE_KURAMOTO_PAPER:  /* additive: g_jj = p_j */
    case ORACLE_OU:              /* additive */
    case ORACLE_LINEAR_ODE:      /* no noise */
        return 0;
    case ORACLE_FHN_NET:         /* g_jj = sigma v_j, channel j drives v_j = x_j */
    case ORACLE_GBM:             /* g_jj = sigma x_j */
        for (int j = 0; j < m; ++j) dg[j] = pb->model == ORACLE_GBM ? p[1] : p[5];
        return 0;
    default:
        return -1;
    }
}

/* Jacobian of the drift, from the drifts above (Kuramoto by the pairwise
 * definition: d/dx_l of sum_j sin(x_j - x_i)). */
int oracle_drift_jacobian(const oracle_problem *pb, double t, const double *x, const double *p, double *J)
{
    (void)t;
    int n = pb->n;
    for (int i = 0; i < n * n; ++i) J[i] = 0.0;
    switch (pb->model) {
    case ORACLE_KURAMOTO:
    case ORACLE_KURAMOTO_PAPER: {
        double kn = p[0] / n;
        for (int i = 0; i < n; ++i) {
            double diag = 0.0;
            for (int l = 0; l < n; ++l) {
                if (l == i) continue;
                double cl = cos(x[l] - x[i]);
                J[i * n + l] = kn * cl;
                diag -= kn * cl;
            }
            J[i * n + i] = diag;
        }
        return 0;
    }
    case ORACLE_FHN_NET: {
        int u = n / 2;
        double b = p[1], eps = p[2], c = p[4];
        for (int i = 0; i < u; ++i) {
            for (int j = 0; j < u; ++j) J[i * n + j] = c / u;          /* c mean(v) */
            J[i * n + i] += 1.0 - x[i] * x[i] - c;                     /* v - v^3/3 - c v */
            J[i * n + u + i] = -1.0;                                    /* - w */
            J[(u + i) * n + i] = eps;                                   /* eps v */
            J[(u + i) * n + u + i] = -eps * b;                          /* - eps b w */
        }
        return 0;
    }
    case ORACLE_OU:
    case ORACLE_LINEAR_ODE:
        for (int i = 0; i < n; ++i) J[i * n + i] = -p[0];
        return 0;
    case ORACLE_GBM:
        for (int i = 0; i < n; ++i) J[i * n + i] = p[0];
        return 0;
    default:
        return -1;
    }
}

/* Solves A z = r in place (z overwrites r) by Gaussian elimination with
 * partial pivoting; A (n x n, row-major) is overwritten. */
static void dense_solve(int n, double *A, double *r)
{
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(A[i * n + col]) > fabs(A[piv * n + col])) piv = i;
        if (piv != col) {
            for (int j = 0; j < n; ++j) {
                double tmp = A[col * n + j];
                A[col * n + j] = A[piv * n + j];
                A[piv * n + j] = tmp;
            }
            double tmp = r[col];
            r[col] = r[piv];
            r[piv] = tmp;
        }
        for (int i = col + 1; i < n; ++i) {
            double m = A[i * n + col] / A[col * n + col];
            for (int j = col; j < n; ++j) A[i * n + j] -= m * A[col * n + j];
            r[i] -= m * r[col];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double acc = r[i];
        for (int j = i + 1; j < n; ++j) acc -= A[i * n + j] * r[j];
        r[i] = acc / A[i * n + i];
    }
}

/* ------------------------------------------------------------------------ */
/* Euler-Maruyama, Eq. 2, and the Milstein step.                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    double *f, *g, *N, *xn, *dg, *k[4], *y, *J;
} em_scratch;

static int scratch_alloc(em_scratch *s, int n, int m)
{
    s->f = (double *)malloc(sizeof(double) * (size_t)n);
    s->g = (double *)malloc(sizeof(double) * (size_t)(n * (m > 0 ? m : 1)));
    s->N = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    s->xn = (double *)malloc(sizeof(double) * (size_t)n);
    s->dg = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    s->y = (double *)malloc(sizeof(double) * (size_t)n);
    s->J = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    int ok = s->f && s->g && s->N && s->xn && s->dg && s->y && s->J;
    for (int q = 0; q < 4; ++q) {
        s->k[q] = (double *)malloc(sizeof(double) * (size_t)n);
        ok = ok && s->k[q];
    }
    return ok ? 0 : -1;
}

static void scratch_free(em_scratch *s)
{
    free(s->f); free(s->g); free(s->N); free(s->xn); free(s->dg); free(s->y); free(s->J);
    for (int q = 0; q < 4; ++q) free(s->k[q]);
}

/* One step of the classical fourth-order Runge-Kutta method on the drift
 * alone, dx/dt = f(t, x) (the ODE path; the paper lists Runge-Kutta among
 * the ODE integrators, Sec. 1.5):
 *   k1 = f(t, x), k2 = f(t + h/2, x + h k1/2), k3 = f(t + h/2, x + h k2/2),
 *   k4 = f(t + h, x + h k3), x <- x + h (k1 + 2 k2 + 2 k3 + k4) / 6. */
static void rk4_step(const oracle_problem *pb, const double *p, int64_t k, double *x, em_scratch *s)
{
    int n = pb->n;
    double h = pb->dt, t = pb->t0 + (double)k * h;
    oracle_drift(pb, t, x, p, s->k[0]);
    for (int i = 0; i < n; ++i) s->y[i] = x[i] + 0.5 * h * s->k[0][i];
    oracle_drift(pb, t + 0.5 * h, s->y, p, s->k[1]);
    for (int i = 0; i < n; ++i) s->y[i] = x[i] + 0.5 * h * s->k[1][i];
    oracle_drift(pb, t + 0.5 * h, s->y, p, s->k[2]);
    for (int i = 0; i < n; ++i) s->y[i] = x[i] + h * s->k[2][i];
    oracle_drift(pb, t + h, s->y, p, s->k[3]);
    for (int i = 0; i < n; ++i)
        x[i] += h * (s->k[0][i] + 2.0 * s->k[1][i] + 2.0 * s->k[2][i] + s->k[3][i]) / 6.0;
}

/* One step of an implicit ODE scheme on the drift alone (the paper lists
 * implicit Euler and implicit midpoint among its ODE integrators, Sec. 1.5):
 *   implicit Euler:    y = x + h f(t + h, y),
 *   implicit midpoint: y = x + h f(t + h/2, (x + y) / 2),
 * solved by ORACLE_NEWTON_ITERS Newton iterations from y = x on
 * G(y) = y - x - h f(t + theta h, x + theta (y - x)) (theta = 1 or 1/2),
 * G'(y) = I - theta h J(x + theta (y - x)), with a dense solve. */
static void implicit_step(const oracle_problem *pb, const double *p, int64_t k, double *x, em_scratch *s)
{
    int n = pb->n;
    double h = pb->dt, theta = pb->implicit == 1 ? 1.0 : 0.5;
    double t = pb->t0 + ((double)k + theta) * h;
    double *y = s->xn, *z = s->y, *r = s->k[0];
    memcpy(y, x, sizeof(double) * (size_t)n);
    for (int it = 0; it < ORACLE_NEWTON_ITERS; ++it) {
        for (int i = 0; i < n; ++i) z[i] = x[i] + theta * (y[i] - x[i]);
        oracle_drift(pb, t, z, p, s->f);
        oracle_drift_jacobian(pb, t, z, p, s->J);
        for (int i = 0; i < n; ++i) {
            r[i] = -(y[i] - x[i] - h * s->f[i]);
            for (int j = 0; j < n; ++j) s->J[i * n + j] = (i == j ? 1.0 : 0.0) - theta * h * s->J[i * n + j];
        }
        dense_solve(n, s->J, r);
        for (int i = 0; i < n; ++i) y[i] += r[i];
    }
    memcpy(x, y, sizeof(double) * (size_t)n);
}

/* One step of Eq. 2 at step index k (reading of Eq. 2's t: the drift and
 * diffusion of step k are evaluated at t_k = t0 + k dt and at the old state,
 * the update of all components is simultaneous). */
static void em_step(const oracle_problem *pb, const double *p, int64_t k, uint32_t orbit,
                    double *x, em_scratch *s)
{
    if (pb->rk4) {
        rk4_step(pb, p, k, x, s);
        return;
    }
    if (pb->implicit) {
        implicit_step(pb, p, k, x, s);
        return;
    }
    int n = pb->n, m = pb->m;
    double t = pb->t0 + (double)k * pb->dt;
    double sqdt = sqrt(pb->dt);
    oracle_drift(pb, t, x, p, s->f);
    if (m > 0) {
        oracle_diffusion(pb, t, x, p, s->g);
        oracle_normals(pb->seed, (uint32_t)k, orbit, m, s->N);
    }
    for (int i = 0; i < n; ++i) {
        double noise = 0.0;
        for (int j = 0; j < m; ++j) noise += s->g[i * m + j] * sqdt * s->N[j];
        s->xn[i] = x[i] + s->f[i] * pb->dt + noise;
    }
    if (pb->milstein && m > 0) {
        /* channel j drives component j: + 1/2 g_jj g_jj' (dW_j^2 - dt) */
        oracle_diffusion_diag_derivative(pb, t, x, p, s->dg);
        for (int j = 0; j < m; ++j) {
            double dW = sqdt * s->N[j];
            s->xn[j] += 0.5 * s->g[j * m + j] * s->dg[j] * (dW * dW - pb->dt);
        }
    }
    memcpy(x, s->xn, sizeof(double) * (size_t)n);
}

typedef struct {
    const oracle_problem *pb;
    const double *params, *x_in;
    int64_t orbit_begin, lo, hi, count, k_begin, k_end;
    double *frames, *x_out;
    int status;
} integrate_job;

static void *integrate_worker(void *arg)
{
    integrate_job *job = (integrate_job *)arg;
    const oracle_problem *pb = job->pb;
    int n = pb->n;
    int64_t nframes = pb->steps / pb->stride + 1;
    em_scratch s;
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    if (!x || scratch_alloc(&s, n, pb->m) != 0) {
        job->status = -1;
        free(x);
        return NULL;
    }
    for (int64_t o = job->lo; o < job->hi; ++o) {
        const double *p = pb->shared_params ? job->params : job->params + o * pb->d;
        uint32_t orbit = (uint32_t)(job->orbit_begin + o);
        memcpy(x, job->x_in + o * n, sizeof(double) * (size_t)n);
        if (job->frames && job->k_begin == 0)
            memcpy(job->frames + (0 * job->count + o) * n, x, sizeof(double) * (size_t)n);
        for (int64_t k = job->k_begin; k < job->k_end; ++k) {
            em_step(pb, p, k, orbit, x, &s);
            if (job->frames && (k + 1) % pb->stride == 0) {
                int64_t fidx = (k + 1) / pb->stride;
                if (fidx < nframes)
                    memcpy(job->frames + (fidx * job->count + o) * n, x, sizeof(double) * (size_t)n);
            }
        }
        memcpy(job->x_out + o * n, x, sizeof(double) * (size_t)n);
    }
    scratch_free(&s);
    free(x);
    job->status = 0;
    return NULL;
}

int oracle_integrate(const oracle_problem *pb, const double *params, const double *x_in,
                     int64_t orbit_begin, int64_t count, int64_t k_begin, int64_t k_end,
                     double *frames, double *x_out, int32_t nthreads)
{
    if (oracle_check_problem(pb) != 0 || pb->stride < 1 || count < 0 || k_begin < 0 ||
        k_end < k_begin || k_end > pb->steps || pb->steps > 0xffffffffLL ||
        orbit_begin < 0 || orbit_begin + count > 0x100000000LL)
        return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > count) nthreads = count > 0 ? (int32_t)count : 1;
    /* x_in and x_out may alias: work from a private copy of the inputs. */
    double *xin_copy = (double *)malloc(sizeof(double) * (size_t)(count * pb->n + 1));
    if (!xin_copy) return -1;
    memcpy(xin_copy, x_in, sizeof(double) * (size_t)(count * pb->n));
    integrate_job *jobs = (integrate_job *)calloc((size_t)nthreads, sizeof(integrate_job));
    pthread_t *tids = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int *created = (int *)calloc((size_t)nthreads, sizeof(int));
    if (!jobs || !tids || !created) {
        free(xin_copy); free(jobs); free(tids); free(created);
        return -1;
    }
    int status = 0;
    for (int t = 0; t < nthreads; ++t) {
        integrate_job *j = &jobs[t];
        j->pb = pb; j->params = params; j->x_in = xin_copy;
        j->orbit_begin = orbit_begin; j->count = count;
        j->lo = count * t / nthreads; j->hi = count * (t + 1) / nthreads;
        j->k_begin = k_begin; j->k_end = k_end;
        j->frames = frames; j->x_out = x_out; j->status = -1;
        if (nthreads > 1 && pthread_create(&tids[t], NULL, integrate_worker, j) == 0)
            created[t] = 1;
        else
            integrate_worker(j);   /* single thread, or thread creation failed */
    }
    for (int t = 0; t < nthreads; ++t) {
        if (created[t]) pthread_join(tids[t], NULL);
        if (jobs[t].status < 0) status = -1;
    }
    free(created);
    free(jobs); free(tids); free(xin_copy);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of Eq. 2 (not in the paper; it serves the parameter       */
/* optimisation use of Sec. 1.2).  For X^{k+1} = X^k + dt f(X^k) +            */
/* sqrt(dt) G(X^k) N^k the gradient of L(X^K) is                              */
/*   lambda^K = dL/dX^K,                                                      */
/*   lambda^k = lambda^{k+1} + (dt df/dx + sqrt(dt) d(GN)/dx)^T lambda^{k+1}, */
/*   dL/dp   += (dt df/dp + sqrt(dt) d(GN)/dp)^T lambda^{k+1},                */
/* with every derivative written out by hand from the model formulas.         */
/* ------------------------------------------------------------------------ */

/* Fills jx (n x n): d(f_i)/d(x_l) and jp (n x d): d(f_i)/d(p_q), and the
 * noise parts gx (n x n): d(sum_j g_ij N_j)/d(x_l), gp (n x d). */
static int model_jacobians(const oracle_problem *pb, const double *x, const double *p,
                           const double *N, double *jx, double *jp, double *gx, double *gp)
{
    int n = pb->n, d = pb->d;
    memset(jx, 0, sizeof(double) * (size_t)(n * n));
    memset(gx, 0, sizeof(double) * (size_t)(n * n));
    memset(jp, 0, sizeof(double) * (size_t)(n * d));
    memset(gp, 0, sizeof(double) * (size_t)(n * d));
    switch (pb->model) {
    case ORACLE_KURAMOTO:
    case ORACLE_KURAMOTO_PAPER: {
        int paper = pb->model == ORACLE_KURAMOTO_PAPER;
        double K = p[0];
        for (int i = 0; i < n; ++i) {
            double sum_sin = 0.0;
            for (int j = 0; j < n; ++j) {
                /* d/dtheta_j and d/dtheta_i of (K/n) sin(theta_j - theta_i) */
                double c = (K / n) * cos(x[j] - x[i]);
                jx[i * n + j] += c;
                jx[i * n + i] -= c;
                sum_sin += sin(x[j] - x[i]);
            }
            jp[i * d + 0] = sum_sin / n;                   /* d f_i / dK */
            jp[i * d + (paper ? 1 + i : 2 + i)] = 1.0;     /* d f_i / d omega_i */
            if (paper)
                gp[i * d + 1 + n + i] = N[i];              /* d(p_i N_i)/d p_i */
            else
                gp[i * d + 1] = N[i];                      /* d(sigma N_i)/d sigma */
        }
        return 0;
    }
    case ORACLE_FHN_NET: {
        int u = n / 2;
        double a = p[0], b = p[1], eps = p[2], c = p[4], sigma = p[5];
        const double *v = x, *w = x + u;
        double mean_v = 0.0;
        for (int j = 0; j < u; ++j) mean_v += v[j];
        mean_v /= u;
        for (int i = 0; i < u; ++i) {
            int vi = i, wi = u + i;
            for (int l = 0; l < u; ++l) jx[vi * n + l] += c / u;    /* c mean(v) */
            jx[vi * n + vi] += 1.0 - v[i] * v[i] - c;
            jx[vi * n + wi] += -1.0;
            jx[wi * n + vi] += eps;
            jx[wi * n + wi] += -eps * b;
            jp[vi * d + 3] = 1.0;                           /* I */
            jp[vi * d + 4] = mean_v - v[i];                 /* c */
            jp[wi * d + 0] = eps;                           /* a */
            jp[wi * d + 1] = -eps * w[i];                   /* b */
            jp[wi * d + 2] = v[i] + a - b * w[i];           /* eps */
            gx[vi * n + vi] = sigma * N[i];                 /* d(sigma v_i N_i)/d v_i */
            gp[vi * d + 5] = v[i] * N[i];                   /* d(sigma v_i N_i)/d sigma */
        }
        return 0;
    }
    case ORACLE_OU:
        for (int i = 0; i < n; ++i) {
            jx[i * n + i] = -p[0];
            jp[i * d + 0] = -x[i];
            gp[i * d + 1] = N[i];
        }
        return 0;
    case ORACLE_GBM:
        for (int i = 0; i < n; ++i) {
            jx[i * n + i] = p[0];
            jp[i * d + 0] = x[i];
            gx[i * n + i] = p[1] * N[i];
            gp[i * d + 1] = x[i] * N[i];
        }
        return 0;
    case ORACLE_LINEAR_ODE:
        for (int i = 0; i < n; ++i) {
            jx[i * n + i] = -p[0];
            jp[i * d + 0] = -x[i];
        }
        return 0;
    default:
        return -1;
    }
}

int oracle_adjoint(const oracle_problem *pb, const double *params, const double *x0,
                   int64_t orbit_begin, int64_t count, const double *dL_dxK,
                   double *dL_dp, double *dL_dx0)
{
    /* the adjoint of the Euler-Maruyama recursion only */
    if (oracle_check_problem(pb) != 0 || count < 0 || pb->steps > 0xffffffffLL || pb->rk4 || pb->milstein ||
        pb->implicit)
        return -1;
    int n = pb->n, m = pb->m, d = pb->d;
    int64_t K = pb->steps;
    double sqdt = sqrt(pb->dt);
    double *traj = (double *)malloc(sizeof(double) * (size_t)((K + 1) * n));
    double *jx = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *gx = (double *)malloc(sizeof(double) * (size_t)(n * n));
    double *jp = (double *)malloc(sizeof(double) * (size_t)(n * d));
    double *gp = (double *)malloc(sizeof(double) * (size_t)(n * d));
    double *N = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double *lam = (double *)malloc(sizeof(double) * (size_t)n);
    double *lam_new = (double *)malloc(sizeof(double) * (size_t)n);
    em_scratch s;
    int ok = traj && jx && gx && jp && gp && N && lam && lam_new && scratch_alloc(&s, n, m) == 0;
    if (!ok) {
        free(traj); free(jx); free(gx); free(jp); free(gp); free(N); free(lam); free(lam_new);
        return -1;
    }
    for (int64_t o = 0; o < count; ++o) {
        const double *p = pb->shared_params ? params : params + o * d;
        uint32_t orbit = (uint32_t)(orbit_begin + o);
        /* forward, keeping every state */
        memcpy(traj, x0 + o * n, sizeof(double) * (size_t)n);
        for (int64_t k = 0; k < K; ++k) {
            memcpy(traj + (k + 1) * n, traj + k * n, sizeof(double) * (size_t)n);
            em_step(pb, p, k, orbit, traj + (k + 1) * n, &s);
        }
        /* reverse sweep */
        memcpy(lam, dL_dxK + o * n, sizeof(double) * (size_t)n);
        double *gpo = dL_dp + o * d;
        for (int q = 0; q < d; ++q) gpo[q] = 0.0;
        for (int64_t k = K - 1; k >= 0; --k) {
            const double *xk = traj + k * n;
            if (m > 0) oracle_normals(pb->seed, (uint32_t)k, orbit, m, N);
            model_jacobians(pb, xk, p, N, jx, jp, gx, gp);
            for (int q = 0; q < d; ++q) {
                double acc = 0.0;
                for (int i = 0; i < n; ++i)
                    acc += (pb->dt * jp[i * d + q] + sqdt * gp[i * d + q]) * lam[i];
                gpo[q] += acc;
            }
            for (int l = 0; l < n; ++l) {
                double acc = lam[l];
                for (int i = 0; i < n; ++i)
                    acc += (pb->dt * jx[i * n + l] + sqdt * gx[i * n + l]) * lam[i];
                lam_new[l] = acc;
            }
            memcpy(lam, lam_new, sizeof(double) * (size_t)n);
        }
        if (dL_dx0) memcpy(dL_dx0 + o * n, lam, sizeof(double) * (size_t)n);
    }
    scratch_free(&s);
    free(traj); free(jx); free(gx); free(jp); free(gp); free(N); free(lam); free(lam_new);
    return 0;
}

/* Eq. 7: r e^{i Phi} = (1/n) sum_j e^{i theta_j}.  With Cm, Sm the means of
 * cos and sin, r = sqrt(Cm^2 + Sm^2) and dr/dtheta_l = (Sm cos theta_l -
 * Cm sin theta_l) / (n r). */
void oracle_order_param(int32_t n, const double *theta, double *r, double *dr_dtheta)
{
    double Cm = 0.0, Sm = 0.0;
    for (int j = 0; j < n; ++j) {
        Cm += cos(theta[j]);
        Sm += sin(theta[j]);
    }
    Cm /= n;
    Sm /= n;
    double rr = sqrt(Cm * Cm + Sm * Sm);
    *r = rr;
    if (dr_dtheta) {
        for (int l = 0; l < n; ++l)
            dr_dtheta[l] = rr > 0.0 ? (Sm * cos(theta[l]) - Cm * sin(theta[l])) / (n * rr) : 0.0;
    }
}
