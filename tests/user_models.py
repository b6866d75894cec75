"""CUDA C++ sources of user-defined models (sdeb_create_user) used by the
tests: each restates a model the oracle knows, so the run-time compiled path
can be compared with the oracle, plus one with dense (non-diagonal) noise."""

# GBM, p = (mu, sigma): f_i = mu x_i, g_ii = sigma x_i.
GBM = r"""
__device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f) {
    for (int i = 0; i < SDEB_N; ++i) f[i] = p[0] * x[i];
}
__device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g) {
    for (int i = 0; i < SDEB_N * SDEB_M; ++i) g[i] = 0;
    for (int i = 0; i < SDEB_N; ++i) g[i * SDEB_M + i] = p[1] * x[i];
}
"""

# Kuramoto by its pairwise definition (Eq. 6), p = (K, sigma, omega_1..omega_n).
KURAMOTO_PAIRWISE = r"""
__device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f) {
    for (int i = 0; i < SDEB_N; ++i) {
        sdeb_real s = 0;
        for (int j = 0; j < SDEB_N; ++j) s += sin(x[j] - x[i]);
        f[i] = p[2 + i] + p[0] / SDEB_N * s;
    }
}
__device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g) {
    for (int i = 0; i < SDEB_N * SDEB_M; ++i) g[i] = 0;
    for (int i = 0; i < SDEB_N; ++i) g[i * SDEB_M + i] = p[1];
}
"""

# FitzHugh-Nagumo network, x = (v_1..v_u, w_1..w_u), p = (a, b, eps, I, c, sigma).
FHN = r"""
__device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f) {
    const int u = SDEB_N / 2;
    sdeb_real mean = 0;
    for (int i = 0; i < u; ++i) mean += x[i];
    mean /= u;
    for (int i = 0; i < u; ++i) {
        const sdeb_real v = x[i], w = x[u + i];
        f[i] = v - v * v * v / 3 - w + p[3] + p[4] * mean - p[4] * v;
        f[u + i] = p[2] * (v + p[0] - p[1] * w);
    }
}
__device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g) {
    for (int i = 0; i < SDEB_N * SDEB_M; ++i) g[i] = 0;
    for (int i = 0; i < SDEB_M; ++i) g[i * SDEB_M + i] = p[5] * x[i];
}
"""

# Linear SDE with dense noise: dX = A X dt + B dW, n = 2, m = 3,
# p = (a11, a12, a21, a22, b11, b12, b13, b21, b22, b23).
LINEAR_DENSE = r"""
__device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f) {
    f[0] = p[0] * x[0] + p[1] * x[1];
    f[1] = p[2] * x[0] + p[3] * x[1];
}
__device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g) {
    for (int i = 0; i < SDEB_N * SDEB_M; ++i) g[i] = p[4 + i];
}
"""

BROKEN = r"""
__device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f) {
    f[0] = undefined_symbol_here * x[0];
}
__device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g) {}
"""

# The same network with the diagonal-noise form: g[j] drives v_j.
FHN_DIAGONAL = r"""
#define SDEB_DIAGONAL_NOISE 1
__device__ void sdeb_drift(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *f) {
    const int u = SDEB_N / 2;
    sdeb_real mean = 0;
    for (int i = 0; i < u; ++i) mean += x[i];
    mean /= u;
    for (int i = 0; i < u; ++i) {
        const sdeb_real v = x[i], w = x[u + i];
        f[i] = v - v * v * v / 3 - w + p[3] + p[4] * mean - p[4] * v;
        f[u + i] = p[2] * (v + p[0] - p[1] * w);
    }
}
__device__ void sdeb_diffusion(double t, const sdeb_real *x, const sdeb_real *p, sdeb_real *g) {
    for (int j = 0; j < SDEB_M; ++j) g[j] = p[5] * x[j];
}
"""
