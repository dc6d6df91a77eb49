/*
 * FP64 CPU oracle: classical RK4 of the frozen Gaussian ODE system.
 * TEST INFRASTRUCTURE ONLY: called by the tests and the CPU baseline of the
 * benchmark through oracle/trajectories.py; the CUDA library never links it.
 *
 * Eq. 2.3-2.7 of the paper, with the Jacobian blocks written out:
 *   Q' = P,  P' = -grad V(Q),  S' = |P|^2/2 - V(Q),
 *   F = dQ/dq, G = dQ/dp, H = dP/dq, K = dP/dp   (d x d real matrices)
 *   F' = H,  G' = K,  H' = -Hess V(Q) F,  K' = -Hess V(Q) G,
 *   Z = dz(Q + iP) with dz = d/dq - i d/dp  =>  Z = F - iG + iH + K,
 *   Z' = H - iK - i HessV F - HessV G,
 *   A' = (A/2) tr(Z^{-1} Z'),
 * initial data F = K = I, G = H = 0 (so Z(0) = 2I), S(0) = 0.
 *
 * The amplitude is integrated as a complex number (no logarithm, hence no
 * branch choice).  tr(Z^{-1} Z') is computed by solving Z X = Z' with complex
 * Gaussian elimination (partial pivoting) and summing diag(X).
 *
 * Time stepping: nsteps = round(t/dt) when t/dt is within 1e-9 of an integer,
 * else ceil(t/dt); every step has length t/nsteps.
 *
 * Potentials (all of them separable, but handled here through the general
 * gradient/Hessian):
 *   kind 0 free      V = 0
 *   kind 1 cossum    V = c0 + amp * sum_l cos(k x_l)
 *   kind 2 harmonic  V = omega^2 |x|^2 / 2
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#define DMAX 3

typedef struct {
    int kind;
    double c0, amp, k, omega;
} potential;

static double pot_value(const potential *v, int d, const double *x) {
    double s = 0.0;
    switch (v->kind) {
    case 1:
        for (int l = 0; l < d; ++l) s += cos(v->k * x[l]);
        return v->c0 + v->amp * s;
    case 2:
        for (int l = 0; l < d; ++l) s += x[l] * x[l];
        return 0.5 * v->omega * v->omega * s;
    default:
        return 0.0;
    }
}

/* gradient g[d] and Hessian hs[d][d] */
static void pot_derivs(const potential *v, int d, const double *x, double *g, double hs[DMAX][DMAX]) {
    for (int i = 0; i < d; ++i) {
        g[i] = 0.0;
        for (int j = 0; j < d; ++j) hs[i][j] = 0.0;
    }
    switch (v->kind) {
    case 1:
        for (int l = 0; l < d; ++l) {
            g[l] = -v->amp * v->k * sin(v->k * x[l]);
            hs[l][l] = -v->amp * v->k * v->k * cos(v->k * x[l]);
        }
        break;
    case 2:
        for (int l = 0; l < d; ++l) {
            g[l] = v->omega * v->omega * x[l];
            hs[l][l] = v->omega * v->omega;
        }
        break;
    default:
        break;
    }
}

/* state layout: Q[d] P[d] S F[d*d] G[d*d] H[d*d] K[d*d] Are Aim */
static int state_len(int d) { return 2 * d + 1 + 4 * d * d + 2; }

static double complex trace_zinv_zdot(int d, double complex Z[DMAX][DMAX],
                                      double complex Zd[DMAX][DMAX]) {
    /* solve Z X = Zd, return trace(X) */
    double complex a[DMAX][2 * DMAX];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            a[i][j] = Z[i][j];
            a[i][d + j] = Zd[i][j];
        }
    for (int c = 0; c < d; ++c) {
        int piv = c;
        for (int r = c + 1; r < d; ++r)
            if (cabs(a[r][c]) > cabs(a[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 2 * d; ++j) {
                double complex t = a[c][j];
                a[c][j] = a[piv][j];
                a[piv][j] = t;
            }
        for (int r = 0; r < d; ++r) {
            if (r == c) continue;
            double complex f = a[r][c] / a[c][c];
            for (int j = c; j < 2 * d; ++j) a[r][j] -= f * a[c][j];
        }
    }
    double complex tr = 0.0;
    for (int i = 0; i < d; ++i) tr += a[i][d + i] / a[i][i];
    return tr;
}

static void rhs(const potential *v, int d, const double *y, double *dy) {
    const double *Q = y, *P = y + d;
    const double *F = y + 2 * d + 1, *G = F + d * d, *H = G + d * d, *K = H + d * d;
    double A_re = y[2 * d + 1 + 4 * d * d], A_im = y[2 * d + 2 + 4 * d * d];
    double g[DMAX], hs[DMAX][DMAX];
    pot_derivs(v, d, Q, g, hs);
    double p2 = 0.0;
    for (int l = 0; l < d; ++l) {
        dy[l] = P[l];
        dy[d + l] = -g[l];
        p2 += P[l] * P[l];
    }
    dy[2 * d] = 0.5 * p2 - pot_value(v, d, Q);
    double *dF = dy + 2 * d + 1, *dG = dF + d * d, *dH = dG + d * d, *dK = dH + d * d;
    double complex Z[DMAX][DMAX], Zd[DMAX][DMAX];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double hf = 0.0, hg = 0.0;
            for (int l = 0; l < d; ++l) {
                hf += hs[i][l] * F[l * d + j];
                hg += hs[i][l] * G[l * d + j];
            }
            dF[i * d + j] = H[i * d + j];
            dG[i * d + j] = K[i * d + j];
            dH[i * d + j] = -hf;
            dK[i * d + j] = -hg;
            Z[i][j] = F[i * d + j] - I * G[i * d + j] + I * H[i * d + j] + K[i * d + j];
            Zd[i][j] = H[i * d + j] - I * K[i * d + j] - I * hf - hg;
        }
    double complex tr = trace_zinv_zdot(d, Z, Zd);
    double complex A = A_re + I * A_im;
    double complex dA = 0.5 * A * tr;
    dy[2 * d + 1 + 4 * d * d] = creal(dA);
    dy[2 * d + 2 + 4 * d * d] = cimag(dA);
}

int64_t oracle_rk4_nsteps(double t, double dt) {
    double r = t / dt;
    double n = nearbyint(r);
    if (fabs(r - n) <= 1e-9 * (n > 1.0 ? n : 1.0)) return (int64_t)n;
    return (int64_t)ceil(r);
}

/* Integrates packet j of m in place; if jac != NULL also stores the final
 * Jacobian blocks F, G, H, K (4*d*d values, row-major d x d each). */
static void integrate_one(const potential *v, int d, int64_t m, int64_t j, double *q, double *p,
                          double *s, double *a, int64_t nsteps, double h, double *jac) {
    int n = state_len(d);
    double y[64], k1[64], k2[64], k3[64], k4[64], tmp[64];
    memset(y, 0, sizeof(y));
    for (int l = 0; l < d; ++l) {
        y[l] = q[l * m + j];
        y[d + l] = p[l * m + j];
    }
    y[2 * d] = s[j];
    double *F = y + 2 * d + 1, *K = F + 3 * d * d;
    for (int l = 0; l < d; ++l) {
        F[l * d + l] = 1.0;
        K[l * d + l] = 1.0;
    }
    y[2 * d + 1 + 4 * d * d] = a[j];
    y[2 * d + 2 + 4 * d * d] = a[m + j];
    for (int64_t it = 0; it < nsteps; ++it) {
        rhs(v, d, y, k1);
        for (int i = 0; i < n; ++i) tmp[i] = y[i] + 0.5 * h * k1[i];
        rhs(v, d, tmp, k2);
        for (int i = 0; i < n; ++i) tmp[i] = y[i] + 0.5 * h * k2[i];
        rhs(v, d, tmp, k3);
        for (int i = 0; i < n; ++i) tmp[i] = y[i] + h * k3[i];
        rhs(v, d, tmp, k4);
        for (int i = 0; i < n; ++i)
            y[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    for (int l = 0; l < d; ++l) {
        q[l * m + j] = y[l];
        p[l * m + j] = y[d + l];
    }
    s[j] = y[2 * d];
    a[j] = y[2 * d + 1 + 4 * d * d];
    a[m + j] = y[2 * d + 2 + 4 * d * d];
    if (jac)
        for (int i = 0; i < 4 * d * d; ++i) jac[j * 4 * d * d + i] = y[2 * d + 1 + i];
}

/*
 * Integrates m packets in place from 0 to t (OpenMP over packets).
 * q[d*m], p[d*m] (dimension-major), s[m], a[2*m] (real plane then imaginary).
 * On entry S is taken from s (normally 0) and the Jacobians start at identity.
 * jac: NULL, or room for m*4*d*d doubles receiving the final F, G, H, K.
 * Returns 0, or -1 on bad arguments.
 */
int oracle_rk4(int d, int64_t m, double *q, double *p, double *s, double *a, int kind, double c0,
               double amp, double k, double omega, double t, double dt, double *jac) {
    if (d < 1 || d > DMAX || m < 0 || !(dt > 0.0) || t < 0.0) return -1;
    potential v = {kind, c0, amp, k, omega};
    int64_t nsteps = oracle_rk4_nsteps(t, dt);
    double h = nsteps > 0 ? t / (double)nsteps : 0.0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < m; ++j) integrate_one(&v, d, m, j, q, p, s, a, nsteps, h, jac);
    return 0;
}
