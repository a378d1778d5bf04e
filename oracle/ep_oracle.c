/*
 * ep_oracle.c -- plain FP64 CPU oracle of the geodesic landmark-shooting method
 * of Camassa, Kuang & Lee (arXiv 1510.03816).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test suite, the package smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA path.
 *
 * Every routine is the plain definition from the paper, written as double
 * loops in FP64 with no blocking, fusion or reordering:
 *   - kernel functors G, phi = G'/r, psi = phi'/r        (Sec. 3, Eq. Green-nD,
 *     the conon of Eq. nu=3/2, the Gaussian G_inf of Sec. 6, and the
 *     compactly supported tent cone used by the cell list)
 *   - right-hand side of the N-particle system            (Sec. 3.1, Eq. N-particle)
 *   - discrete Hamiltonian                                (Sec. 3.1, Eq. H)
 *   - classical Runge-Kutta shoot on [0, t1]              (Sec. 4, Note 1 item 5)
 *   - feedback-control iteration, gain M = h I            (Sec. 4, Algorithm 1;
 *     Sec. 5, Note 2 item 2)
 *   - Hessian-vector product of H and the exact discrete adjoint of the RK4
 *     shoot for the inexact-matching energy               (Sec. 6, Eq. inexact-E)
 *   - brute-force neighbour sets of the cell-list predicate (a written
 *     definition of the GPU path's FP32 acceptance test; see orc_cell_*)
 *   - the velocity field at arbitrary points             (Sec. 3.1, Eq. u)
 *     and the transport of points by the flow it generates along a shoot
 *     (the deformation phi_t with d phi_t(x)/dt = u(phi_t(x), t))
 *   - the inexact particle system, its shoot and its matching loop with the
 *     momentum-difference stop                           (Sec. 6, Eq. N-particle-inexact)
 *   - the tangent-linear RK4 shoot (directional derivative of the shooting
 *     map), the building block of the Newton-type gain M = h (D phi)^-1 of
 *     Sec. 5 (Theorem 1).
 *
 * Parity pins (tests/test_oracle_pins.py): every function here is checked
 * against something other than itself -- finite differences of H, closed
 * forms, conservation laws, the concentric-circle 1-DOF reduction and the
 * Hamiltonian values the paper prints.
 *
 * Build:  gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC -o libep_oracle.so ep_oracle.c -lm
 * -ffp-contract=off keeps every expression rounded exactly as written.  The
 * OpenMP pragmas only split the outer particle loop; each particle's sum is
 * still taken sequentially over j, so results do not depend on thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_GAUSS = 0, ORC_TENT = 1, ORC_EXPCONE = 2 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOTCONVERGED = 4, ORC_EDIVERGED = 5 };

int orc_version(void) { return 1; }

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ------------------------------------------------------------------------ */
/* Kernel functors.  r = |q_i - q_j| >= 0.                                   */
/*   Gaussian  G = exp(-r^2 / (2 sigma^2))          (metric H^inf, Sec. 6)   */
/*   tent      G = max(1 - r/sigma, 0)              (compact "conical" cone) */
/*   expcone   G = exp(-r / sigma)                  (Eq. nu=3/2 normalised,  */
/*                                                   sigma = alpha; Sec. 7)  */
/* phi = G'(r)/r and psi = phi'(r)/r.  Conventions where the derivative is   */
/* undefined: at r = 0 the tent and expcone phi/psi are taken as 0 (the      */
/* direction q_i - q_j is undefined there, and this keeps sum_i dp_i = 0);   */
/* at r >= sigma the tent G, phi and psi are all 0 (right derivative).       */
/* ------------------------------------------------------------------------ */
double orc_G(int kernel, double sigma, double r)
{
    switch (kernel) {
    case ORC_GAUSS: return exp(-(r * r) / (2.0 * sigma * sigma));
    case ORC_TENT: return r < sigma ? 1.0 - r / sigma : 0.0;
    case ORC_EXPCONE: return exp(-r / sigma);
    }
    return NAN;
}

double orc_phi(int kernel, double sigma, double r)
{
    switch (kernel) {
    case ORC_GAUSS: return -orc_G(kernel, sigma, r) / (sigma * sigma);
    case ORC_TENT: return (r > 0.0 && r < sigma) ? -1.0 / (sigma * r) : 0.0;
    case ORC_EXPCONE: return r > 0.0 ? -exp(-r / sigma) / (sigma * r) : 0.0;
    }
    return NAN;
}

double orc_psi(int kernel, double sigma, double r)
{
    switch (kernel) {
    case ORC_GAUSS: return orc_G(kernel, sigma, r) / (sigma * sigma * sigma * sigma);
    case ORC_TENT: return (r > 0.0 && r < sigma) ? 1.0 / (sigma * r * r * r) : 0.0;
    case ORC_EXPCONE:
        if (r <= 0.0) return 0.0;
        return exp(-r / sigma) * (1.0 / (sigma * sigma * r * r) + 1.0 / (sigma * r * r * r));
    }
    return NAN;
}

static double dist(int dim, const double* a, const double* b)
{
    double s = 0.0;
    for (int c = 0; c < dim; ++c) {
        double d = a[c] - b[c];
        s += d * d;
    }
    return sqrt(s);
}

static double dot(int dim, const double* a, const double* b)
{
    double s = 0.0;
    for (int c = 0; c < dim; ++c) s += a[c] * b[c];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Eq. N-particle:                                                           */
/*   dq_i/dt =  sum_{j=1..N}   G(|q_i - q_j|) p_j            (j = i included) */
/*   dp_i/dt = -sum_{j != i} (p_i . p_j) G'(r_ij) (q_i - q_j) / r_ij          */
/*           = -sum_{j != i} (p_i . p_j) phi(r_ij) (q_i - q_j)                */
/* q, p, dq, dp are (n, dim) row-major.                                      */
/* ------------------------------------------------------------------------ */
void orc_rhs(int dim, int kernel, double sigma, long n, const double* q, const double* p,
             double* dq, double* dp)
{
    long i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double sq[3] = {0, 0, 0}, sp[3] = {0, 0, 0};
        const double* qi = q + i * dim;
        const double* pi = p + i * dim;
        for (long j = 0; j < n; ++j) {
            const double* qj = q + j * dim;
            const double* pj = p + j * dim;
            double r = dist(dim, qi, qj);
            double g = orc_G(kernel, sigma, r);
            for (int c = 0; c < dim; ++c) sq[c] += g * pj[c];
            if (j != i) {
                double w = dot(dim, pi, pj) * orc_phi(kernel, sigma, r);
                for (int c = 0; c < dim; ++c) sp[c] -= w * (qi[c] - qj[c]);
            }
        }
        for (int c = 0; c < dim; ++c) {
            dq[i * dim + c] = sq[c];
            dp[i * dim + c] = sp[c];
        }
    }
}

/* Eq. H:  H = 1/2 sum_i sum_j (p_i . p_j) G(|q_i - q_j|).  The kinetic      */
/* energy of Eq. E=2H is twice this value.                                   */
double orc_hamiltonian(int dim, int kernel, double sigma, long n, const double* q, const double* p)
{
    double total = 0.0;
    for (long i = 0; i < n; ++i) {
        double row = 0.0;
        for (long j = 0; j < n; ++j)
            row += dot(dim, p + i * dim, p + j * dim) *
                   orc_G(kernel, sigma, dist(dim, q + i * dim, q + j * dim));
        total += row;
    }
    return 0.5 * total;
}

/* ------------------------------------------------------------------------ */
/* Classical fourth-order Runge-Kutta on the state x = (q, p), S uniform     */
/* steps of size dt = t1 / S (Sec. 4, Note 1 item 5 names the classical RK   */
/* scheme; the flow is normalised to end at t = 1, Eq. exact-matching).      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *q, *p;
} orc_state;

static void rk4_step(int dim, int kernel, double sigma, long n, double dt, double* q, double* p,
                     double* work /* 10 * n * dim */)
{
    long m = n * dim;
    double *k1q = work, *k1p = work + m, *k2q = work + 2 * m, *k2p = work + 3 * m;
    double *k3q = work + 4 * m, *k3p = work + 5 * m, *k4q = work + 6 * m, *k4p = work + 7 * m;
    double *yq = work + 8 * m, *yp = work + 9 * m;

    orc_rhs(dim, kernel, sigma, n, q, p, k1q, k1p);
    for (long a = 0; a < m; ++a) {
        yq[a] = q[a] + 0.5 * dt * k1q[a];
        yp[a] = p[a] + 0.5 * dt * k1p[a];
    }
    orc_rhs(dim, kernel, sigma, n, yq, yp, k2q, k2p);
    for (long a = 0; a < m; ++a) {
        yq[a] = q[a] + 0.5 * dt * k2q[a];
        yp[a] = p[a] + 0.5 * dt * k2p[a];
    }
    orc_rhs(dim, kernel, sigma, n, yq, yp, k3q, k3p);
    for (long a = 0; a < m; ++a) {
        yq[a] = q[a] + dt * k3q[a];
        yp[a] = p[a] + dt * k3p[a];
    }
    orc_rhs(dim, kernel, sigma, n, yq, yp, k4q, k4p);
    for (long a = 0; a < m; ++a) {
        q[a] += dt / 6.0 * (k1q[a] + 2.0 * k2q[a] + 2.0 * k3q[a] + k4q[a]);
        p[a] += dt / 6.0 * (k1p[a] + 2.0 * k2p[a] + 2.0 * k3p[a] + k4p[a]);
    }
}

int orc_shoot(int dim, int kernel, double sigma, int steps, double t1, long n, const double* q0,
              const double* p0, double* q1, double* p1)
{
    if (dim < 1 || dim > 3 || steps < 1 || n < 0) return ORC_EINVAL;
    long m = n * dim;
    double* work = (double*)malloc(sizeof(double) * (size_t)(10 * m + 1));
    if (!work) return ORC_EINVAL;
    memcpy(q1, q0, sizeof(double) * (size_t)m);
    memcpy(p1, p0, sizeof(double) * (size_t)m);
    double dt = t1 / steps;
    for (int s = 0; s < steps; ++s) rk4_step(dim, kernel, sigma, n, dt, q1, p1, work);
    free(work);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Eq. u: the velocity at m points x (m, dim) of the momenta p carried by    */
/* the particles q (n, dim):  u(x_k) = sum_{j=1..N} G(|x_k - q_j|) p_j.       */
/* ------------------------------------------------------------------------ */
void orc_velocity(int dim, int kernel, double sigma, long n, const double* q, const double* p, long m,
                  const double* x, double* u)
{
    long k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < m; ++k) {
        const double* xk = x + k * dim;
        double s[3] = {0.0, 0.0, 0.0};
        for (long j = 0; j < n; ++j) {
            double g = orc_G(kernel, sigma, dist(dim, xk, q + j * dim));
            for (int c = 0; c < dim; ++c) s[c] += g * p[j * dim + c];
        }
        for (int c = 0; c < dim; ++c) u[k * dim + c] = s[c];
    }
}

/* ------------------------------------------------------------------------ */
/* Transport of m points by the flow of a shoot: the joint system            */
/*   dq/dt, dp/dt = Eq. N-particle,   dx_k/dt = u(x_k, t)  (Eq. u at q(t), p(t)) */
/* integrated by the classical RK4 of the shoot (the same steps on [0, t1]), */
/* so x1 = phi_{t1}(x0).  The particles' endpoint goes to q1, p1.            */
/* ------------------------------------------------------------------------ */
int orc_flow(int dim, int kernel, double sigma, int steps, double t1, long n, const double* q0,
             const double* p0, long m, const double* x0, double* q1, double* p1, double* x1)
{
    if (dim < 1 || dim > 3 || steps < 1 || n < 0 || m < 0) return ORC_EINVAL;
    long a, nd = n * dim, md = m * dim;
    double* w = (double*)malloc(sizeof(double) * (size_t)(10 * nd + 5 * md + 1));
    if (!w) return ORC_EINVAL;
    double *k1q = w, *k1p = w + nd, *k2q = w + 2 * nd, *k2p = w + 3 * nd, *k3q = w + 4 * nd;
    double *k3p = w + 5 * nd, *k4q = w + 6 * nd, *k4p = w + 7 * nd, *yq = w + 8 * nd, *yp = w + 9 * nd;
    double *k1x = w + 10 * nd, *k2x = k1x + md, *k3x = k2x + md, *k4x = k3x + md, *yx = k4x + md;
    memcpy(q1, q0, sizeof(double) * (size_t)nd);
    memcpy(p1, p0, sizeof(double) * (size_t)nd);
    memcpy(x1, x0, sizeof(double) * (size_t)md);
    double dt = t1 / steps;
    for (int s = 0; s < steps; ++s) {
        /* stage 1 at (q, p, x) */
        orc_rhs(dim, kernel, sigma, n, q1, p1, k1q, k1p);
        orc_velocity(dim, kernel, sigma, n, q1, p1, m, x1, k1x);
        /* stage 2 at the half step along k1 */
        for (a = 0; a < nd; ++a) { yq[a] = q1[a] + 0.5 * dt * k1q[a]; yp[a] = p1[a] + 0.5 * dt * k1p[a]; }
        for (a = 0; a < md; ++a) yx[a] = x1[a] + 0.5 * dt * k1x[a];
        orc_rhs(dim, kernel, sigma, n, yq, yp, k2q, k2p);
        orc_velocity(dim, kernel, sigma, n, yq, yp, m, yx, k2x);
        /* stage 3 at the half step along k2 */
        for (a = 0; a < nd; ++a) { yq[a] = q1[a] + 0.5 * dt * k2q[a]; yp[a] = p1[a] + 0.5 * dt * k2p[a]; }
        for (a = 0; a < md; ++a) yx[a] = x1[a] + 0.5 * dt * k2x[a];
        orc_rhs(dim, kernel, sigma, n, yq, yp, k3q, k3p);
        orc_velocity(dim, kernel, sigma, n, yq, yp, m, yx, k3x);
        /* stage 4 at the full step along k3 */
        for (a = 0; a < nd; ++a) { yq[a] = q1[a] + dt * k3q[a]; yp[a] = p1[a] + dt * k3p[a]; }
        for (a = 0; a < md; ++a) yx[a] = x1[a] + dt * k3x[a];
        orc_rhs(dim, kernel, sigma, n, yq, yp, k4q, k4p);
        orc_velocity(dim, kernel, sigma, n, yq, yp, m, yx, k4x);
        for (a = 0; a < nd; ++a) {
            q1[a] += dt / 6.0 * (k1q[a] + 2.0 * k2q[a] + 2.0 * k3q[a] + k4q[a]);
            p1[a] += dt / 6.0 * (k1p[a] + 2.0 * k2p[a] + 2.0 * k3p[a] + k4p[a]);
        }
        for (a = 0; a < md; ++a) x1[a] += dt / 6.0 * (k1x[a] + 2.0 * k2x[a] + 2.0 * k3x[a] + k4x[a]);
    }
    free(w);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 with the constant gain M = h I of Sec. 5 (Note 2 item 2),    */
/* applied to the initial momenta: p0 <- p0 + h (Y - Q(1)).  p0 enters as    */
/* the initial guess (Note 1 item 4: normally zero).  Each iteration shoots  */
/* (step 1), takes the max-norm residual (step 2; the maximum norm is the    */
/* one of Sec. 6 and Table 5), stops when it is below eps, and otherwise     */
/* updates (steps 3-4).  *iters counts updates; shoots = *iters + 1.         */
/* hist (optional, maxit + 1 entries) receives the residual of each shoot.   */
/* A non-finite residual stops with ORC_EDIVERGED (the paper's NaN / "x"     */
/* entries of Tables 2-3).                                                   */
/* ------------------------------------------------------------------------ */
double orc_default_gain(int dim, int kernel, double sigma, long n, const double* X)
{
    /* Gershgorin bound on the largest eigenvalue of G(X): h = 1 / max_i sum_j |G_ij|. */
    double best = 0.0;
    for (long i = 0; i < n; ++i) {
        double row = 0.0;
        for (long j = 0; j < n; ++j) row += fabs(orc_G(kernel, sigma, dist(dim, X + i * dim, X + j * dim)));
        if (row > best) best = row;
    }
    return best > 0.0 ? 1.0 / best : 1.0;
}

int orc_match(int dim, int kernel, double sigma, int steps, double t1, long n, const double* X,
              const double* Y, double h, double eps, int maxit, double* p0, int* iters,
              double* resid, double* hist)
{
    if (dim < 1 || dim > 3 || steps < 1 || n < 0 || maxit < 0) return ORC_EINVAL;
    long m = n * dim;
    double* q1 = (double*)malloc(sizeof(double) * (size_t)(2 * m + 1));
    double* p1 = q1 + m;
    if (!q1) return ORC_EINVAL;
    if (h <= 0.0) h = orc_default_gain(dim, kernel, sigma, n, X);
    int status = ORC_ENOTCONVERGED;
    int k = 0;
    double res = 0.0;
    for (;;) {
        orc_shoot(dim, kernel, sigma, steps, t1, n, X, p0, q1, p1);
        res = 0.0;
        int finite = 1;
        for (long a = 0; a < m; ++a) {
            double r = Y[a] - q1[a];
            if (!isfinite(r)) finite = 0;
            if (fabs(r) > res) res = fabs(r);
        }
        if (!finite) res = NAN;
        if (hist) hist[k] = res;
        if (!finite) { status = ORC_EDIVERGED; break; }
        if (res < eps) { status = ORC_OK; break; }
        if (k == maxit) { status = ORC_ENOTCONVERGED; break; }
        for (long a = 0; a < m; ++a) p0[a] += h * (Y[a] - q1[a]);
        ++k;
    }
    if (iters) *iters = k;
    if (resid) *resid = res;
    free(q1);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Eq. N-particle-inexact (Sec. 6): the inexact-matching particle system.    */
/*   dq_i/dt = sum_j G(|q_i - q_j|) p_j + s2 p_i      (s2 = sigma_n^2 > 0)     */
/*   dp_i/dt = as in Eq. N-particle.                                         */
/* ------------------------------------------------------------------------ */
void orc_rhs_inexact(int dim, int kernel, double sigma, double s2, long n, const double* q, const double* p,
                     double* dq, double* dp)
{
    orc_rhs(dim, kernel, sigma, n, q, p, dq, dp);
    for (long a = 0; a < n * dim; ++a) dq[a] += s2 * p[a];
}

/* Classical RK4 of the inexact system (the shoot's scheme). */
int orc_shoot_inexact(int dim, int kernel, double sigma, double s2, int steps, double t1, long n,
                      const double* q0, const double* p0, double* q1, double* p1)
{
    if (dim < 1 || dim > 3 || steps < 1 || n < 0) return ORC_EINVAL;
    long a, m = n * dim;
    double* w = (double*)malloc(sizeof(double) * (size_t)(10 * m + 1));
    if (!w) return ORC_EINVAL;
    double *k1q = w, *k1p = w + m, *k2q = w + 2 * m, *k2p = w + 3 * m, *k3q = w + 4 * m;
    double *k3p = w + 5 * m, *k4q = w + 6 * m, *k4p = w + 7 * m, *yq = w + 8 * m, *yp = w + 9 * m;
    memcpy(q1, q0, sizeof(double) * (size_t)m);
    memcpy(p1, p0, sizeof(double) * (size_t)m);
    double dt = t1 / steps;
    for (int s = 0; s < steps; ++s) {
        orc_rhs_inexact(dim, kernel, sigma, s2, n, q1, p1, k1q, k1p);
        for (a = 0; a < m; ++a) { yq[a] = q1[a] + 0.5 * dt * k1q[a]; yp[a] = p1[a] + 0.5 * dt * k1p[a]; }
        orc_rhs_inexact(dim, kernel, sigma, s2, n, yq, yp, k2q, k2p);
        for (a = 0; a < m; ++a) { yq[a] = q1[a] + 0.5 * dt * k2q[a]; yp[a] = p1[a] + 0.5 * dt * k2p[a]; }
        orc_rhs_inexact(dim, kernel, sigma, s2, n, yq, yp, k3q, k3p);
        for (a = 0; a < m; ++a) { yq[a] = q1[a] + dt * k3q[a]; yp[a] = p1[a] + dt * k3p[a]; }
        orc_rhs_inexact(dim, kernel, sigma, s2, n, yq, yp, k4q, k4p);
        for (a = 0; a < m; ++a) {
            q1[a] += dt / 6.0 * (k1q[a] + 2.0 * k2q[a] + 2.0 * k3q[a] + k4q[a]);
            p1[a] += dt / 6.0 * (k1p[a] + 2.0 * k2p[a] + 2.0 * k3p[a] + k4p[a]);
        }
    }
    free(w);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 on the inexact system with the stopping rule of Sec. 6: stop  */
/* when the initial momenta of two consecutive iterates differ by less than  */
/* eps (maximum norm).  Each iterate shoots, records the residual            */
/* |Y - Q(1)|_inf, and updates p0 <- p0 + h (Y - Q(1)); the loop ends after  */
/* the update whose size is below eps (converged), at maxit updates (not     */
/* converged) or at a non-finite residual (diverged).  h <= 0 selects        */
/* 1 / (max_i sum_j |G_ij| + s2), the Gershgorin bound on lambda_max of the  */
/* linearised map G(X) + s2 I.  *iters counts updates; *resid is the last    */
/* shoot's residual.                                                         */
/* ------------------------------------------------------------------------ */
int orc_match_inexact(int dim, int kernel, double sigma, double s2, int steps, double t1, long n,
                      const double* X, const double* Y, double h, double eps, int maxit, double* p0,
                      int* iters, double* resid, double* hist)
{
    if (dim < 1 || dim > 3 || steps < 1 || n < 0 || maxit < 0) return ORC_EINVAL;
    long m = n * dim;
    double* q1 = (double*)malloc(sizeof(double) * (size_t)(2 * m + 1));
    double* p1 = q1 + m;
    if (!q1) return ORC_EINVAL;
    if (h <= 0.0) {
        double best = 0.0;
        for (long i = 0; i < n; ++i) {
            double row = 0.0;
            for (long j = 0; j < n; ++j) row += fabs(orc_G(kernel, sigma, dist(dim, X + i * dim, X + j * dim)));
            if (row > best) best = row;
        }
        h = 1.0 / (best + s2);
    }
    int status = ORC_ENOTCONVERGED;
    int k = 0;
    double res = 0.0;
    for (;;) {
        orc_shoot_inexact(dim, kernel, sigma, s2, steps, t1, n, X, p0, q1, p1);
        res = 0.0;
        int finite = 1;
        for (long a = 0; a < m; ++a) {
            double r = Y[a] - q1[a];
            if (!isfinite(r)) finite = 0;
            if (fabs(r) > res) res = fabs(r);
        }
        if (!finite) res = NAN;
        if (hist) hist[k] = res;
        if (!finite) { status = ORC_EDIVERGED; break; }
        if (k == maxit) { status = ORC_ENOTCONVERGED; break; }
        double dmax = 0.0;
        for (long a = 0; a < m; ++a) {
            double d = h * (Y[a] - q1[a]);
            p0[a] += d;
            if (fabs(d) > dmax) dmax = fabs(d);
        }
        ++k;
        if (dmax < eps) { status = ORC_OK; break; }
    }
    if (iters) *iters = k;
    if (resid) *resid = res;
    free(q1);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Hessian-vector product of H (Eq. H) along v = (vq, vp):                   */
/*  (d2H v)_{p_i} = sum_j [ G_ij vp_j + phi_ij (d_ij . dv_ij) p_j ]          */
/*  (d2H v)_{q_i} = sum_{j!=i} [ (vp_i . p_j + p_i . vp_j) phi_ij d_ij        */
/*                   + (p_i . p_j)(phi_ij dv_ij + psi_ij (d_ij . dv_ij) d_ij)] */
/* with d_ij = q_i - q_j and dv_ij = vq_i - vq_j.  These are the directional  */
/* derivatives of dH/dp_i = sum_j G_ij p_j and dH/dq_i = sum_{j!=i}           */
/* (p_i . p_j) phi_ij d_ij, i.e. of the two sums of Eq. N-particle.           */
/* ------------------------------------------------------------------------ */
void orc_hvp(int dim, int kernel, double sigma, long n, const double* q, const double* p,
             const double* vq, const double* vp, double* hq, double* hp)
{
    long i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double aq[3] = {0, 0, 0}, ap[3] = {0, 0, 0};
        const double *qi = q + i * dim, *pi = p + i * dim, *vqi = vq + i * dim, *vpi = vp + i * dim;
        for (long j = 0; j < n; ++j) {
            const double *qj = q + j * dim, *pj = p + j * dim, *vqj = vq + j * dim, *vpj = vp + j * dim;
            double d[3], dv[3];
            for (int c = 0; c < dim; ++c) {
                d[c] = qi[c] - qj[c];
                dv[c] = vqi[c] - vqj[c];
            }
            double r = dist(dim, qi, qj);
            double g = orc_G(kernel, sigma, r), phi = orc_phi(kernel, sigma, r),
                   psi = orc_psi(kernel, sigma, r);
            double ddv = dot(dim, d, dv);
            for (int c = 0; c < dim; ++c) ap[c] += g * vpj[c] + phi * ddv * pj[c];
            if (j != i) {
                double a = dot(dim, vpi, pj) + dot(dim, pi, vpj);
                double b = dot(dim, pi, pj);
                for (int c = 0; c < dim; ++c)
                    aq[c] += a * phi * d[c] + b * (phi * dv[c] + psi * ddv * d[c]);
            }
        }
        for (int c = 0; c < dim; ++c) {
            hq[i * dim + c] = aq[c];
            hp[i * dim + c] = ap[c];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Tangent-linear shoot: the derivative of the RK4 shoot (Q(1), P(1)) at     */
/* (q0, p0) along (vq0, vp0), obtained by differentiating each RK4 stage.    */
/* With F = (dH/dp, -dH/dq) (Eq. N-particle) its Jacobian acts as            */
/*   J_F(y) v = ( (d2H v)_p , -(d2H v)_q )          (d2H: Hessian of Eq. H)  */
/* and a step is                                                             */
/*   dk1 = J_F(x) dx,          dk2 = J_F(y2) (dx + dt/2 dk1),                */
/*   dk3 = J_F(y3) (dx + dt/2 dk2),  dk4 = J_F(y4) (dx + dt dk3),            */
/*   dx <- dx + dt/6 (dk1 + 2 dk2 + 2 dk3 + dk4),                            */
/* at the stage states y_s of the primal step, which is advanced alongside.  */
/* ------------------------------------------------------------------------ */
int orc_shoot_tangent(int dim, int kernel, double sigma, int steps, double t1, long n, const double* q0,
                      const double* p0, const double* vq0, const double* vp0, double* q1, double* p1,
                      double* vq1, double* vp1)
{
    if (dim < 1 || dim > 3 || steps < 1 || n < 0) return ORC_EINVAL;
    long a, m = n * dim;
    double* w = (double*)malloc(sizeof(double) * (size_t)(24 * m + 1));
    if (!w) return ORC_EINVAL;
    double *kq[4], *kp[4], *dkq[4], *dkp[4];
    for (int s = 0; s < 4; ++s) {
        kq[s] = w + (4 * s + 0) * m;
        kp[s] = w + (4 * s + 1) * m;
        dkq[s] = w + (4 * s + 2) * m;
        dkp[s] = w + (4 * s + 3) * m;
    }
    double *yq = w + 16 * m, *yp = w + 17 * m, *dyq = w + 18 * m, *dyp = w + 19 * m;
    double *hq = w + 20 * m, *hp = w + 21 * m;
    memcpy(q1, q0, sizeof(double) * (size_t)m);
    memcpy(p1, p0, sizeof(double) * (size_t)m);
    memcpy(vq1, vq0, sizeof(double) * (size_t)m);
    memcpy(vp1, vp0, sizeof(double) * (size_t)m);
    const double dt = t1 / steps;
    const double c[4] = {0.0, 0.5, 0.5, 1.0};  /* stage s input: x + c_s dt k_{s-1} */
    for (int st = 0; st < steps; ++st) {
        for (int s = 0; s < 4; ++s) {
            for (a = 0; a < m; ++a) {
                yq[a] = s == 0 ? q1[a] : q1[a] + c[s] * dt * kq[s - 1][a];
                yp[a] = s == 0 ? p1[a] : p1[a] + c[s] * dt * kp[s - 1][a];
                dyq[a] = s == 0 ? vq1[a] : vq1[a] + c[s] * dt * dkq[s - 1][a];
                dyp[a] = s == 0 ? vp1[a] : vp1[a] + c[s] * dt * dkp[s - 1][a];
            }
            orc_rhs(dim, kernel, sigma, n, yq, yp, kq[s], kp[s]);
            orc_hvp(dim, kernel, sigma, n, yq, yp, dyq, dyp, hq, hp);
            for (a = 0; a < m; ++a) {
                dkq[s][a] = hp[a];
                dkp[s][a] = -hq[a];
            }
        }
        for (a = 0; a < m; ++a) {
            q1[a] += dt / 6.0 * (kq[0][a] + 2.0 * kq[1][a] + 2.0 * kq[2][a] + kq[3][a]);
            p1[a] += dt / 6.0 * (kp[0][a] + 2.0 * kp[1][a] + 2.0 * kp[2][a] + kp[3][a]);
            vq1[a] += dt / 6.0 * (dkq[0][a] + 2.0 * dkq[1][a] + 2.0 * dkq[2][a] + dkq[3][a]);
            vp1[a] += dt / 6.0 * (dkp[0][a] + 2.0 * dkp[1][a] + 2.0 * dkp[2][a] + dkp[3][a]);
        }
    }
    free(w);
    return ORC_OK;
}

/* Transposed Jacobian of F = (dH/dp, -dH/dq) applied to w = (wq, wp):       */
/*   J_F^T w = d2H . (-wp, wq), since J_F = S d2H with S the symplectic form. */
static void jac_t(int dim, int kernel, double sigma, long n, const double* q, const double* p,
                  const double* wq, const double* wp, double* oq, double* op, double* tmp)
{
    long m = n * dim;
    double* negwp = tmp;
    for (long a = 0; a < m; ++a) negwp[a] = -wp[a];
    orc_hvp(dim, kernel, sigma, n, q, p, negwp, wq, oq, op);
}

/* ------------------------------------------------------------------------ */
/* Inexact-matching energy (Eq. inexact-E written with Eq. E=2H):            */
/*   E(p0) = 1/2 p0^T G(X) p0 + lambda/2 || Q(1) - Y ||^2                     */
/*         = H(X, p0)          + lambda/2 || Q(1) - Y ||^2                     */
/* (the paper's form is 2E with lambda = 1/sigma_n^2).  The gradient dE/dp0  */
/* is the exact discrete adjoint of the RK4 shoot: all S + 1 step states are */
/* kept (no checkpointing here), and the four stages of each step are        */
/* recomputed and reversed:                                                  */
/*   kb4 = kb1 = dt/6 a,  kb2 = kb3 = dt/3 a,  xb = a                        */
/*   stage 4: y = J(y4)^T kb4, xb += y, kb3 += dt y                          */
/*   stage 3: y = J(y3)^T kb3, xb += y, kb2 += dt/2 y                        */
/*   stage 2: y = J(y2)^T kb2, xb += y, kb1 += dt/2 y                        */
/*   stage 1: xb += J(x)^T kb1                                               */
/* starting from a = (lambda (Q(1) - Y), 0).  dE/dp0 = G(X) p0 + xb_p.       */
/* Returns E; writes grad (n, dim).                                          */
/* ------------------------------------------------------------------------ */
double orc_adjoint(int dim, int kernel, double sigma, int steps, double t1, long n,
                   const double* X, const double* p0, const double* Y, double lambda, double* grad)
{
    long m = n * dim;
    double dt = t1 / steps;
    double* traj = (double*)malloc(sizeof(double) * (size_t)(2 * m * (steps + 1) + 1));
    double* work = (double*)malloc(sizeof(double) * (size_t)(10 * m + 1));
    double* st = (double*)malloc(sizeof(double) * (size_t)(24 * m + 1));
    if (!traj || !work || !st) {
        free(traj); free(work); free(st);
        return NAN;
    }
    /* forward, storing every step state (q_n, p_n) */
    memcpy(traj, X, sizeof(double) * (size_t)m);
    memcpy(traj + m, p0, sizeof(double) * (size_t)m);
    for (int s = 0; s < steps; ++s) {
        double* cur = traj + 2 * m * s;
        double* nxt = traj + 2 * m * (s + 1);
        memcpy(nxt, cur, sizeof(double) * (size_t)(2 * m));
        rk4_step(dim, kernel, sigma, n, dt, nxt, nxt + m, work);
    }
    const double* Q1 = traj + 2 * m * steps;
    double mis = 0.0;
    for (long a = 0; a < m; ++a) mis += (Q1[a] - Y[a]) * (Q1[a] - Y[a]);
    double energy = orc_hamiltonian(dim, kernel, sigma, n, X, p0) + 0.5 * lambda * mis;

    /* adjoint state xb = (xbq, xbp) */
    double *xbq = st, *xbp = st + m;
    double *kb1q = st + 2 * m, *kb1p = st + 3 * m, *kb2q = st + 4 * m, *kb2p = st + 5 * m;
    double *kb3q = st + 6 * m, *kb3p = st + 7 * m, *kb4q = st + 8 * m, *kb4p = st + 9 * m;
    double *y2q = st + 10 * m, *y2p = st + 11 * m, *y3q = st + 12 * m, *y3p = st + 13 * m;
    double *y4q = st + 14 * m, *y4p = st + 15 * m, *k1q = st + 16 * m, *k1p = st + 17 * m;
    double *k2q = st + 18 * m, *k2p = st + 19 * m, *k3q = st + 20 * m, *k3p = st + 21 * m;
    double *yq = st + 22 * m, *yp = st + 23 * m;
    double* tmp = work;
    for (long a = 0; a < m; ++a) {
        xbq[a] = lambda * (Q1[a] - Y[a]);
        xbp[a] = 0.0;
    }
    for (int s = steps - 1; s >= 0; --s) {
        const double* xq = traj + 2 * m * s;
        const double* xp = xq + m;
        /* recompute the stage inputs of step s */
        orc_rhs(dim, kernel, sigma, n, xq, xp, k1q, k1p);
        for (long a = 0; a < m; ++a) { y2q[a] = xq[a] + 0.5 * dt * k1q[a]; y2p[a] = xp[a] + 0.5 * dt * k1p[a]; }
        orc_rhs(dim, kernel, sigma, n, y2q, y2p, k2q, k2p);
        for (long a = 0; a < m; ++a) { y3q[a] = xq[a] + 0.5 * dt * k2q[a]; y3p[a] = xp[a] + 0.5 * dt * k2p[a]; }
        orc_rhs(dim, kernel, sigma, n, y3q, y3p, k3q, k3p);
        for (long a = 0; a < m; ++a) { y4q[a] = xq[a] + dt * k3q[a]; y4p[a] = xp[a] + dt * k3p[a]; }
        /* reverse */
        for (long a = 0; a < m; ++a) {
            kb1q[a] = kb4q[a] = dt / 6.0 * xbq[a];
            kb1p[a] = kb4p[a] = dt / 6.0 * xbp[a];
            kb2q[a] = kb3q[a] = dt / 3.0 * xbq[a];
            kb2p[a] = kb3p[a] = dt / 3.0 * xbp[a];
        }
        jac_t(dim, kernel, sigma, n, y4q, y4p, kb4q, kb4p, yq, yp, tmp);
        for (long a = 0; a < m; ++a) {
            xbq[a] += yq[a]; xbp[a] += yp[a];
            kb3q[a] += dt * yq[a]; kb3p[a] += dt * yp[a];
        }
        jac_t(dim, kernel, sigma, n, y3q, y3p, kb3q, kb3p, yq, yp, tmp);
        for (long a = 0; a < m; ++a) {
            xbq[a] += yq[a]; xbp[a] += yp[a];
            kb2q[a] += 0.5 * dt * yq[a]; kb2p[a] += 0.5 * dt * yp[a];
        }
        jac_t(dim, kernel, sigma, n, y2q, y2p, kb2q, kb2p, yq, yp, tmp);
        for (long a = 0; a < m; ++a) {
            xbq[a] += yq[a]; xbp[a] += yp[a];
            kb1q[a] += 0.5 * dt * yq[a]; kb1p[a] += 0.5 * dt * yp[a];
        }
        jac_t(dim, kernel, sigma, n, xq, xp, kb1q, kb1p, yq, yp, tmp);
        for (long a = 0; a < m; ++a) { xbq[a] += yq[a]; xbp[a] += yp[a]; }
    }
    /* dE/dp0 = G(X) p0 (= dH/dp at t = 0) + xb_p */
    orc_rhs(dim, kernel, sigma, n, X, p0, k1q, k1p);
    for (long a = 0; a < m; ++a) grad[a] = k1q[a] + xbp[a];
    free(traj); free(work); free(st);
    return energy;
}

/* ------------------------------------------------------------------------ */
/* Brute-force neighbour sets of the cell-list acceptance test.  This is a   */
/* written definition, not arithmetic of the method: it fixes which pairs   */
/* the GPU cell-list path evaluates, so that its neighbour sets can be      */
/* compared bit for bit.  The grid and the FP32 local coordinates are        */
/*   h      = sigma * 1.00390625                (cell edge, sigma (1 + 2^-8)) */
/*   lo_c   = min_i q_ic - 2 h                  (per axis)                   */
/*   nc_c   = min(floor((max_i q_ic - min_i q_ic) / h) + 5, cap_c)            */
/*            cap_c = 2048 (2-D) or 256 (3-D); when capped, h is replaced by  */
/*            h_c = (max - min + 4 h) / (cap_c - 1) on that axis (h_c >= h)   */
/*   t      = q_ic - lo_c                        (FP64)                      */
/*   cell_c = clamp((long)floor(t * (1 / h_c)), 0, nc_c - 1)                  */
/*   o_c    = (float)((t - cell_c * h_c) * (1 / sigma))     (FP64, one round) */
/*   e_c    = (float)(h_c * (1 / sigma))                                     */
/* and a pair (i, j) with |cell_ic - cell_jc| <= 1 on every axis is accepted  */
/* iff, in FP32 round-to-nearest with no contraction,                        */
/*   d_c = (o_ic - o_jc) + (float)(cell_ic - cell_jc) * e_c                   */
/*   r2  = fmaf(d_0, d_0, d_1 * d_1)                 (2-D)                   */
/*   r2  = fmaf(d_0, d_0, fmaf(d_1, d_1, d_2 * d_2)) (3-D)                   */
/*   r2 < 1.0f.                                                              */
/* Pairs in non-adjacent cells are never accepted (their true distance is    */
/* >= h > sigma).  Self pairs (i = j) are accepted.                          */
/* out_count[i] = number of accepted j; out_hash[i] = sum over accepted j of */
/* (j + 1) * 2654435761 mod 2^64 (an order-independent set fingerprint).     */
/* Returns the total number of accepted pairs.                               */
/* ------------------------------------------------------------------------ */
void orc_cell_grid(int dim, double sigma, long n, const double* q, double* lo, double* hc, long* nc)
{
    double h = sigma * 1.00390625;
    long cap = dim == 2 ? 2048 : 256;
    for (int c = 0; c < dim; ++c) {
        double mn = INFINITY, mx = -INFINITY;
        for (long i = 0; i < n; ++i) {
            if (q[i * dim + c] < mn) mn = q[i * dim + c];
            if (q[i * dim + c] > mx) mx = q[i * dim + c];
        }
        if (n == 0) { mn = 0.0; mx = 0.0; }
        lo[c] = mn - 2.0 * h;
        double cells = floor((mx - mn) / h) + 5.0;
        if (cells > (double)cap) {
            nc[c] = cap;
            hc[c] = (mx - mn + 4.0 * h) / (double)(cap - 1);
        } else {
            nc[c] = (long)cells;
            hc[c] = h;
        }
    }
}

long orc_cell_neighbors(int dim, double sigma, long n, const double* q, long* out_count,
                        unsigned long long* out_hash)
{
    double lo[3] = {0, 0, 0}, hc[3] = {1, 1, 1};
    long nc[3] = {1, 1, 1};
    orc_cell_grid(dim, sigma, n, q, lo, hc, nc);
    long* cell = (long*)malloc(sizeof(long) * (size_t)(n * dim + 1));
    float* off = (float*)malloc(sizeof(float) * (size_t)(n * dim + 1));
    float e[3];
    double inv_sigma = 1.0 / sigma;
    for (int c = 0; c < dim; ++c) e[c] = (float)(hc[c] * inv_sigma);
    for (long i = 0; i < n; ++i) {
        for (int c = 0; c < dim; ++c) {
            double t = q[i * dim + c] - lo[c];
            double inv_h = 1.0 / hc[c];
            long k = (long)floor(t * inv_h);
            if (k < 0) k = 0;
            if (k > nc[c] - 1) k = nc[c] - 1;
            cell[i * dim + c] = k;
            off[i * dim + c] = (float)((t - (double)k * hc[c]) * inv_sigma);
        }
    }
    long total = 0;
    long i;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (i = 0; i < n; ++i) {
        long cnt = 0;
        unsigned long long hsum = 0ULL;
        for (long j = 0; j < n; ++j) {
            int adjacent = 1;
            float d[3] = {0.f, 0.f, 0.f};
            for (int c = 0; c < dim; ++c) {
                long dc = cell[i * dim + c] - cell[j * dim + c];
                if (dc < -1 || dc > 1) { adjacent = 0; break; }
                float diff = off[i * dim + c] - off[j * dim + c];
                float shift = (float)dc * e[c];
                d[c] = diff + shift;
            }
            if (!adjacent) continue;
            float r2;
            if (dim == 2) {
                float t1 = d[1] * d[1];
                r2 = fmaf(d[0], d[0], t1);
            } else {
                float t2 = d[2] * d[2];
                float t1 = fmaf(d[1], d[1], t2);
                r2 = fmaf(d[0], d[0], t1);
            }
            if (r2 < 1.0f) {
                ++cnt;
                hsum += (unsigned long long)(j + 1) * 2654435761ULL;
            }
        }
        out_count[i] = cnt;
        out_hash[i] = hsum;
        total += cnt;
    }
    free(cell);
    free(off);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Row-sampled variants, for checks at sizes where the full double loop is   */
/* too slow: the same sums for the listed particles i only (all j).          */
/* ------------------------------------------------------------------------ */
void orc_rhs_rows(int dim, int kernel, double sigma, long n, const double* q, const double* p,
                  const long* rows, long nrows, double* dq, double* dp)
{
    long r;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < nrows; ++r) {
        const long i = rows[r];
        double sq[3] = {0, 0, 0}, sp[3] = {0, 0, 0};
        const double* qi = q + i * dim;
        const double* pi = p + i * dim;
        for (long j = 0; j < n; ++j) {
            const double* qj = q + j * dim;
            const double* pj = p + j * dim;
            double rr = dist(dim, qi, qj);
            double g = orc_G(kernel, sigma, rr);
            for (int c = 0; c < dim; ++c) sq[c] += g * pj[c];
            if (j != i) {
                double w = dot(dim, pi, pj) * orc_phi(kernel, sigma, rr);
                for (int c = 0; c < dim; ++c) sp[c] -= w * (qi[c] - qj[c]);
            }
        }
        for (int c = 0; c < dim; ++c) {
            dq[r * dim + c] = sq[c];
            dp[r * dim + c] = sp[c];
        }
    }
}

void orc_cell_neighbors_rows(int dim, double sigma, long n, const double* q, const long* rows, long nrows,
                             long* out_count, unsigned long long* out_hash)
{
    double lo[3] = {0, 0, 0}, hc[3] = {1, 1, 1};
    long nc[3] = {1, 1, 1};
    orc_cell_grid(dim, sigma, n, q, lo, hc, nc);
    long* cell = (long*)malloc(sizeof(long) * (size_t)(n * dim + 1));
    float* off = (float*)malloc(sizeof(float) * (size_t)(n * dim + 1));
    float e[3];
    double inv_sigma = 1.0 / sigma;
    for (int c = 0; c < dim; ++c) e[c] = (float)(hc[c] * inv_sigma);
    for (long i = 0; i < n; ++i)
        for (int c = 0; c < dim; ++c) {
            double t = q[i * dim + c] - lo[c];
            double inv_h = 1.0 / hc[c];
            long k = (long)floor(t * inv_h);
            if (k < 0) k = 0;
            if (k > nc[c] - 1) k = nc[c] - 1;
            cell[i * dim + c] = k;
            off[i * dim + c] = (float)((t - (double)k * hc[c]) * inv_sigma);
        }
    long r;
#pragma omp parallel for schedule(dynamic, 16)
    for (r = 0; r < nrows; ++r) {
        const long i = rows[r];
        long cnt = 0;
        unsigned long long hsum = 0ULL;
        for (long j = 0; j < n; ++j) {
            int adjacent = 1;
            float d[3] = {0.f, 0.f, 0.f};
            for (int c = 0; c < dim; ++c) {
                long dc = cell[i * dim + c] - cell[j * dim + c];
                if (dc < -1 || dc > 1) { adjacent = 0; break; }
                float diff = off[i * dim + c] - off[j * dim + c];
                float shift = (float)dc * e[c];
                d[c] = diff + shift;
            }
            if (!adjacent) continue;
            float r2;
            if (dim == 2) {
                float t1 = d[1] * d[1];
                r2 = fmaf(d[0], d[0], t1);
            } else {
                float t2 = d[2] * d[2];
                float t1 = fmaf(d[1], d[1], t2);
                r2 = fmaf(d[0], d[0], t1);
            }
            if (r2 < 1.0f) {
                ++cnt;
                hsum += (unsigned long long)(j + 1) * 2654435761ULL;
            }
        }
        out_count[r] = cnt;
        out_hash[r] = hsum;
    }
    free(cell);
    free(off);
}
