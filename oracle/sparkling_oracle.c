/*
 * FP64 CPU oracle for the SPARKLING hot path (arxiv 2108.02991).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header
 * or constant with the CUDA library and never calls it.
 *
 * Everything is computed in IEEE double, built with -ffp-contract=off so the
 * arithmetic is the same sequence of roundings on every host.  Sums run in
 * index order; OpenMP only splits independent targets (or shots), so results
 * do not depend on the thread count.
 *
 * Notation (Sec. II-B, eqs. attraction_term / repulsion_term with H = |.|_2):
 *   K[i] in [-1/2,1/2]^3, i = 0..N-1 (shot after shot);
 *   density points x_q at the cell centres of an nx x ny x nz grid over
 *   [lo,hi]^3, weights rho_q (array [nz][ny][nx], x fastest);
 *   A_i = sum_q rho_q (K_i - x_q) / |K_i - x_q|          (attraction force)
 *   R_i = (1/N) sum_{j != i} (K_i - K_j) / |K_i - K_j|   (repulsion force)
 *   G_i = A_i - R_i = N dF/dK_i                          (eq. Fr_grad, H' = 1)
 *   F^a = (1/N) sum_i sum_q rho_q |K_i - x_q|
 *   F^r = (1/(2N^2)) sum_{i != j} |K_i - K_j|
 * A term whose difference vector is exactly zero contributes nothing (the
 * minimum-norm subgradient of |.| at 0; the paper only excludes j = i).
 *
 * Every entry point also takes eps >= 0 for the regularised kernel
 * H(r) = sqrt(r^2 + eps^2) of Sec. II-C (choice of step size): each |d|
 * above becomes |d|_eps = sqrt(|d|^2 + eps^2) and each unit vector
 * d / |d| becomes d / |d|_eps (the gradient of |d|_eps).  eps = 0 is the
 * plain norm; with eps > 0 no term is singular and none is skipped (F^r
 * still sums over j != i only).
 *
 * Projection (Sec. II-D and Suppl. Sec. I): each shot s in R^{Ns x 3} is
 * projected onto {|s|_inf <= box, s[pin] = v, |D1 s|_{2,inf} <= alpha,
 * |D2 s|_{2,inf} <= beta} (eq. constraints) by accelerated proximal gradient
 * (FISTA) on the Fenchel dual of min 1/2 |s - k|^2.  The paper delegates the
 * algorithm to its reference [Chauffert TMI'16]; the dual form used here is:
 *   D1 s[n] = s[n+1] - s[n]            n = 0..Ns-2
 *   D2 s[n] = s[n+2] - 2 s[n+1] + s[n] n = 0..Ns-3
 *   primal map  s(q) = pin(clip_box(k - D1^T q1 - D2^T q2))
 *   step tau = 1/20  (|D1|^2 <= 4, |D2|^2 <= 16)
 *   z = y + tau D s(y);  q+ = z - P_{ball(tau*alpha)}(z) row-wise (and beta)
 *   t+ = (1 + sqrt(1 + 4 t^2)) / 2;  y = q+ + ((t - 1) / t+) (q+ - q)
 *   output s(q) after n_iter iterations (q = y = 0, t = 1 at the start).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ENOTCONV 6

/* Cell-centre coordinate of cell q of n over [lo, hi]. */
static double centre(int64_t q, int64_t n, double lo, double hi)
{
    return lo + ((double)q + 0.5) * ((hi - lo) / (double)n);
}

/* Attraction force and energy sum of one target position (kx,ky,kz). */
static void attraction_one(double kx, double ky, double kz, const double *rho,
                           int64_t nx, int64_t ny, int64_t nz, double lo, double hi,
                           double eps, double out[3], double *energy)
{
    double ax = 0.0, ay = 0.0, az = 0.0, e = 0.0;
    for (int64_t iz = 0; iz < nz; ++iz) {
        double z = centre(iz, nz, lo, hi);
        for (int64_t iy = 0; iy < ny; ++iy) {
            double y = centre(iy, ny, lo, hi);
            const double *row = rho + (iz * ny + iy) * nx;
            for (int64_t ix = 0; ix < nx; ++ix) {
                double x = centre(ix, nx, lo, hi);
                double dx = kx - x, dy = ky - y, dz = kz - z;
                double r = sqrt(dx * dx + dy * dy + dz * dz + eps * eps);
                if (r == 0.0)
                    continue;
                double w = row[ix];
                ax += w * (dx / r);
                ay += w * (dy / r);
                az += w * (dz / r);
                e += w * r;
            }
        }
    }
    out[0] = ax; out[1] = ay; out[2] = az;
    *energy = e;
}

/* Sum over j != skip of the unit vectors (p - K_j)/|p - K_j| and of the
 * distances |p - K_j| for a point p = (kx, ky, kz) (not yet scaled by 1/N). */
static void repulsion_at(const double *K, int64_t N, int64_t skip, double kx, double ky,
                         double kz, double eps, double out[3], double *energy)
{
    double rx = 0.0, ry = 0.0, rz = 0.0, e = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        if (j == skip)
            continue;
        double dx = kx - K[3 * j], dy = ky - K[3 * j + 1], dz = kz - K[3 * j + 2];
        double r = sqrt(dx * dx + dy * dy + dz * dz + eps * eps);
        if (r == 0.0)
            continue;
        rx += dx / r;
        ry += dy / r;
        rz += dz / r;
        e += r;
    }
    out[0] = rx; out[1] = ry; out[2] = rz;
    *energy = e;
}

/* The same sums for sample i at its own position K_i. */
static void repulsion_one(const double *K, int64_t N, int64_t i, double eps, double out[3],
                          double *energy)
{
    repulsion_at(K, N, i, K[3 * i], K[3 * i + 1], K[3 * i + 2], eps, out, energy);
}

/*
 * Forces for M targets.  targets[m] is an index into K (targets == NULL means
 * m itself, with M = N).  Writes A, R and G = A - R as [M][3] (any of them may
 * be NULL), and per-target energy sums ea[m] = sum_q rho_q |K_i - x_q|,
 * er[m] = sum_{j != i} |K_i - K_j| (may be NULL).
 */
int oracle_forces(const double *K, int64_t N, const double *rho, int64_t nx, int64_t ny,
                  int64_t nz, double lo, double hi, const int64_t *targets, int64_t M,
                  double *A, double *R, double *G, double *ea, double *er, double eps)
{
    if (!K || N < 1 || !rho || nx < 1 || ny < 1 || nz < 1 || !(hi > lo) || M < 0 || !(eps >= 0.0))
        return ORACLE_EINVAL;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t m = 0; m < M; ++m) {
        int64_t i = targets ? targets[m] : m;
        if (i < 0 || i >= N) {
            bad = 1;
            continue;
        }
        double a[3], r[3], eA, eR;
        attraction_one(K[3 * i], K[3 * i + 1], K[3 * i + 2], rho, nx, ny, nz, lo, hi, eps, a, &eA);
        repulsion_one(K, N, i, eps, r, &eR);
        for (int c = 0; c < 3; ++c) {
            double rc = r[c] / (double)N;
            if (A) A[3 * m + c] = a[c];
            if (R) R[3 * m + c] = rc;
            if (G) G[3 * m + c] = a[c] - rc;
        }
        if (ea) ea[m] = eA;
        if (er) er[m] = eR;
    }
    return bad ? ORACLE_EINVAL : ORACLE_OK;
}

/* Attraction force A(y) = sum_q rho_q (y - x_q)/|y - x_q| and potential
 * phi(y) = sum_q rho_q |y - x_q| at M arbitrary points P[M][3] (the field
 * whose gradient enters eq. attraction_derivative_basic; the paper evaluates
 * it on a grid and interpolates). Either output may be NULL. */
int oracle_attraction_at(const double *P, int64_t M, const double *rho, int64_t nx, int64_t ny,
                         int64_t nz, double lo, double hi, double *A, double *phi, double eps)
{
    if (!P || M < 0 || !rho || nx < 1 || ny < 1 || nz < 1 || !(hi > lo) || !(eps >= 0.0))
        return ORACLE_EINVAL;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < M; ++m) {
        double a[3], e;
        attraction_one(P[3 * m], P[3 * m + 1], P[3 * m + 2], rho, nx, ny, nz, lo, hi, eps, a, &e);
        if (A) { A[3 * m] = a[0]; A[3 * m + 1] = a[1]; A[3 * m + 2] = a[2]; }
        if (phi) phi[m] = e;
    }
    return ORACLE_OK;
}

/* The terms of F that contain one sample, with that sample moved: for M
 * pairs (idx[m], P[m]), sample i = idx[m] placed at the point p = P[m]:
 *   ea[m] = sum_q rho_q |p - x_q|,   er[m] = sum_{j != i} |p - K_j|.
 * In eq. global_minimization only (1/N) ea - (1/N^2) er depends on K_i (the
 * repulsion's double sum holds each pair twice), so central differences of
 * it in one coordinate of p give dF/dK_i without subtracting two energies of
 * size O(1).  OpenMP splits the M pairs. */
int oracle_energy_terms(const double *K, int64_t N, const double *rho, int64_t nx, int64_t ny,
                        int64_t nz, double lo, double hi, const int64_t *idx, const double *P,
                        int64_t M, double *ea, double *er, double eps)
{
    if (!K || N < 1 || !rho || nx < 1 || ny < 1 || nz < 1 || !(hi > lo) || M < 0 || !idx ||
        !P || !ea || !er || !(eps >= 0.0))
        return ORACLE_EINVAL;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (int64_t m = 0; m < M; ++m) {
        const int64_t i = idx[m];
        if (i < 0 || i >= N) {
            bad = 1;
            continue;
        }
        double a[3], r[3], eA, eR;
        attraction_one(P[3 * m], P[3 * m + 1], P[3 * m + 2], rho, nx, ny, nz, lo, hi, eps, a, &eA);
        repulsion_at(K, N, i, P[3 * m], P[3 * m + 1], P[3 * m + 2], eps, r, &eR);
        ea[m] = eA;
        er[m] = eR;
    }
    return bad ? ORACLE_EINVAL : ORACLE_OK;
}

/* Energy F = F^a - F^r (eqs. global_minimization, attraction_term,
 * repulsion_term); the per-target sums are added in index order. */
int oracle_energy(const double *K, int64_t N, const double *rho, int64_t nx, int64_t ny,
                  int64_t nz, double lo, double hi, double *Fa, double *Fr, double eps)
{
    double *ea = (double *)malloc(sizeof(double) * (size_t)N);
    double *er = (double *)malloc(sizeof(double) * (size_t)N);
    if (!ea || !er) {
        free(ea); free(er);
        return ORACLE_EINVAL;
    }
    int st = oracle_forces(K, N, rho, nx, ny, nz, lo, hi, NULL, N, NULL, NULL, NULL, ea, er, eps);
    if (st == ORACLE_OK) {
        double sa = 0.0, sr = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            sa += ea[i];
            sr += er[i];
        }
        *Fa = sa / (double)N;
        *Fr = sr / (2.0 * (double)N * (double)N);
    }
    free(ea); free(er);
    return st;
}

/* ---------------------------------------------------------------------- */
/* Projection onto the per-shot constraint set (eq. constraints).           */

/* Primal map s = pin(clip(k - D1^T q1 - D2^T q2)); q1 has Ns-1 rows, q2 Ns-2. */
static void primal(const double *k, const double *q1, const double *q2, int Ns, double box,
                   int pin_index, const double *pin, double *s)
{
    for (int m = 0; m < Ns; ++m) {
        for (int c = 0; c < 3; ++c) {
            double d1 = 0.0, d2 = 0.0;
            /* (D1^T q1)[m] = q1[m-1] - q1[m] */
            if (m - 1 >= 0 && m - 1 < Ns - 1) d1 += q1[3 * (m - 1) + c];
            if (m < Ns - 1) d1 -= q1[3 * m + c];
            /* (D2^T q2)[m] = q2[m-2] - 2 q2[m-1] + q2[m] */
            if (m - 2 >= 0 && m - 2 < Ns - 2) d2 += q2[3 * (m - 2) + c];
            if (m - 1 >= 0 && m - 1 < Ns - 2) d2 -= 2.0 * q2[3 * (m - 1) + c];
            if (m < Ns - 2) d2 += q2[3 * m + c];
            double v = k[3 * m + c] - d1 - d2;
            if (v > box) v = box;
            if (v < -box) v = -box;
            s[3 * m + c] = v;
        }
    }
    if (pin_index >= 0 && pin_index < Ns)
        for (int c = 0; c < 3; ++c)
            s[3 * pin_index + c] = pin[c];
}

/* z - P_{ball(radius)}(z) for one 3-vector, i.e. z * max(0, 1 - radius/|z|). */
static void shrink(double z[3], double radius, double out[3])
{
    double nz = sqrt(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
    double f = 0.0;
    if (nz > radius)
        f = 1.0 - radius / nz;
    out[0] = z[0] * f; out[1] = z[1] * f; out[2] = z[2] * f;
}

/* Largest constraint violation of one shot: out[0] amplitude (|D1 s| - alpha)+,
 * out[1] slew (|D2 s| - beta)+, out[2] box, out[3] pin error (max abs). */
static void violation_one(const double *s, int Ns, double alpha, double beta, double box,
                          int pin_index, const double *pin, double out[4])
{
    double v1 = 0.0, v2 = 0.0, vb = 0.0, vp = 0.0;
    for (int n = 0; n + 1 < Ns; ++n) {
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = s[3 * (n + 1) + c] - s[3 * n + c];
        double e = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - alpha;
        if (e > v1) v1 = e;
    }
    for (int n = 0; n + 2 < Ns; ++n) {
        double d[3];
        for (int c = 0; c < 3; ++c)
            d[c] = s[3 * (n + 2) + c] - 2.0 * s[3 * (n + 1) + c] + s[3 * n + c];
        double e = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - beta;
        if (e > v2) v2 = e;
    }
    for (int m = 0; m < 3 * Ns; ++m) {
        double e = fabs(s[m]) - box;
        if (e > vb) vb = e;
    }
    if (pin_index >= 0 && pin_index < Ns)
        for (int c = 0; c < 3; ++c) {
            double e = fabs(s[3 * pin_index + c] - pin[c]);
            if (e > vp) vp = e;
        }
    out[0] = v1; out[1] = v2; out[2] = vb; out[3] = vp;
}

/* Duality gap of the dual point q at its primal image s = s(q):
 *   gap = sum_n (alpha |q1_n| - <q1_n, D1 s_n>) + (beta |q2_n| - <q2_n, D2 s_n>).
 * When s is feasible, 1/2 |s - s*|^2 <= gap (the primal objective is
 * 1-strongly convex and bounded below by the dual one). */
static double dual_gap(const double *s, const double *q1, const double *q2, int Ns, double alpha,
                       double beta)
{
    double g = 0.0;
    for (int n = 0; n + 1 < Ns; ++n) {
        double nq = 0.0, ip = 0.0;
        for (int c = 0; c < 3; ++c) {
            double d = s[3 * (n + 1) + c] - s[3 * n + c];
            nq += q1[3 * n + c] * q1[3 * n + c];
            ip += q1[3 * n + c] * d;
        }
        g += alpha * sqrt(nq) - ip;
    }
    for (int n = 0; n + 2 < Ns; ++n) {
        double nq = 0.0, ip = 0.0;
        for (int c = 0; c < 3; ++c) {
            double d = s[3 * (n + 2) + c] - 2.0 * s[3 * (n + 1) + c] + s[3 * n + c];
            nq += q2[3 * n + c] * q2[3 * n + c];
            ip += q2[3 * n + c] * d;
        }
        g += beta * sqrt(nq) - ip;
    }
    return g;
}

/* Converged-mode certificate: every violation of the (possibly shrunk) set
 * and the duality gap are <= tol. */
static int certified(const double *s, const double *q1, const double *q2, int Ns, double alpha,
                     double beta, double box, int pin_index, const double *pin, double tol)
{
    double v[4];
    violation_one(s, Ns, alpha, beta, box, pin_index, pin, v);
    if (!(v[0] <= tol && v[1] <= tol && v[2] <= tol && v[3] <= tol))
        return 0;
    return dual_gap(s, q1, q2, Ns, alpha, beta) <= tol;
}

/* Dual FISTA for one shot.  Returns the iterations run; *conv is set to 1 when
 * tol > 0 and the violation test passed (always 1 in fixed-iteration mode). */
static int project_one(const double *k, double *s, int Ns, double alpha, double beta, double box,
                       int pin_index, const double *pin, int n_iter, double tol, double margin,
                       int check_every, int *conv)
{
    int n1 = Ns > 1 ? Ns - 1 : 0, n2 = Ns > 2 ? Ns - 2 : 0;
    double *q1 = (double *)calloc((size_t)(3 * n1 + 3), sizeof(double));
    double *q2 = (double *)calloc((size_t)(3 * n2 + 3), sizeof(double));
    double *y1 = (double *)calloc((size_t)(3 * n1 + 3), sizeof(double));
    double *y2 = (double *)calloc((size_t)(3 * n2 + 3), sizeof(double));
    const double tau = 1.0 / 20.0;
    /* Converged mode aims at the shrunk set so that the final iterate can be
     * strictly inside the requested one. */
    double a_eff = tol > 0.0 ? alpha * (1.0 - margin) : alpha;
    double b_eff = tol > 0.0 ? beta * (1.0 - margin) : beta;
    double t = 1.0;
    int it = 0;
    *conv = tol > 0.0 ? 0 : 1;
    for (it = 0; it < n_iter; ++it) {
        primal(k, y1, y2, Ns, box, pin_index, pin, s);
        double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double mom = (t - 1.0) / tn;
        for (int n = 0; n < n1; ++n) {
            double z[3], qn[3];
            for (int c = 0; c < 3; ++c)
                z[c] = y1[3 * n + c] + tau * (s[3 * (n + 1) + c] - s[3 * n + c]);
            shrink(z, tau * a_eff, qn);
            for (int c = 0; c < 3; ++c) {
                y1[3 * n + c] = qn[c] + mom * (qn[c] - q1[3 * n + c]);
                q1[3 * n + c] = qn[c];
            }
        }
        for (int n = 0; n < n2; ++n) {
            double z[3], qn[3];
            for (int c = 0; c < 3; ++c)
                z[c] = y2[3 * n + c] +
                       tau * (s[3 * (n + 2) + c] - 2.0 * s[3 * (n + 1) + c] + s[3 * n + c]);
            shrink(z, tau * b_eff, qn);
            for (int c = 0; c < 3; ++c) {
                y2[3 * n + c] = qn[c] + mom * (qn[c] - q2[3 * n + c]);
                q2[3 * n + c] = qn[c];
            }
        }
        t = tn;
        if (tol > 0.0 && check_every > 0 && (it + 1) % check_every == 0) {
            primal(k, q1, q2, Ns, box, pin_index, pin, s);
            if (certified(s, q1, q2, Ns, a_eff, b_eff, box, pin_index, pin, tol)) {
                *conv = 1;
                ++it;
                break;
            }
        }
    }
    primal(k, q1, q2, Ns, box, pin_index, pin, s);
    if (tol > 0.0 && !*conv)
        *conv = certified(s, q1, q2, Ns, a_eff, b_eff, box, pin_index, pin, tol);
    free(q1); free(q2); free(y1); free(y2);
    return it;
}

/*
 * Project Nc shots of Ns samples (Kin, Kout: [Nc*Ns][3], may alias).
 * alpha/beta may be +inf (constraint off).  pin_index < 0: no pin.
 * tol <= 0: exactly n_iter iterations.  tol > 0: aim at the set shrunk by
 * (1 - margin) and stop at the first check (every check_every iterations)
 * where every violation of that set and the duality gap are <= tol; returns
 * ORACLE_ENOTCONV if a shot did not get there within n_iter.  iters_out (optional, [Nc]) receives the iterations run.
 */
int oracle_project(const double *Kin, double *Kout, int64_t Nc, int64_t Ns, double alpha,
                   double beta, double box, int64_t pin_index, const double *pin, int64_t n_iter,
                   double tol, double margin, int64_t check_every, int64_t *iters_out)
{
    if (!Kin || !Kout || Nc < 0 || Ns < 1 || !(alpha > 0) || !(beta > 0) || !(box > 0) ||
        n_iter < 0 || (pin_index >= 0 && !pin))
        return ORACLE_EINVAL;
    int notconv = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : notconv)
    for (int64_t c = 0; c < Nc; ++c) {
        double *k = (double *)malloc(sizeof(double) * (size_t)(3 * Ns));
        memcpy(k, Kin + 3 * c * Ns, sizeof(double) * (size_t)(3 * Ns));
        int conv = 1;
        int it = project_one(k, Kout + 3 * c * Ns, (int)Ns, alpha, beta, box, (int)pin_index, pin,
                             (int)n_iter, tol, margin, (int)check_every, &conv);
        if (iters_out) iters_out[c] = it;
        if (!conv) notconv = 1;
        free(k);
    }
    return notconv ? ORACLE_ENOTCONV : ORACLE_OK;
}

/* Largest violation over all shots (same four entries as violation_one). */
int oracle_violation(const double *K, int64_t Nc, int64_t Ns, double alpha, double beta,
                     double box, int64_t pin_index, const double *pin, double out[4])
{
    if (!K || Nc < 0 || Ns < 1 || (pin_index >= 0 && !pin))
        return ORACLE_EINVAL;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    for (int64_t c = 0; c < Nc; ++c) {
        double v[4];
        violation_one(K + 3 * c * Ns, (int)Ns, alpha, beta, box, (int)pin_index, pin, v);
        for (int e = 0; e < 4; ++e)
            if (v[e] > out[e]) out[e] = v[e];
    }
    return ORACLE_OK;
}

/* One projected-gradient step (eq. proj_grad_descent with the scaled gradient
 * G = N dF/dK): K <- Pi(K - eta G), in place, K is [Nc*Ns][3]. */
int oracle_step(double *K, int64_t Nc, int64_t Ns, const double *rho, int64_t nx, int64_t ny,
                int64_t nz, double lo, double hi, double eta, double alpha, double beta, double box,
                int64_t pin_index, const double *pin, int64_t n_iter, double eps)
{
    int64_t N = Nc * Ns;
    double *G = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    if (!G) return ORACLE_EINVAL;
    int st = oracle_forces(K, N, rho, nx, ny, nz, lo, hi, NULL, N, NULL, NULL, G, NULL, NULL, eps);
    if (st == ORACLE_OK) {
        for (int64_t m = 0; m < 3 * N; ++m)
            G[m] = K[m] - eta * G[m];
        st = oracle_project(G, K, Nc, Ns, alpha, beta, box, pin_index, pin, n_iter, 0.0, 0.0, 0,
                            NULL);
    }
    free(G);
    return st;
}

/* ---------------------------------------------------------------------- */
/* Multi-resolution driver (Algorithm 1, Secs. II-C "choice of step size",  */
/* II-E "multi-resolution strategy" and "overall algorithm").               */

/* The linear interpolator L_{2d}: a shot of d samples (time 2n on the fine
 * raster) becomes 2d samples at times m = 0 .. 2d-1: even samples are the
 * coarse ones, odd samples the midpoints of consecutive coarse samples, and
 * the last one continues the last coarse segment (linear extrapolation).
 * A one-sample shot is repeated.  Kc [Nc][d][3] -> Kf [Nc][2d][3]. */
int oracle_upsample(const double *Kc, int64_t Nc, int64_t d, double *Kf)
{
    if (!Kc || !Kf || Nc < 0 || d < 1)
        return ORACLE_EINVAL;
    for (int64_t s = 0; s < Nc; ++s) {
        const double *c = Kc + 3 * d * s;
        double *f = Kf + 6 * d * s;
        for (int64_t n = 0; n < d; ++n)
            for (int a = 0; a < 3; ++a) {
                double here = c[3 * n + a];
                double next;
                if (n + 1 < d)
                    next = 0.5 * (here + c[3 * (n + 1) + a]);
                else if (d > 1)
                    next = here + 0.5 * (here - c[3 * (n - 1) + a]);
                else
                    next = here;
                f[6 * n + a] = here;
                f[6 * n + 3 + a] = next;
            }
    }
    return ORACLE_OK;
}

/* n_git projected-gradient iterations at one resolution (the inner loop of
 * Algorithm 1, eq. proj_grad_descent): K <- Pi(K - eta_t G(K)) with the
 * fixed step eta for the first n_fixed iterations and the Barzilai-Borwein
 * step eta_t = <s, s> / <s, y> afterwards, s = K_t - K_{t-1} and
 * y = G(K_t) - G(K_{t-1}) (G = N dF/dK, so eta stays in G units).  When
 * <s, y> <= 0 the previous step is kept; every BB step is clamped to
 * [eta_min, eta_max].  trace[t] (optional) receives the step of iteration t.
 * K [Nc*Ns][3] is updated in place. */
int oracle_optimize(double *K, int64_t Nc, int64_t Ns, const double *rho, int64_t nx, int64_t ny,
                    int64_t nz, double lo, double hi, double alpha, double beta, double box,
                    int64_t pin_index, const double *pin, int64_t n_pit, int64_t n_git,
                    int64_t n_fixed, double eta, double eta_min, double eta_max, double eps,
                    double *trace)
{
    const int64_t N = Nc * Ns;
    if (!K || Nc < 1 || Ns < 1 || N < 2 || n_git < 0 || n_fixed < 0 || !(eta_min > 0) ||
        !(eta_max >= eta_min))
        return ORACLE_EINVAL;
    double *G = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    double *Kp = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    double *Gp = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    double *half = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    int st = (G && Kp && Gp && half) ? ORACLE_OK : ORACLE_EINVAL;
    double step = eta;
    for (int64_t t = 0; t < n_git && st == ORACLE_OK; ++t) {
        st = oracle_forces(K, N, rho, nx, ny, nz, lo, hi, NULL, N, NULL, NULL, G, NULL, NULL, eps);
        if (st != ORACLE_OK)
            break;
        if (t < n_fixed) {
            step = eta;
        } else if (t > 0) {
            double ss = 0.0, sy = 0.0;
            for (int64_t m = 0; m < 3 * N; ++m) {
                double s = K[m] - Kp[m], y = G[m] - Gp[m];
                ss += s * s;
                sy += s * y;
            }
            if (sy > 0.0 && isfinite(ss / sy)) {
                step = ss / sy;
                if (step < eta_min) step = eta_min;
                if (step > eta_max) step = eta_max;
            }
        }
        if (trace)
            trace[t] = step;
        for (int64_t m = 0; m < 3 * N; ++m) {
            Kp[m] = K[m];
            Gp[m] = G[m];
            half[m] = K[m] - step * G[m];
        }
        st = oracle_project(half, K, Nc, Ns, alpha, beta, box, pin_index, pin, n_pit, 0.0, 0.0, 0,
                            NULL);
    }
    free(G); free(Kp); free(Gp); free(half);
    return st;
}

/* Algorithm 1: levels l = start_level .. 0, level l with Ns / 2^l samples
 * per shot, per-step constraints alpha * alpha_factor^l and
 * beta * beta_factor^l, the pinned sample pin_index / 2^l (floor), n_git
 * iterations of oracle_optimize, then L_{2d} up to the next level.  K holds
 * Nc * (Ns >> start_level) samples on entry and Nc * Ns on exit (its buffer
 * is sized for Nc * Ns).  levels_out (optional) receives the result of
 * every level before up-sampling, level after level; trace (optional) the
 * steps, n_git per level. */
int oracle_multires(double *K, int64_t Nc, int64_t Ns, const double *rho, int64_t nx, int64_t ny,
                    int64_t nz, double lo, double hi, double alpha, double beta, double box,
                    int64_t pin_index, const double *pin, int64_t n_pit, int64_t start_level,
                    int64_t n_git, int64_t n_fixed, double eta, double eta_min, double eta_max,
                    double alpha_factor, double beta_factor, double eps, double *levels_out,
                    double *trace)
{
    if (!K || Nc < 1 || start_level < 0 || start_level > 30 || (Ns % ((int64_t)1 << start_level)))
        return ORACLE_EINVAL;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(3 * Nc * Ns));
    if (!tmp)
        return ORACLE_EINVAL;
    int st = ORACLE_OK;
    for (int64_t l = start_level; l >= 0 && st == ORACLE_OK; --l) {
        const int64_t Nsl = Ns >> l;
        const double al = alpha * pow(alpha_factor, (double)l);
        const double bl = beta * pow(beta_factor, (double)l);
        const int64_t pl = pin_index >= 0 ? pin_index >> l : -1;
        st = oracle_optimize(K, Nc, Nsl, rho, nx, ny, nz, lo, hi, al, bl, box, pl, pin, n_pit,
                             n_git, n_fixed, eta, eta_min, eta_max, eps, trace);
        if (st != ORACLE_OK)
            break;
        if (levels_out) {
            memcpy(levels_out, K, sizeof(double) * (size_t)(3 * Nc * Nsl));
            levels_out += 3 * Nc * Nsl;
        }
        if (trace)
            trace += n_git;
        if (l > 0) {
            st = oracle_upsample(K, Nc, Nsl, tmp);
            memcpy(K, tmp, sizeof(double) * (size_t)(6 * Nc * Nsl));
        }
    }
    free(tmp);
    return st;
}

/* ---------------------------------------------------------------------- */
/* Split of the repulsion for a fast (particle-mesh) summation.             */

/* The repulsion kernel d / |d|_eps = d / r (r = sqrt(|d|^2 + eps^2)) splits
 * exactly into a short-range part d / r * erfc(r / sigma), which decays like
 * a Gaussian, and a smooth long-range part d / r * erf(r / sigma) (the
 * gradient of r erf(r/sigma) + sigma/sqrt(pi) exp(-r^2/sigma^2)).  For M
 * targets (indices into K, or 0..N-1 when targets is NULL) this returns the
 * directed sums over j != i of
 *   S: the short-range part, only for pairs with |d| < rc (rc <= 0: all);
 *   L: the long-range part (all pairs);
 * and the matching energy sums eS (short: r erfc(r/sigma) -
 * sigma/sqrt(pi) exp(-r^2/sigma^2), only |d| < rc) and eL (the long-range
 * potential) -- none scaled by 1/N.  S + L (rc <= 0) is the repulsion sum
 * and eS + eL the distance sum of oracle_forces.  Any output may be NULL. */
int oracle_repulsion_split(const double *K, int64_t N, double sigma, double rc, double eps,
                           const int64_t *targets, int64_t M, double *S, double *L, double *eS,
                           double *eL)
{
    if (!K || N < 1 || !(sigma > 0) || M < 0 || !(eps >= 0.0))
        return ORACLE_EINVAL;
    const double spi = sigma / sqrt(3.14159265358979323846);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t m = 0; m < M; ++m) {
        int64_t i = targets ? targets[m] : m;
        if (i < 0 || i >= N) {
            bad = 1;
            continue;
        }
        double s[3] = {0, 0, 0}, l[3] = {0, 0, 0}, es = 0.0, el = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i)
                continue;
            double d[3] = {K[3 * i] - K[3 * j], K[3 * i + 1] - K[3 * j + 1],
                           K[3 * i + 2] - K[3 * j + 2]};
            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double r = sqrt(d2 + eps * eps);
            if (r == 0.0)
                continue;
            double x = r / sigma;
            double gauss = spi * exp(-x * x);
            double wl = erf(x) / r, ws = erfc(x) / r;
            for (int c = 0; c < 3; ++c)
                l[c] += d[c] * wl;
            el += r * erf(x) + gauss;
            if (rc <= 0.0 || sqrt(d2) < rc) {
                for (int c = 0; c < 3; ++c)
                    s[c] += d[c] * ws;
                es += r * erfc(x) - gauss;
            }
        }
        for (int c = 0; c < 3; ++c) {
            if (S) S[3 * m + c] = s[c];
            if (L) L[3 * m + c] = l[c];
        }
        if (eS) eS[m] = es;
        if (eL) eL[m] = el;
    }
    return bad ? ORACLE_EINVAL : ORACLE_OK;
}
