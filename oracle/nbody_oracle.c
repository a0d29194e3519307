/*
 * nbody_oracle.c -- plain FP64 CPU reference ("oracle") for the all-pairs
 * N-body force evaluation of Elsen, Vishal, Houston, Pande, Hanrahan, Darve,
 * "N-Body Simulations on GPUs" (arXiv 0706.3060).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the timed CPU
 * baseline of the benchmark may load this code. It shares nothing with the
 * CUDA library: no header, no helper, no constant table.
 *
 * Every function is the textbook definition written out in double precision,
 * with no blocking, fusion or reordering:
 *   - oracle_grav       Eq. 1 of Sec. 3.3 / Table 1 "Gravity (accel)"
 *   - oracle_ljc        Table 1 "LJC (constant)" (readings C1, C2, C4 below)
 *   - oracle_grav_jerk  Table 1 "Gravity (accel & jerk)"
 *   - oracle_ljc_model  Table 1 "LJC (linear)" as well (reading C3 below)
 *   - oracle_grav_vjp   transpose of the Jacobian of Eq. 1, block by block
 *   - oracle_grav_vjp_rows  selected rows of the same product, gathered per row
 *   - oracle_ljc_vjp    transpose of the Jacobian of the LJC law, plus the
 *                       derivatives w.r.t. per-type sigma, epsilon and masses
 *
 * Readings of the paper used here (the paper is silent or garbled on these):
 *   C1  Table 1 prints the Lennard-Jones term as a bare scalar
 *       eps_ij[(sigma/r)^6 - (sigma/r)^12]; we use the standard 12-6
 *       potential 4 eps_ij[(sigma/r)^12 - (sigma/r)^6] and its force
 *       (24 eps_ij / r^2)[2 (sigma/r)^12 - (sigma/r)^6] r_ij.
 *   C2  Coulomb in a continuum solvent of constant dielectric eps_r:
 *       force k_e q_i q_j r_ij / (eps_r r^3); the caller passes
 *       ke_over_epsr = k_e / eps_r.
 *   C3  "LJC(linear)" prints q_i q_j r_ij / r^4 without the factor 2 of
 *       -grad(1/r^2); we use the energy kq q_i q_j / r^2 (dielectric D r,
 *       kq = k_e / D) and its force 2 kq q_i q_j r_ij / r^4.
 *   C4  Lorentz-Berthelot mixing: sigma_ij = (sigma_i + sigma_j)/2,
 *       eps_ij = sqrt(eps_i eps_j).
 *   C5  The self pair i == j is excluded by its index, as the Appendix
 *       listing does with an index comparison.
 *   C6  r_ij = x_i - x_j; Eq. 1 carries the leading minus (attraction);
 *       the Appendix's "eps" is the squared softening eps^2.
 *
 * All arrays are row-major: x is n x 3, forces n x 3.
 * Built with -O2 -fopenmp -ffp-contract=off so that results do not depend on
 * whether the host compiler fuses multiply-adds.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int oracle_version(void) { return 1; }

/* Thread count of the OpenMP loops below (n < 1: leave it unchanged); returns
 * the count now in force. The force sums do not depend on it (each target's
 * sum runs in index order inside one thread); the VJPs' array reductions add
 * per-thread partial sums, so their last bits do. */
int oracle_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

/* ---------------------------------------------------------------------------
 * Softened gravity, Eq. 1:
 *   a_i   = -G sum_{j != i} m_j r_ij / (|r_ij|^2 + eps^2)^{3/2}
 *   phi_i = -G sum_{j != i} m_j / (|r_ij|^2 + eps^2)^{1/2}
 * (phi is the potential whose negative gradient is a; U = 1/2 sum m_i phi_i.)
 * idx (length ni) selects the target particles; idx == NULL means all n.
 * phi may be NULL.
 * ------------------------------------------------------------------------- */
void oracle_grav(int64_t n, const double *x, const double *m, double G,
                 double eps2, int64_t ni, const int64_t *idx, double *acc,
                 double *phi)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < ni; ++k) {
        int64_t i = idx ? idx[k] : k;
        double ax = 0.0, ay = 0.0, az = 0.0, p = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double rx = x[3 * i + 0] - x[3 * j + 0];
            double ry = x[3 * i + 1] - x[3 * j + 1];
            double rz = x[3 * i + 2] - x[3 * j + 2];
            double s2 = rx * rx + ry * ry + rz * rz + eps2;
            double s = sqrt(s2);
            double s3 = s2 * s;
            ax -= m[j] * rx / s3;
            ay -= m[j] * ry / s3;
            az -= m[j] * rz / s3;
            p -= m[j] / s;
        }
        acc[3 * k + 0] = G * ax;
        acc[3 * k + 1] = G * ay;
        acc[3 * k + 2] = G * az;
        if (phi)
            phi[k] = G * p;
    }
}

/* ---------------------------------------------------------------------------
 * Softened gravity with jerk, Table 1 "Gravity (accel & jerk)". With
 * r = x_j - x_i, u = v_j - v_i and s^2 = |r|^2 + eps^2:
 *   a_i = G sum_{j != i} m_j r / s^3
 *   j_i = G sum_{j != i} m_j [ u / s^3 - 3 (r . u) r / s^5 ]   (= d a_i / dt)
 * ------------------------------------------------------------------------- */
void oracle_grav_jerk(int64_t n, const double *x, const double *v, const double *m, double G,
                      double eps2, int64_t ni, const int64_t *idx, double *acc, double *jerk)
{
    /* idx (length ni) selects the targets; idx == NULL means all n (ni = n) */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < ni; ++k) {
        const int64_t i = idx ? idx[k] : k;
        double a[3] = {0.0, 0.0, 0.0}, jk[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double r[3], u[3];
            for (int c = 0; c < 3; ++c) {
                r[c] = x[3 * j + c] - x[3 * i + c];
                u[c] = v[3 * j + c] - v[3 * i + c];
            }
            double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
            double s = sqrt(s2);
            double s3 = s2 * s, s5 = s3 * s2;
            double ru = r[0] * u[0] + r[1] * u[1] + r[2] * u[2];
            for (int c = 0; c < 3; ++c) {
                a[c] += m[j] * r[c] / s3;
                jk[c] += m[j] * (u[c] / s3 - 3.0 * ru * r[c] / s5);
            }
        }
        for (int c = 0; c < 3; ++c) {
            acc[3 * k + c] = G * a[c];
            jerk[3 * k + c] = G * jk[c];
        }
    }
}

void oracle_ljc_model(int64_t n, const double *x, const double *q, const double *sig,
                      const double *eps, double kq, int model, int64_t ni,
                      const int64_t *idx, double *force, double *phi);

/* ---------------------------------------------------------------------------
 * Lennard-Jones + Coulomb with a constant dielectric, Table 1 "LJC(constant)"
 * with readings C1, C2, C4, C5:
 *   F_i   = sum_{j != i} [ kq q_i q_j / r^3
 *                          + 24 eps_ij / r^2 (2 (s_ij/r)^12 - (s_ij/r)^6) ] r_ij
 *   phi_i = sum_{j != i} [ kq q_i q_j / r + 4 eps_ij ((s_ij/r)^12 - (s_ij/r)^6) ]
 * with kq = k_e / eps_r, s_ij = (sig_i + sig_j)/2, eps_ij = sqrt(eps_i eps_j).
 * F is a force (the acceleration is F_i / m_i); U = 1/2 sum_i phi_i.
 * ------------------------------------------------------------------------- */
void oracle_ljc(int64_t n, const double *x, const double *q, const double *sig,
                const double *eps, double kq, int64_t ni, const int64_t *idx,
                double *force, double *phi)
{
    oracle_ljc_model(n, x, q, sig, eps, kq, 0, ni, idx, force, phi);
}

/* ---------------------------------------------------------------------------
 * LJC with a dielectric model: model 0 is the constant dielectric above; model 1
 * is Table 1 "LJC(linear)", a dielectric growing linearly with distance,
 * eps(r) = D r (reading C3: the Coulomb energy is kq q_i q_j / r^2 with
 * kq = k_e / D, so its force is 2 kq q_i q_j r_ij / r^4).
 * ------------------------------------------------------------------------- */
void oracle_ljc_model(int64_t n, const double *x, const double *q, const double *sig,
                      const double *eps, double kq, int model, int64_t ni,
                      const int64_t *idx, double *force, double *phi)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < ni; ++k) {
        int64_t i = idx ? idx[k] : k;
        double fx = 0.0, fy = 0.0, fz = 0.0, p = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double rx = x[3 * i + 0] - x[3 * j + 0];
            double ry = x[3 * i + 1] - x[3 * j + 1];
            double rz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = rx * rx + ry * ry + rz * rz;
            double r = sqrt(r2);
            double sij = 0.5 * (sig[i] + sig[j]);
            double eij = sqrt(eps[i] * eps[j]);
            double sr6 = pow(sij / r, 6.0);
            double sr12 = sr6 * sr6;
            double fc = model == 1 ? 2.0 * kq * q[i] * q[j] / (r2 * r2)
                                   : kq * q[i] * q[j] / (r2 * r);
            double flj = 24.0 * eij * (2.0 * sr12 - sr6) / r2;
            double f = fc + flj;
            fx += f * rx;
            fy += f * ry;
            fz += f * rz;
            p += (model == 1 ? kq * q[i] * q[j] / r2 : kq * q[i] * q[j] / r)
                 + 4.0 * eij * (sr12 - sr6);
        }
        force[3 * k + 0] = fx;
        force[3 * k + 1] = fy;
        force[3 * k + 2] = fz;
        if (phi)
            phi[k] = p;
    }
}

/* ---------------------------------------------------------------------------
 * Vector-Jacobian product of Eq. 1, written out block by block.
 * For every ordered pair (i, j != i) with r = x_i - x_j, s^2 = |r|^2 + eps^2:
 *   d a_i / d x_j = G m_j T(r),   d a_i / d x_i (from j) = -G m_j T(r),
 *   T(r) = I / s^3 - 3 r r^T / s^5   (symmetric),
 *   d a_i / d m_j = -G r / s^3.
 * Outputs  g_k  = sum_i (d a_i / d x_k)^T lam_i      (n x 3)
 *          gm_k = sum_i lam_i . d a_i / d m_k        (n), may be NULL.
 * The loop scatters each block into the rows it touches; OpenMP array
 * reductions keep it a plain sum.
 * ------------------------------------------------------------------------- */
void oracle_grav_vjp(int64_t n, const double *x, const double *m, double G,
                     double eps2, const double *lam, double *g, double *gm)
{
    double *gl = (double *)calloc((size_t)(3 * n), sizeof(double));
    double *ml = (double *)calloc((size_t)n, sizeof(double));
#pragma omp parallel for schedule(static) reduction(+ : gl[:3 * n], ml[:n])
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            double r[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1],
                           x[3 * i + 2] - x[3 * j + 2]};
            double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
            double s = sqrt(s2);
            double s3 = s2 * s, s5 = s3 * s2;
            double T[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    T[a][b] = (a == b ? 1.0 / s3 : 0.0) - 3.0 * r[a] * r[b] / s5;
            for (int a = 0; a < 3; ++a) {
                double Tl = 0.0;
                for (int b = 0; b < 3; ++b)
                    Tl += T[b][a] * lam[3 * i + b];
                gl[3 * j + a] += G * m[j] * Tl;  /* block (i, j)   */
                gl[3 * i + a] -= G * m[j] * Tl;  /* block (i, i)   */
            }
            double dm = 0.0;
            for (int a = 0; a < 3; ++a)
                dm += lam[3 * i + a] * (-G * r[a] / s3);
            ml[j] += dm;
        }
    }
    memcpy(g, gl, sizeof(double) * (size_t)(3 * n));
    if (gm)
        memcpy(gm, ml, sizeof(double) * (size_t)n);
    free(gl);
    free(ml);
}

/* ---------------------------------------------------------------------------
 * Rows idx[0..nk) of the same product, each gathered on its own instead of
 * scattered: row k collects the blocks (i, k) and (k, k) of the sum above,
 *   g_k  = sum_{i != k} G m_k T(x_i - x_k) lam_i - sum_{j != k} G m_j T(x_k - x_j) lam_k,
 *   gm_k = sum_{i != k} lam_i . (-G (x_i - x_k) / s_ik^3),
 * with T(r) = I / s^3 - 3 r r^T / s^5 (even in r). Outputs g (nk x 3), gm (nk).
 * ------------------------------------------------------------------------- */
void oracle_grav_vjp_rows(int64_t n, const double *x, const double *m, double G,
                          double eps2, const double *lam, int64_t nk, const int64_t *idx,
                          double *g, double *gm)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < nk; ++q) {
        const int64_t k = idx[q];
        double acc[3] = {0.0, 0.0, 0.0}, dm = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (i == k)
                continue;
            double r[3] = {x[3 * i] - x[3 * k], x[3 * i + 1] - x[3 * k + 1],
                           x[3 * i + 2] - x[3 * k + 2]};
            double s2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + eps2;
            double s = sqrt(s2);
            double s3 = s2 * s, s5 = s3 * s2;
            for (int a = 0; a < 3; ++a) {
                double Ti = 0.0, Tk = 0.0;  /* (T lam_i)_a and (T lam_k)_a */
                for (int b = 0; b < 3; ++b) {
                    double T = (a == b ? 1.0 / s3 : 0.0) - 3.0 * r[a] * r[b] / s5;
                    Ti += T * lam[3 * i + b];
                    Tk += T * lam[3 * k + b];
                }
                acc[a] += G * m[k] * Ti - G * m[i] * Tk;
            }
            for (int a = 0; a < 3; ++a)
                dm += lam[3 * i + a] * (-G * r[a] / s3);
        }
        for (int a = 0; a < 3; ++a)
            g[3 * q + a] = acc[a];
        if (gm)
            gm[q] = dm;
    }
}

/* ---------------------------------------------------------------------------
 * Vector-Jacobian product of the LJC(constant) acceleration a_i = F_i / m_i,
 * with F_i = sum_{j != i} phi(rho_ij) r_ij, rho = |r|^2, and
 *   phi(rho)  = kq q_i q_j rho^{-3/2} + 24 eps_ij (2 s^12 rho^{-7} - s^6 rho^{-4})
 *   phi'(rho) = -3/2 kq q_i q_j rho^{-5/2}
 *               + 24 eps_ij (-14 s^12 rho^{-8} + 4 s^6 rho^{-5}).
 * d F_i / d x_i (from j) = H,  d F_i / d x_j = -H,  H = phi I + 2 phi' r r^T.
 * Parameters are per type: sig_i = sig_t[type_i], eps_i = eps_t[type_i].
 *   d s_ij   / d sig_t = ([t_i = t] + [t_j = t]) / 2
 *   d eps_ij / d eps_t = ([t_i = t] eps_{t_j} + [t_j = t] eps_{t_i}) / (2 eps_ij)
 *   d phi / d s_ij     = 24 eps_ij (24 s^11 rho^{-7} - 6 s^5 rho^{-4})
 *   d phi / d eps_ij   = 24 (2 s^12 rho^{-7} - s^6 rho^{-4})
 *   d a_i / d m_i      = -F_i / m_i^2
 * Outputs: g (n x 3), gm (n, may be NULL), gsig and geps (ntypes, may be NULL).
 * ------------------------------------------------------------------------- */
/* model 0: constant dielectric (force coefficient kq q_i q_j / rho^{3/2});
 * model 1: linear dielectric, reading C3 (2 kq q_i q_j / rho^2). rho = r^2. */
void oracle_ljc_vjp_model(int64_t n, const double *x, const double *m,
                          const double *q, const int32_t *type, int32_t ntypes,
                          const double *sig_t, const double *eps_t, double kq, int model,
                          const double *lam, double *g, double *gm, double *gsig,
                          double *geps)
{
    double *gl = (double *)calloc((size_t)(3 * n), sizeof(double));
    double *ml = (double *)calloc((size_t)n, sizeof(double));
    double *sl = (double *)calloc((size_t)ntypes, sizeof(double));
    double *el = (double *)calloc((size_t)ntypes, sizeof(double));
#pragma omp parallel for schedule(static) \
    reduction(+ : gl[:3 * n], ml[:n], sl[:ntypes], el[:ntypes])
    for (int64_t i = 0; i < n; ++i) {
        double Fi[3] = {0.0, 0.0, 0.0};
        double u[3] = {lam[3 * i] / m[i], lam[3 * i + 1] / m[i],
                       lam[3 * i + 2] / m[i]};
        int32_t ti = type[i];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            int32_t tj = type[j];
            double r[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1],
                           x[3 * i + 2] - x[3 * j + 2]};
            double rho = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            double s = 0.5 * (sig_t[ti] + sig_t[tj]);
            double e = sqrt(eps_t[ti] * eps_t[tj]);
            double qq = kq * q[i] * q[j];
            double s6 = pow(s, 6.0), s12 = s6 * s6;
            /* Coulomb part of the force coefficient and of its rho-derivative */
            double phi_c = model ? 2.0 * qq * pow(rho, -2.0) : qq * pow(rho, -1.5);
            double dphi_c = model ? -4.0 * qq * pow(rho, -3.0) : -1.5 * qq * pow(rho, -2.5);
            double phi = phi_c
                       + 24.0 * e * (2.0 * s12 * pow(rho, -7.0) - s6 * pow(rho, -4.0));
            double dphi = dphi_c
                        + 24.0 * e * (-14.0 * s12 * pow(rho, -8.0) + 4.0 * s6 * pow(rho, -5.0));
            double H[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    H[a][b] = (a == b ? phi : 0.0) + 2.0 * dphi * r[a] * r[b];
            for (int a = 0; a < 3; ++a) {
                double Hu = 0.0;
                for (int b = 0; b < 3; ++b)
                    Hu += H[b][a] * u[b];
                gl[3 * i + a] += Hu;  /* block (i, i) */
                gl[3 * j + a] -= Hu;  /* block (i, j) */
                Fi[a] += phi * r[a];
            }
            double ur = u[0] * r[0] + u[1] * r[1] + u[2] * r[2];
            double dphi_ds = 24.0 * e * (24.0 * pow(s, 11.0) * pow(rho, -7.0)
                                         - 6.0 * pow(s, 5.0) * pow(rho, -4.0));
            double dphi_de = 24.0 * (2.0 * s12 * pow(rho, -7.0) - s6 * pow(rho, -4.0));
            /* d s_ij / d sig_t and d eps_ij / d eps_t, one type at a time */
            sl[ti] += ur * dphi_ds * 0.5;
            sl[tj] += ur * dphi_ds * 0.5;
            el[ti] += ur * dphi_de * eps_t[tj] / (2.0 * e);
            el[tj] += ur * dphi_de * eps_t[ti] / (2.0 * e);
        }
        ml[i] += -(lam[3 * i] * Fi[0] + lam[3 * i + 1] * Fi[1] + lam[3 * i + 2] * Fi[2])
                 / (m[i] * m[i]);
    }
    memcpy(g, gl, sizeof(double) * (size_t)(3 * n));
    if (gm)
        memcpy(gm, ml, sizeof(double) * (size_t)n);
    if (gsig)
        memcpy(gsig, sl, sizeof(double) * (size_t)ntypes);
    if (geps)
        memcpy(geps, el, sizeof(double) * (size_t)ntypes);
    free(gl);
    free(ml);
    free(sl);
    free(el);
}

void oracle_ljc_vjp(int64_t n, const double *x, const double *m,
                    const double *q, const int32_t *type, int32_t ntypes,
                    const double *sig_t, const double *eps_t, double kq,
                    const double *lam, double *g, double *gm, double *gsig,
                    double *geps)
{
    oracle_ljc_vjp_model(n, x, m, q, type, ntypes, sig_t, eps_t, kq, 0, lam, g, gm, gsig,
                         geps);
}
