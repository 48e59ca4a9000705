/*
 * Plain FP64 CPU oracle for the direct O(N^2) softened N-body sum.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm may load this code.  It shares nothing with the
 * CUDA library (no headers, no helpers, no constants) and is written to be
 * checked against the paper by eye: one i at a time, j in increasing order,
 * every quantity formed exactly as its definition reads.  The only speed
 * concession is an OpenMP loop over independent i.
 *
 * Definitions (Sect. 2, Eq. 1 with the attractive sign; Sect. 3: acceleration,
 * its time derivative "jerk" and the potential by direct summation; Sect. 3.3.1:
 * Plummer softening eps):
 *   d_ij = x_j - x_i,  w_ij = v_j - v_i,  s_ij^2 = |d_ij|^2 + eps^2
 *   a_i    =  G sum_{j != i} m_j d_ij / s^3
 *   jerk_i =  G sum_{j != i} m_j [ w_ij / s^3 - 3 (d_ij . w_ij) d_ij / s^5 ]
 *   phi_i  = -G sum_{j != i} m_j / s
 * Zero softening (Sect. 3.3.1): a pair with s^2 == 0 contributes nothing, and
 * s^2 is raised to r_min^2 when it is smaller (r_min = 0 disables the guard).
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* x, v: n_j x 3 row-major.  i_idx[k] is the index (into the j set) of the k-th
 * i-particle; the pair j == i_idx[k] is left out.  acc, jerk: n_i x 3; pot: n_i. */
void oracle_acc_jerk_pot(int64_t n_i, const int64_t *i_idx, int64_t n_j,
                         const double *m, const double *x, const double *v,
                         double eps, double r_min, double G,
                         double *acc, double *jerk, double *pot)
{
    const double eps2 = eps * eps;
    const double rmin2 = r_min * r_min;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < n_i; ++k) {
        const int64_t i = i_idx[k];
        double ax = 0, ay = 0, az = 0, jx = 0, jy = 0, jz = 0, p = 0;
        for (int64_t j = 0; j < n_j; ++j) {
            if (j == i)
                continue;
            const double dx = x[3 * j + 0] - x[3 * i + 0];
            const double dy = x[3 * j + 1] - x[3 * i + 1];
            const double dz = x[3 * j + 2] - x[3 * i + 2];
            const double wx = v[3 * j + 0] - v[3 * i + 0];
            const double wy = v[3 * j + 1] - v[3 * i + 1];
            const double wz = v[3 * j + 2] - v[3 * i + 2];
            double s2 = dx * dx + dy * dy + dz * dz + eps2;
            if (s2 == 0.0)
                continue;
            if (s2 < rmin2)
                s2 = rmin2;
            const double s = sqrt(s2);
            const double s3 = s2 * s;
            const double s5 = s3 * s2;
            const double dw = dx * wx + dy * wy + dz * wz;
            ax += m[j] * dx / s3;
            ay += m[j] * dy / s3;
            az += m[j] * dz / s3;
            jx += m[j] * (wx / s3 - 3.0 * dw * dx / s5);
            jy += m[j] * (wy / s3 - 3.0 * dw * dy / s5);
            jz += m[j] * (wz / s3 - 3.0 * dw * dz / s5);
            p -= m[j] / s;
        }
        acc[3 * k + 0] = G * ax;
        acc[3 * k + 1] = G * ay;
        acc[3 * k + 2] = G * az;
        jerk[3 * k + 0] = G * jx;
        jerk[3 * k + 1] = G * jy;
        jerk[3 * k + 2] = G * jz;
        pot[k] = G * p;
    }
}

/* Acceleration and potential only (the leapfrog clients of Sect. 4.3 need no jerk). */
void oracle_acc_pot(int64_t n_i, const int64_t *i_idx, int64_t n_j,
                    const double *m, const double *x, double eps, double G,
                    double *acc, double *pot)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < n_i; ++k) {
        const int64_t i = i_idx[k];
        double ax = 0, ay = 0, az = 0, p = 0;
        for (int64_t j = 0; j < n_j; ++j) {
            if (j == i)
                continue;
            const double dx = x[3 * j + 0] - x[3 * i + 0];
            const double dy = x[3 * j + 1] - x[3 * i + 1];
            const double dz = x[3 * j + 2] - x[3 * i + 2];
            const double s2 = dx * dx + dy * dy + dz * dz + eps2;
            if (s2 == 0.0)
                continue;
            const double s = sqrt(s2);
            const double s3 = s2 * s;
            ax += m[j] * dx / s3;
            ay += m[j] * dy / s3;
            az += m[j] * dz / s3;
            p -= m[j] / s;
        }
        acc[3 * k + 0] = G * ax;
        acc[3 * k + 1] = G * ay;
        acc[3 * k + 2] = G * az;
        pot[k] = G * p;
    }
}

/* Total kinetic energy K = sum 1/2 m |v|^2 and potential energy
 * W = 1/2 sum_i m_i phi_i, with phi the softened potential above (the energy
 * of Eq. 2 is K + W). */
void oracle_energy(int64_t n, const double *m, const double *x, const double *v,
                   double eps, double G, double *kin, double *wpot)
{
    const double eps2 = eps * eps;
    double k_sum = 0.0;
    for (int64_t i = 0; i < n; ++i)
        k_sum += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                               v[3 * i + 2] * v[3 * i + 2]);
    double w_sum = 0.0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : w_sum)
    for (int64_t i = 0; i < n; ++i) {
        double p = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i)
                continue;
            const double dx = x[3 * j + 0] - x[3 * i + 0];
            const double dy = x[3 * j + 1] - x[3 * i + 1];
            const double dz = x[3 * j + 2] - x[3 * i + 2];
            const double s2 = dx * dx + dy * dy + dz * dz + eps2;
            if (s2 == 0.0)
                continue;
            p -= m[j] / sqrt(s2);
        }
        w_sum += 0.5 * m[i] * G * p;
    }
    *kin = k_sum;
    *wpot = w_sum;
}

/* Reverse-mode derivative of the softened accelerations.  Given g_i = dL/da_i
 * for every particle (all n are i-particles), returns
 *   dL/dx_k = G sum_{j != k} K(d_kj) (m_k g_j - m_j g_k),
 *             K(d) = I / s^3 - 3 d d^T / s^5,  d_kj = x_j - x_k
 *   dL/dm_k = G sum_{i != k} g_i . (x_k - x_i) / s_ik^3
 * which is the transpose of the Jacobian of a_i = G sum m_j d_ij / s^3 applied
 * to g (the paper has no adjoint; this is the chain rule written out). */
void oracle_force_adjoint(int64_t n, const double *m, const double *x, const double *g,
                          double eps, double G, double *gx, double *gm)
{
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < n; ++k) {
        double sx = 0, sy = 0, sz = 0, sm = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == k)
                continue;
            const double dx = x[3 * j + 0] - x[3 * k + 0];
            const double dy = x[3 * j + 1] - x[3 * k + 1];
            const double dz = x[3 * j + 2] - x[3 * k + 2];
            const double s2 = dx * dx + dy * dy + dz * dz + eps2;
            const double s = sqrt(s2);
            const double s3 = s2 * s;
            const double s5 = s3 * s2;
            const double wx = m[k] * g[3 * j + 0] - m[j] * g[3 * k + 0];
            const double wy = m[k] * g[3 * j + 1] - m[j] * g[3 * k + 1];
            const double wz = m[k] * g[3 * j + 2] - m[j] * g[3 * k + 2];
            const double dw = dx * wx + dy * wy + dz * wz;
            sx += wx / s3 - 3.0 * dx * dw / s5;
            sy += wy / s3 - 3.0 * dy * dw / s5;
            sz += wz / s3 - 3.0 * dz * dw / s5;
            /* x_k - x_j = -d */
            sm += -(g[3 * j + 0] * dx + g[3 * j + 1] * dy + g[3 * j + 2] * dz) / s3;
        }
        gx[3 * k + 0] = G * sx;
        gx[3 * k + 1] = G * sy;
        gx[3 * k + 2] = G * sz;
        gm[k] = G * sm;
    }
}

/* Nearest neighbour of each i (Sect. 3.3.1): the j != i with the smallest
 * |x_j - x_i|^2, the smallest such j on ties. */
void oracle_nearest(int64_t n_i, const int64_t *i_idx, int64_t n_j, const double *x,
                    int64_t *nn, double *nn_r2)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < n_i; ++k) {
        const int64_t i = i_idx[k];
        int64_t best = -1;
        double best_r2 = INFINITY;
        for (int64_t j = 0; j < n_j; ++j) {
            if (j == i)
                continue;
            const double dx = x[3 * j + 0] - x[3 * i + 0];
            const double dy = x[3 * j + 1] - x[3 * i + 1];
            const double dz = x[3 * j + 2] - x[3 * i + 2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < best_r2) {
                best_r2 = r2;
                best = j;
            }
        }
        nn[k] = best;
        nn_r2[k] = best_r2;
    }
}
