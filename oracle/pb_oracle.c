/*
 * pb_oracle.c -- plain, slow, FP64 CPU oracle for the well-conditioned direct-sum
 * boundary-integral linear Poisson-Boltzmann method of Geng & Jacob,
 * "A GPU-accelerated Direct-sum Boundary Integral Poisson-Boltzmann Solver".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code with
 * the CUDA library and must never be used as a fallback for it.
 *
 * Everything here is the plain definition written out:
 *   - G0, G_kappa and their normal derivatives: Eq. (5) and the kernel
 *     definitions K1..K4 of Eq. (10), with eps = eps2/eps1 (the reading under
 *     which Eqs. (8)-(9) follow from Eqs. (6)-(7) and the jump conditions (3)).
 *   - the source terms S1, S2 of Eq. (11), with the charge divided by eps1
 *     (the Poisson equation (1) carries eps1 on its left-hand side).
 *   - the discrete matrix-vector product of Eqs. (12)-(13): flat triangles,
 *     centroid collocation, weight W_j = area_j, the singular j = i term dropped
 *     (Section 2.2).  Pairs at zero distance (duplicate centroids) are dropped too.
 *   - the reaction energy of Eq. (14).
 * Unknown ordering: u = [phi_1..phi_N, dphi/dnu_1..dphi/dnu_N].
 * Rows are summed over j = 0..N-1 in index order.  Rows are independent, so an
 * OpenMP loop over rows does not change any row's result.
 */
#include <math.h>
#include <stdint.h>

static const double PI_ORACLE = 3.14159265358979323846;

/* Eq. (5) and its first and second normal derivatives at target x (unit normal
 * nx) and source y (unit normal ny), with r = x - y.  Output order:
 *   g[0] = G0, g[1] = Gk, g[2] = dG0/dny, g[3] = dGk/dny,
 *   g[4] = dG0/dnx, g[5] = dGk/dnx, g[6] = d2G0/dnx dny, g[7] = d2Gk/dnx dny. */
void oracle_green(const double *x, const double *nx, const double *y, const double *ny,
                  double kappa, double *g)
{
    double r0 = x[0] - y[0], r1 = x[1] - y[1], r2 = x[2] - y[2];
    double rho2 = r0 * r0 + r1 * r1 + r2 * r2;
    double rho = sqrt(rho2);
    double four_pi = 4.0 * PI_ORACLE;
    double e = exp(-kappa * rho);
    double kr = kappa * rho;
    double cx = r0 * nx[0] + r1 * nx[1] + r2 * nx[2];   /* r . nu_x */
    double cy = r0 * ny[0] + r1 * ny[1] + r2 * ny[2];   /* r . nu_y */
    double nn = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    double rho3 = rho2 * rho, rho5 = rho3 * rho2;

    g[0] = 1.0 / (four_pi * rho);
    g[1] = e / (four_pi * rho);
    /* grad_y rho = -r/rho, so grad_y (1/rho) = r/rho^3 */
    g[2] = cy / (four_pi * rho3);
    g[3] = e * (1.0 + kr) * cy / (four_pi * rho3);
    /* grad_x rho = r/rho, so grad_x (1/rho) = -r/rho^3 */
    g[4] = -cx / (four_pi * rho3);
    g[5] = -e * (1.0 + kr) * cx / (four_pi * rho3);
    g[6] = (nn / rho3 - 3.0 * cx * cy / rho5) / four_pi;
    g[7] = (e * (1.0 + kr) * nn / rho3 - e * (3.0 + 3.0 * kr + kr * kr) * cx * cy / rho5) / four_pi;
}

/* Eq. (10): K1 = G0 - Gk, K2 = eps dGk/dny - dG0/dny,
 *           K3 = dG0/dnx - (1/eps) dGk/dnx, K4 = d2Gk/dnxdny - d2G0/dnxdny. */
void oracle_kernels(const double *x, const double *nx, const double *y, const double *ny,
                    double eps, double kappa, double *K)
{
    double g[8];
    oracle_green(x, nx, y, ny, kappa, g);
    K[0] = g[0] - g[1];
    K[1] = eps * g[3] - g[2];
    K[2] = g[4] - g[5] / eps;
    K[3] = g[7] - g[6];
}

/* Eqs. (12)-(13).  c, nrm: (N,3) row-major; area: (N); u, y: (2N). */
void oracle_matvec(int64_t N, const double *c, const double *nrm, const double *area,
                   double eps, double kappa, const double *u, double *y)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < N; ++i) {
        double s1 = 0.0, s2 = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d0 = c[3 * i] - c[3 * j], d1 = c[3 * i + 1] - c[3 * j + 1], d2 = c[3 * i + 2] - c[3 * j + 2];
            if (d0 * d0 + d1 * d1 + d2 * d2 == 0.0) continue;
            double K[4];
            oracle_kernels(c + 3 * i, nrm + 3 * i, c + 3 * j, nrm + 3 * j, eps, kappa, K);
            double phi_j = u[j], dphi_j = u[N + j];
            s1 += area[j] * (K[0] * dphi_j + K[1] * phi_j);
            s2 += area[j] * (K[2] * dphi_j + K[3] * phi_j);
        }
        y[i] = 0.5 * (1.0 + eps) * u[i] - s1;
        y[N + i] = 0.5 * (1.0 + 1.0 / eps) * u[N + i] - s2;
    }
}

/* A sampled subset of the rows of Eqs. (12)-(13): rows[r] in [0, N); writes
 * y_rows[2r] = (Au)_{rows[r]} and y_rows[2r+1] = (Au)_{rows[r]+N}. */
void oracle_matvec_rows(int64_t N, const double *c, const double *nrm, const double *area,
                        double eps, double kappa, const double *u,
                        int64_t nrows, const int64_t *rows, double *y_rows)
{
    int64_t r;
#pragma omp parallel for schedule(dynamic, 4)
    for (r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        double s1 = 0.0, s2 = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d0 = c[3 * i] - c[3 * j], d1 = c[3 * i + 1] - c[3 * j + 1], d2 = c[3 * i + 2] - c[3 * j + 2];
            if (d0 * d0 + d1 * d1 + d2 * d2 == 0.0) continue;
            double K[4];
            oracle_kernels(c + 3 * i, nrm + 3 * i, c + 3 * j, nrm + 3 * j, eps, kappa, K);
            s1 += area[j] * (K[0] * u[N + j] + K[1] * u[j]);
            s2 += area[j] * (K[2] * u[N + j] + K[3] * u[j]);
        }
        y_rows[2 * r] = 0.5 * (1.0 + eps) * u[i] - s1;
        y_rows[2 * r + 1] = 0.5 * (1.0 + 1.0 / eps) * u[N + i] - s2;
    }
}

/* The dense 2N x 2N matrix A of Eqs. (12)-(13), row-major. */
void oracle_assemble(int64_t N, const double *c, const double *nrm, const double *area,
                     double eps, double kappa, double *A)
{
    int64_t M = 2 * N, i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) {
        for (int64_t j = 0; j < M; ++j) { A[i * M + j] = 0.0; A[(N + i) * M + j] = 0.0; }
        A[i * M + i] = 0.5 * (1.0 + eps);
        A[(N + i) * M + N + i] = 0.5 * (1.0 + 1.0 / eps);
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d0 = c[3 * i] - c[3 * j], d1 = c[3 * i + 1] - c[3 * j + 1], d2 = c[3 * i + 2] - c[3 * j + 2];
            if (d0 * d0 + d1 * d1 + d2 * d2 == 0.0) continue;
            double K[4];
            oracle_kernels(c + 3 * i, nrm + 3 * i, c + 3 * j, nrm + 3 * j, eps, kappa, K);
            A[i * M + j] = -area[j] * K[1];          /* phi_j in row i      */
            A[i * M + N + j] = -area[j] * K[0];      /* dphi_j in row i     */
            A[(N + i) * M + j] = -area[j] * K[3];    /* phi_j in row N+i    */
            A[(N + i) * M + N + j] = -area[j] * K[2];/* dphi_j in row N+i   */
        }
    }
}

/* Eq. (11): b_i = S1(x_i), b_{N+i} = S2(x_i); charges (Nc,4) rows (x,y,z,Q). */
void oracle_source(int64_t N, const double *c, const double *nrm, int64_t Nc,
                   const double *charges, double eps1, double *b)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < N; ++i) {
        double s1 = 0.0, s2 = 0.0;
        for (int64_t k = 0; k < Nc; ++k) {
            double g[8];
            oracle_green(c + 3 * i, nrm + 3 * i, charges + 4 * k, nrm + 3 * i, 0.0, g);
            s1 += charges[4 * k + 3] / eps1 * g[0];
            s2 += charges[4 * k + 3] / eps1 * g[4];
        }
        b[i] = s1;
        b[N + i] = s2;
    }
}

/* Eq. (14) without the unit conversion: 1/2 sum_k Q_k phi_reac(x_k), with
 * phi_reac(x_k) = sum_j W_j [K1(x_k, x_j) dphi_j + K2(x_k, x_j) phi_j].
 * Also returns the per-charge reaction potentials in phi_reac (may be NULL). */
double oracle_energy(int64_t N, const double *c, const double *nrm, const double *area,
                     int64_t Nc, const double *charges, double eps, double kappa,
                     const double *u, double *phi_reac)
{
    double total = 0.0;
    for (int64_t k = 0; k < Nc; ++k) {
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double d0 = charges[4 * k] - c[3 * j], d1 = charges[4 * k + 1] - c[3 * j + 1],
                   d2 = charges[4 * k + 2] - c[3 * j + 2];
            if (d0 * d0 + d1 * d1 + d2 * d2 == 0.0) continue;
            double K[4];
            /* K1 and K2 do not involve the target normal; pass the source one */
            oracle_kernels(charges + 4 * k, nrm + 3 * j, c + 3 * j, nrm + 3 * j, eps, kappa, K);
            s += area[j] * (K[0] * u[N + j] + K[1] * u[j]);
        }
        if (phi_reac) phi_reac[k] = s;
        total += charges[4 * k + 3] * s;
    }
    return 0.5 * total;
}

/* Gauss sums sum_j W_j dG0(p, x_j)/dnu_j at arbitrary points p (P,3).  For a
 * closed surface with outward normals the integral is -1 inside, -1/2 on the
 * surface and 0 outside. */
void oracle_gauss(int64_t N, const double *c, const double *nrm, const double *area,
                  int64_t P, const double *pts, double *out)
{
    int64_t p;
#pragma omp parallel for schedule(static)
    for (p = 0; p < P; ++p) {
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double d0 = pts[3 * p] - c[3 * j], d1 = pts[3 * p + 1] - c[3 * j + 1], d2 = pts[3 * p + 2] - c[3 * j + 2];
            if (d0 * d0 + d1 * d1 + d2 * d2 == 0.0) continue;
            double g[8];
            oracle_green(pts + 3 * p, nrm + 3 * j, c + 3 * j, nrm + 3 * j, 0.0, g);
            s += area[j] * g[2];
        }
        out[p] = s;
    }
}

/* The straightforward system of Eqs. (6)-(7) (the coupled integral equations
 * the paper takes from Yoon and Lenhoff and sets aside as ill-conditioned,
 * Section 2.1), taken to x on the surface and collocated at the centroids,
 * with the same unknowns u = [phi; dphi/dnu] (interior side) and the
 * interface conditions phi2 = phi1, dphi2/dnu = dphi1/dnu / eps:
 *   row i:     1/2 phi_i - sum_j S0_ij dphi_j + sum_{j != i} W_j dG0/dny(x_i, x_j) phi_j    = S1(x_i)
 *   row N + i: 1/2 phi_i + (1/eps) sum_j Sk_ij dphi_j - sum_{j != i} W_j dGk/dny(x_i, x_j) phi_j = 0
 * The 1/2 comes from the limit of the double-layer potential on a smooth
 * surface (its principal value plus or minus half the density).  The
 * single-layer matrices S0, Sk are W_j G(x_i, x_j) off the diagonal; their
 * diagonal is the integral of G over the flat element from its centroid,
 * taken over the disk of equal area (radius R = sqrt(W_i / pi)):
 * R / 2 for G0 and (1 - exp(-kappa R)) / (2 kappa) for Gk.  The double-layer
 * self term is zero on a flat element.  Output y (2N) = A_YL u. */
void oracle_yl_matvec(int64_t N, const double *c, const double *nrm, const double *area,
                      double eps, double kappa, const double *u, double *y)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < N; ++i) {
        double s_int = 0.0, s_ext = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) {
                double R = sqrt(area[i] / PI_ORACLE);
                double self0 = 0.5 * R;
                double selfk = kappa > 0.0 ? (1.0 - exp(-kappa * R)) / (2.0 * kappa) : 0.5 * R;
                s_int += -self0 * u[N + i];
                s_ext += selfk / eps * u[N + i];
                continue;
            }
            double d0 = c[3 * i] - c[3 * j], d1 = c[3 * i + 1] - c[3 * j + 1], d2 = c[3 * i + 2] - c[3 * j + 2];
            if (d0 * d0 + d1 * d1 + d2 * d2 == 0.0) continue;
            double g[8];
            oracle_green(c + 3 * i, nrm + 3 * i, c + 3 * j, nrm + 3 * j, kappa, g);
            s_int += area[j] * (-g[0] * u[N + j] + g[2] * u[j]);
            s_ext += area[j] * (g[1] / eps * u[N + j] - g[3] * u[j]);
        }
        y[i] = 0.5 * u[i] + s_int;
        y[N + i] = 0.5 * u[i] + s_ext;
    }
}

/* Reaction energy of the straightforward system's solution, Eq. (6) minus
 * the Coulomb part at each charge: 1/2 sum_k Q_k sum_j W_j [G0 dphi_j -
 * dG0/dny phi_j], in the units of oracle_energy (G0 with its 1/(4 pi)). */
double oracle_yl_energy(int64_t N, const double *c, const double *nrm, const double *area,
                        int64_t Nc, const double *charges, const double *u)
{
    double total = 0.0;
    for (int64_t k = 0; k < Nc; ++k) {
        double s = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double g[8];
            oracle_green(charges + 4 * k, nrm + 3 * j, c + 3 * j, nrm + 3 * j, 0.0, g);
            s += area[j] * (g[0] * u[N + j] - g[2] * u[j]);
        }
        total += charges[4 * k + 3] * s;
    }
    return 0.5 * total;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops above (timing only; results do not depend on it). */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n < 1 ? 1 : n);
#else
    (void)n;
#endif
}
