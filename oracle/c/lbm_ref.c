/*
 * Plain FP64 C reference of the single-belt Shan-Chen D3Q19 step with the
 * SRT velocity-shift collision (Sec. 2 of arXiv:1905.09554), OpenMP over z
 * planes.  TEST INFRASTRUCTURE ONLY, like the rest of oracle/: it times the
 * method on the host cores beside the numpy oracle (same definition, same
 * velocity order, same layout) and is checked against it; the library never
 * uses it, and it shares nothing with the CUDA sources.
 *
 * Layout: populations f[a][z][y][x] (x fastest), periodic box.  One SRT
 * step, in the order of Sec. 2:
 *   rho = sum_a f_a, j = sum_a c_a f_a                       (Eq. momentum)
 *   psi = rho0 (1 - exp(-rho / rho0))
 *   F(x) = -G psi(x) sum_a w_a psi(x + c_a) c_a              (Eq. SC_force)
 *   u' = (j + tau F) / rho                                   (Eq. vel_shift)
 *   f_eq = w rho [1 + 3 c.u' + 4.5 (c.u')^2 - 1.5 u'.u']     (Eq. local_eq)
 *   f*(x) = f - (f - f_eq) / tau ; f(x + c_a, t + 1) = f*_a(x, t)   (Eq. LBE)
 * The MRT step (Eq. LBE with M^-1 Lambda M, Eq. barycentric) replaces the
 * last three lines by
 *   u_b = (j + F/2) / rho ; S_a = w_a [3 (c_a - u_b) + 9 (c_a.u_b) c_a].F
 *   m = M f, m_eq = M f_eq(rho, u_b), m_S = M S (d'Humieres D3Q19 moments)
 *   f* = f + M^-1 [ -Lambda (m - m_eq) + (I - Lambda/2) m_S ]
 * with M^-1 = M^T diag(1/|M_k|^2) (the rows are orthogonal).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 19

static int cvec[NQ][3];
static double wq[NQ];
static double mrow[NQ][NQ];  /* mrow[k][a]: moment k of velocity a */
static double mnorm[NQ];     /* |M_k|^2 */
static int tables_ready = 0;

/* The 19 d'Humieres moments of velocity c, in the order rho, e, eps, jx,
 * qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz, mx, my, mz. */
static void moments_of(const int *c, double *m) {
    const double x = c[0], y = c[1], z = c[2], c2 = x * x + y * y + z * z;
    m[0] = 1.0;
    m[1] = 19.0 * c2 - 30.0;
    m[2] = (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
    m[3] = x;
    m[4] = (5.0 * c2 - 9.0) * x;
    m[5] = y;
    m[6] = (5.0 * c2 - 9.0) * y;
    m[7] = z;
    m[8] = (5.0 * c2 - 9.0) * z;
    m[9] = 3.0 * x * x - c2;
    m[10] = (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
    m[11] = y * y - z * z;
    m[12] = (3.0 * c2 - 5.0) * (y * y - z * z);
    m[13] = x * y;
    m[14] = y * z;
    m[15] = x * z;
    m[16] = (y * y - z * z) * x;
    m[17] = (z * z - x * x) * y;
    m[18] = (x * x - y * y) * z;
}

/* D3Q19: the vectors of {0, 1, -1}^3 with |c|^2 <= 2, enumerated with the
 * components in the order 0, 1, -1 (z-component fastest); weights 1/3, 1/18,
 * 1/36 by |c|^2 = 0, 1, 2. */
static void make_tables(void) {
    const int v[3] = {0, 1, -1};
    int a = 0;
    if (tables_ready) return;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                const int cx = v[i], cy = v[j], cz = v[k];
                const int s = cx * cx + cy * cy + cz * cz;
                if (abs(cx) + abs(cy) + abs(cz) > 2) continue;
                cvec[a][0] = cx;
                cvec[a][1] = cy;
                cvec[a][2] = cz;
                wq[a] = s == 0 ? 1.0 / 3.0 : (s == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                ++a;
            }
    for (a = 0; a < NQ; ++a) {
        double m[NQ];
        moments_of(cvec[a], m);
        for (int k = 0; k < NQ; ++k) mrow[k][a] = m[k];
    }
    for (int k = 0; k < NQ; ++k) {
        mnorm[k] = 0.0;
        for (a = 0; a < NQ; ++a) mnorm[k] += mrow[k][a] * mrow[k][a];
    }
    tables_ready = 1;
}

static int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

int lbm_ref_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* nsteps steps from f_in (19 * nx*ny*nz doubles) into f_out: SRT with tau
 * when rates is NULL, else MRT with the 19 rates (moment order).  Returns 0,
 * or -1 if memory could not be allocated. */
static int run(const double *f_in, double *f_out, int nx, int ny, int nz, double G, double tau,
               const double *rates, double rho0, int nsteps) {
    const long n = (long)nx * ny * nz;
    double *f = malloc(sizeof(double) * NQ * n), *g = malloc(sizeof(double) * NQ * n);
    double *psi = malloc(sizeof(double) * n);
    if (!f || !g || !psi) {
        free(f);
        free(g);
        free(psi);
        return -1;
    }
    make_tables();
    memcpy(f, f_in, sizeof(double) * NQ * n);
    for (int step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long i = ((long)z * ny + y) * nx + x;
                    double rho = 0.0;
                    for (int a = 0; a < NQ; ++a) rho += f[a * n + i];
                    psi[i] = rho0 * (1.0 - exp(-rho / rho0));
                }
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long i = ((long)z * ny + y) * nx + x;
                    double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, s[3] = {0.0, 0.0, 0.0}, u[3];
                    for (int a = 0; a < NQ; ++a) {
                        const double fa = f[a * n + i];
                        rho += fa;
                        for (int d = 0; d < 3; ++d) j[d] += cvec[a][d] * fa;
                        const long nb = ((long)wrap(z + cvec[a][2], nz) * ny + wrap(y + cvec[a][1], ny)) * nx +
                                        wrap(x + cvec[a][0], nx);
                        for (int d = 0; d < 3; ++d) s[d] += wq[a] * cvec[a][d] * psi[nb];
                    }
                    double usq = 0.0, F[3];
                    for (int d = 0; d < 3; ++d) {
                        F[d] = -G * psi[i] * s[d];
                        /* SRT: shifted velocity; MRT: barycentric velocity */
                        u[d] = rates ? (j[d] + 0.5 * F[d]) / rho : (j[d] + tau * F[d]) / rho;
                        usq += u[d] * u[d];
                    }
                    double post[NQ];
                    if (!rates) {
                        for (int a = 0; a < NQ; ++a) {
                            const double cu = cvec[a][0] * u[0] + cvec[a][1] * u[1] + cvec[a][2] * u[2];
                            const double feq = wq[a] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                            post[a] = f[a * n + i] - (f[a * n + i] - feq) / tau;
                        }
                    } else {
                        double feq[NQ], src[NQ];
                        for (int a = 0; a < NQ; ++a) {
                            const double cu = cvec[a][0] * u[0] + cvec[a][1] * u[1] + cvec[a][2] * u[2];
                            double sF = 0.0;
                            for (int d = 0; d < 3; ++d) sF += (3.0 * (cvec[a][d] - u[d]) + 9.0 * cu * cvec[a][d]) * F[d];
                            feq[a] = wq[a] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                            src[a] = wq[a] * sF;
                            post[a] = f[a * n + i];
                        }
                        for (int k = 0; k < NQ; ++k) {
                            double m = 0.0, me = 0.0, ms = 0.0;
                            for (int a = 0; a < NQ; ++a) {
                                m += mrow[k][a] * f[a * n + i];
                                me += mrow[k][a] * feq[a];
                                ms += mrow[k][a] * src[a];
                            }
                            const double dk = (-rates[k] * (m - me) + (1.0 - 0.5 * rates[k]) * ms) / mnorm[k];
                            for (int a = 0; a < NQ; ++a) post[a] += mrow[k][a] * dk;
                        }
                    }
                    for (int a = 0; a < NQ; ++a) {
                        const long dst = ((long)wrap(z + cvec[a][2], nz) * ny + wrap(y + cvec[a][1], ny)) * nx +
                                         wrap(x + cvec[a][0], nx);
                        g[a * n + dst] = post[a];
                    }
                }
        double *t = f;
        f = g;
        g = t;
    }
    memcpy(f_out, f, sizeof(double) * NQ * n);
    free(f);
    free(g);
    free(psi);
    return 0;
}

int lbm_ref_run_srt(const double *f_in, double *f_out, int nx, int ny, int nz, double G, double tau,
                    double rho0, int nsteps) {
    return run(f_in, f_out, nx, ny, nz, G, tau, NULL, rho0, nsteps);
}

/* MRT with Guo forcing: rates[19] in moment order (rho, e, eps, jx, ...). */
int lbm_ref_run_mrt(const double *f_in, double *f_out, int nx, int ny, int nz, double G, const double *rates,
                    double rho0, int nsteps) {
    if (!rates) return -1;
    return run(f_in, f_out, nx, ny, nz, G, 1.0, rates, rho0, nsteps);
}
