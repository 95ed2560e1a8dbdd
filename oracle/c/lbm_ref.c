/*
 * Plain FP64 C reference of the single-belt Shan-Chen D3Q19 step with the
 * SRT velocity-shift collision (Sec. 2 of arXiv:1905.09554), OpenMP over z
 * planes.  TEST INFRASTRUCTURE ONLY, like the rest of oracle/: it times the
 * method on the host cores beside the numpy oracle (same definition, same
 * velocity order, same layout) and is checked against it; the library never
 * uses it, and it shares nothing with the CUDA sources.
 *
 * Layout: populations f[a][z][y][x] (x fastest), periodic box.  One step, in
 * the order of Sec. 2:
 *   rho = sum_a f_a, j = sum_a c_a f_a                       (Eq. momentum)
 *   psi = rho0 (1 - exp(-rho / rho0))
 *   F(x) = -G psi(x) sum_a w_a psi(x + c_a) c_a              (Eq. SC_force)
 *   u' = (j + tau F) / rho                                   (Eq. vel_shift)
 *   f_eq = w rho [1 + 3 c.u' + 4.5 (c.u')^2 - 1.5 u'.u']     (Eq. local_eq)
 *   f*(x) = f - (f - f_eq) / tau ; f(x + c_a, t + 1) = f*_a(x, t)   (Eq. LBE)
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
static int tables_ready = 0;

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

/* nsteps SRT steps from f_in (19 * nx*ny*nz doubles) into f_out.  Returns 0,
 * or -1 if memory could not be allocated. */
int lbm_ref_run_srt(const double *f_in, double *f_out, int nx, int ny, int nz, double G, double tau,
                    double rho0, int nsteps) {
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
                    double usq = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const double F = -G * psi[i] * s[d];
                        u[d] = (j[d] + tau * F) / rho;
                        usq += u[d] * u[d];
                    }
                    for (int a = 0; a < NQ; ++a) {
                        const double cu = cvec[a][0] * u[0] + cvec[a][1] * u[1] + cvec[a][2] * u[2];
                        const double feq = wq[a] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
                        const double fs = f[a * n + i] - (f[a * n + i] - feq) / tau;
                        const long dst = ((long)wrap(z + cvec[a][2], nz) * ny + wrap(y + cvec[a][1], ny)) * nx +
                                         wrap(x + cvec[a][0], nx);
                        g[a * n + dst] = fs;
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
