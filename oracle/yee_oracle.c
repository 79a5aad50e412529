/*
 * Plain FP64 Yee FDTD oracle for a PEC box cavity.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py load this code.  It shares nothing with the CUDA
 * path: no headers, no helpers, no tables.
 *
 * What it computes (He, Andersson, Markidis, "Optimizing FDTD Solvers for
 * Electromagnetics: A Compiler-Guided Approach with High-Level Tensor
 * Abstractions", arXiv 2504.09118):
 *   - Maxwell's curl equations with J = 0 (Sec. 2, Eq. 1), discretised on the
 *     Yee grid, staggered in space and time (Sec. 2, Eq. 2); oracle_step_sources
 *     adds point currents J, the term of Eq. 1 the benchmark sets to zero;
 *   - one time step = H update from curl E, H boundary handling, E update from
 *     curl H, E boundary handling (Sec. 2.1, Listing 1);
 *   - the per-component update written as a plain triple loop (Listing 2),
 *     with fields updated in place (Sec. 3, in-place bufferisation).
 *
 * Readings where the paper is silent or garbled:
 *   - Listing 2's index range reads one past equal-sized arrays; the arrays
 *     here have the staggered Yee extents implied by Listing 3's slice shapes.
 *   - Eq. 1 prints dH/dt = +(1/mu) curl E, while Eq. 2 and Listing 2 carry
 *     Faraday's minus sign; the minus sign is used (H -= ch * curl E).
 *   - The state is (H^{n-1/2}, E^n); a step applies H then E, as Listing 1 does.
 *   - PEC boundary handling: tangential E on the six faces is held at zero
 *     (handle_E_edge); with staggered extents handle_H_edge has nothing to do,
 *     and normal H on a face keeps its initial value.
 *
 * Layout: every component is a dense array of (nz+1)*(ny+1)*(nx+1) doubles,
 * x fastest; component c at index (i,j,k) sits at its Yee position:
 *   Ex(i+1/2,j,k): i<nx, j<=ny, k<=nz     Hx(i,j+1/2,k+1/2): i<=nx, j<ny, k<nz
 *   Ey(i,j+1/2,k): i<=nx, j<ny, k<=nz     Hy(i+1/2,j,k+1/2): i<nx, j<=ny, k<nz
 *   Ez(i,j,k+1/2): i<=nx, j<=ny, k<nz     Hz(i+1/2,j+1/2,k): i<nx, j<ny, k<=nz
 * Entries outside a component's extent are never read or written.
 * Coefficients: ce = dt/(eps*dx) at E positions, ch = dt/(mu*dx) at H
 * positions, in the same layout, one array per component.
 *
 * The only pragma is "omp parallel for" on outer loops of the field updates,
 * which leaves every result bit-identical to the serial build.
 */
#include <math.h>
#include <stddef.h>

#define AT(a, i, j, k) (a)[(((size_t)(k) * (size_t)(ny + 1) + (size_t)(j)) * (size_t)(nx + 1)) + (size_t)(i)]

/* H^{n+1/2} = H^{n-1/2} - ch * curl E^n over each H component's extent (Eq. 2, right column). */
void oracle_update_h(int nx, int ny, int nz,
                     double *hx, double *hy, double *hz,
                     const double *ex, const double *ey, const double *ez,
                     const double *chx, const double *chy, const double *chz)
{
    int i, j, k;
#pragma omp parallel for private(i, j)
    for (k = 0; k < nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 0; i <= nx; ++i) {
                /* (curl E)_x = dEz/dy - dEy/dz */
                double c = (AT(ez, i, j + 1, k) - AT(ez, i, j, k)) - (AT(ey, i, j, k + 1) - AT(ey, i, j, k));
                AT(hx, i, j, k) -= AT(chx, i, j, k) * c;
            }
#pragma omp parallel for private(i, j)
    for (k = 0; k < nz; ++k)
        for (j = 0; j <= ny; ++j)
            for (i = 0; i < nx; ++i) {
                /* (curl E)_y = dEx/dz - dEz/dx */
                double c = (AT(ex, i, j, k + 1) - AT(ex, i, j, k)) - (AT(ez, i + 1, j, k) - AT(ez, i, j, k));
                AT(hy, i, j, k) -= AT(chy, i, j, k) * c;
            }
#pragma omp parallel for private(i, j)
    for (k = 0; k <= nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 0; i < nx; ++i) {
                /* (curl E)_z = dEy/dx - dEx/dy */
                double c = (AT(ey, i + 1, j, k) - AT(ey, i, j, k)) - (AT(ex, i, j + 1, k) - AT(ex, i, j, k));
                AT(hz, i, j, k) -= AT(chz, i, j, k) * c;
            }
}

/* E^{n+1} = E^n + ce * curl H^{n+1/2} over each E component's non-tangential entries (Eq. 2, left column). */
void oracle_update_e(int nx, int ny, int nz,
                     double *ex, double *ey, double *ez,
                     const double *hx, const double *hy, const double *hz,
                     const double *cex, const double *cey, const double *cez)
{
    int i, j, k;
#pragma omp parallel for private(i, j)
    for (k = 1; k < nz; ++k)
        for (j = 1; j < ny; ++j)
            for (i = 0; i < nx; ++i) {
                /* (curl H)_x = dHz/dy - dHy/dz */
                double c = (AT(hz, i, j, k) - AT(hz, i, j - 1, k)) - (AT(hy, i, j, k) - AT(hy, i, j, k - 1));
                AT(ex, i, j, k) += AT(cex, i, j, k) * c;
            }
#pragma omp parallel for private(i, j)
    for (k = 1; k < nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 1; i < nx; ++i) {
                /* (curl H)_y = dHx/dz - dHz/dx */
                double c = (AT(hx, i, j, k) - AT(hx, i, j, k - 1)) - (AT(hz, i, j, k) - AT(hz, i - 1, j, k));
                AT(ey, i, j, k) += AT(cey, i, j, k) * c;
            }
#pragma omp parallel for private(i, j)
    for (k = 0; k < nz; ++k)
        for (j = 1; j < ny; ++j)
            for (i = 1; i < nx; ++i) {
                /* (curl H)_z = dHy/dx - dHx/dy */
                double c = (AT(hy, i, j, k) - AT(hy, i - 1, j, k)) - (AT(hx, i, j, k) - AT(hx, i, j - 1, k));
                AT(ez, i, j, k) += AT(cez, i, j, k) * c;
            }
}

/* PEC (handle_E_edge of Listing 1): tangential E on the six faces is zero. */
void oracle_pec_e(int nx, int ny, int nz, double *ex, double *ey, double *ez)
{
    int i, j, k;
    for (k = 0; k <= nz; ++k)
        for (j = 0; j <= ny; ++j)
            for (i = 0; i <= nx; ++i) {
                int fx = (i == 0 || i == nx), fy = (j == 0 || j == ny), fz = (k == 0 || k == nz);
                if (i < nx && (fy || fz)) AT(ex, i, j, k) = 0.0;
                if (j < ny && (fx || fz)) AT(ey, i, j, k) = 0.0;
                if (k < nz && (fx || fy)) AT(ez, i, j, k) = 0.0;
            }
}

/* nsteps leapfrog steps in the order of Listing 1: curl H, handle_H_edge (nothing to
 * do on the staggered PEC grid), curl E, handle_E_edge.  f = {Ex,Ey,Ez,Hx,Hy,Hz},
 * ce = {cex,cey,cez}, ch = {chx,chy,chz}. */
void oracle_step(int nx, int ny, int nz, double *const f[6],
                 const double *const ce[3], const double *const ch[3], int nsteps)
{
    for (int n = 0; n < nsteps; ++n) {
        oracle_update_h(nx, ny, nz, f[3], f[4], f[5], f[0], f[1], f[2], ch[0], ch[1], ch[2]);
        oracle_update_e(nx, ny, nz, f[0], f[1], f[2], f[3], f[4], f[5], ce[0], ce[1], ce[2]);
        oracle_pec_e(nx, ny, nz, f[0], f[1], f[2]);
    }
}

/* As oracle_step, with point currents: Eq. 1 of Sec. 2 with J != 0 gives dE/dt = (curl H - J)/eps,
 * so the E update of the step from E^n to E^{n+1} also subtracts ce * dx * J^{n+1/2} at each source.
 * Source s drives component comp[s] (0 Ex, 1 Ey, 2 Ez) at canonical index (i[s], j[s], k[s]) with
 * J^{n+1/2} = wave[s * wave_len + n] for the n-th step counted from n0 (0 once n >= wave_len).  The
 * source term is added after the curl H update and before handle_E_edge. */
void oracle_step_sources(int nx, int ny, int nz, double *const f[6],
                         const double *const ce[3], const double *const ch[3], int nsteps, int n0,
                         int nsrc, const int *comp, const int *si, const int *sj, const int *sk,
                         const double *wave, int wave_len, double dx)
{
    for (int n = 0; n < nsteps; ++n) {
        oracle_update_h(nx, ny, nz, f[3], f[4], f[5], f[0], f[1], f[2], ch[0], ch[1], ch[2]);
        oracle_update_e(nx, ny, nz, f[0], f[1], f[2], f[3], f[4], f[5], ce[0], ce[1], ce[2]);
        const int t = n0 + n;
        for (int q = 0; q < nsrc; ++q) {
            const double J = t < wave_len ? wave[(size_t)q * wave_len + t] : 0.0;
            const int c = comp[q];
            AT(f[c], si[q], sj[q], sk[q]) -= AT(ce[c], si[q], sj[q], sk[q]) * dx * J;
        }
        oracle_pec_e(nx, ny, nz, f[0], f[1], f[2]);
    }
}

/*
 * Discrete Yee energy of the state (H^{n-1/2}, E^n), cell volume 1:
 *   W^n = 1/2 sum eps E^2 + 1/2 sum mu H^{n-1/2} H^{n+1/2},
 * with eps = dt/(ce dx), mu = dt/(ch dx) at each position and
 * H^{n+1/2} = H^{n-1/2} - ch curl E^n formed on the fly (not stored).
 * The paper defines no energy; this is the leapfrog invariant of Eq. 2 on a
 * lossless PEC cavity (exactly conserved in exact arithmetic).
 */
double oracle_energy(int nx, int ny, int nz, const double *const f[6],
                     const double *const ce[3], const double *const ch[3], double dt_over_dx)
{
    const double *ex = f[0], *ey = f[1], *ez = f[2], *hx = f[3], *hy = f[4], *hz = f[5];
    double we = 0.0, wh = 0.0;
    int i, j, k;
    for (k = 0; k <= nz; ++k)
        for (j = 0; j <= ny; ++j)
            for (i = 0; i <= nx; ++i) {
                if (i < nx) we += AT(ex, i, j, k) * AT(ex, i, j, k) / AT(ce[0], i, j, k);
                if (j < ny) we += AT(ey, i, j, k) * AT(ey, i, j, k) / AT(ce[1], i, j, k);
                if (k < nz) we += AT(ez, i, j, k) * AT(ez, i, j, k) / AT(ce[2], i, j, k);
                if (j < ny && k < nz) {
                    double c = (AT(ez, i, j + 1, k) - AT(ez, i, j, k)) - (AT(ey, i, j, k + 1) - AT(ey, i, j, k));
                    double h = AT(hx, i, j, k), cc = AT(ch[0], i, j, k);
                    wh += h * (h - cc * c) / cc;
                }
                if (i < nx && k < nz) {
                    double c = (AT(ex, i, j, k + 1) - AT(ex, i, j, k)) - (AT(ez, i + 1, j, k) - AT(ez, i, j, k));
                    double h = AT(hy, i, j, k), cc = AT(ch[1], i, j, k);
                    wh += h * (h - cc * c) / cc;
                }
                if (i < nx && j < ny) {
                    double c = (AT(ey, i + 1, j, k) - AT(ey, i, j, k)) - (AT(ex, i, j + 1, k) - AT(ex, i, j, k));
                    double h = AT(hz, i, j, k), cc = AT(ch[2], i, j, k);
                    wh += h * (h - cc * c) / cc;
                }
            }
    return 0.5 * dt_over_dx * (we + wh);
}

/*
 * Discrete divergences, the quantities Gauss's laws keep fixed on the Yee grid
 * (the paper states none; div of a discrete curl vanishes identically):
 *   divE at interior nodes (1<=i<=nx-1, 1<=j<=ny-1, 1<=k<=nz-1), written to
 *   out_e in the canonical (nz+1,ny+1,nx+1) layout, zero elsewhere:
 *     sum_c  D_c(node) - D_c(node - e_c),   D_c = E_c / ce_c;
 *   divH at every cell (i<nx, j<ny, k<nz), written to out_h as (nz,ny,nx):
 *     sum_c  B_c(cell + e_c) - B_c(cell),   B_c = H_c / ch_c.
 */
void oracle_divergence(int nx, int ny, int nz, const double *const f[6],
                       const double *const ce[3], const double *const ch[3],
                       double *out_e, double *out_h)
{
    const double *ex = f[0], *ey = f[1], *ez = f[2], *hx = f[3], *hy = f[4], *hz = f[5];
    int i, j, k;
    for (k = 0; k <= nz; ++k)
        for (j = 0; j <= ny; ++j)
            for (i = 0; i <= nx; ++i) {
                double d = 0.0;
                if (i >= 1 && i < nx && j >= 1 && j < ny && k >= 1 && k < nz) {
                    d = AT(ex, i, j, k) / AT(ce[0], i, j, k) - AT(ex, i - 1, j, k) / AT(ce[0], i - 1, j, k)
                      + AT(ey, i, j, k) / AT(ce[1], i, j, k) - AT(ey, i, j - 1, k) / AT(ce[1], i, j - 1, k)
                      + AT(ez, i, j, k) / AT(ce[2], i, j, k) - AT(ez, i, j, k - 1) / AT(ce[2], i, j, k - 1);
                }
                AT(out_e, i, j, k) = d;
            }
    for (k = 0; k < nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 0; i < nx; ++i) {
                double d = AT(hx, i + 1, j, k) / AT(ch[0], i + 1, j, k) - AT(hx, i, j, k) / AT(ch[0], i, j, k)
                         + AT(hy, i, j + 1, k) / AT(ch[1], i, j + 1, k) - AT(hy, i, j, k) / AT(ch[1], i, j, k)
                         + AT(hz, i, j, k + 1) / AT(ch[2], i, j, k + 1) - AT(hz, i, j, k) / AT(ch[2], i, j, k);
                out_h[((size_t)k * (size_t)ny + (size_t)j) * (size_t)nx + (size_t)i] = d;
            }
}

/* Number of OpenMP threads this build runs the field updates on (1 when built without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int oracle_threads(void) { return omp_get_max_threads(); }
#else
int oracle_threads(void) { return 1; }
#endif

/*
 * Fourth-order spatial differences (the "(2,4)" Yee scheme).
 *
 * Sec. 6 of the paper names higher-order schemes as the way to raise the
 * arithmetic intensity of FDTD on accelerators but fixes none.  This is the
 * standard staggered four-point difference, exact for cubic polynomials:
 *   (D f)(p) = c1 [f(p + 1/2) - f(p - 1/2)] + c2 [f(p + 3/2) - f(p - 3/2)],
 *   c1 = 9/8, c2 = -1/24   (passed in, so that c1 = 1, c2 = 0 is Eq. 2 again),
 * used for every derivative of the curls in Eq. 2.  The PEC walls are closed by
 * image theory: about each wall the tangential E is odd and the tangential H
 * even, so a tap one position beyond the cavity reads the mirrored value with
 * that sign.  Every curl term differentiates a component along an axis that it
 * is tangential to, so these two rules cover every tap (a tap reaches at most
 * one position past a wall).  Step order, extents, PEC and in-place updates
 * are those of oracle_step.
 */

/* E component a, node-aligned along `axis` and zero on both walls normal to it, at (i, j, k)
 * where the coordinate along axis may lie one past a wall: odd image. */
static double tap_e(const double *a, int nx, int ny, int nz, int axis, int i, int j, int k)
{
    int *q = axis == 0 ? &i : axis == 1 ? &j : &k;
    const int n = axis == 0 ? nx : axis == 1 ? ny : nz;
    double s = 1.0;
    if (*q < 0) {
        *q = -*q;
        s = -1.0;
    } else if (*q > n) {
        *q = 2 * n - *q;
        s = -1.0;
    }
    return s * AT(a, i, j, k);
}

/* H component a, half-cell aligned along `axis` (index q stands for q + 1/2, 0 <= q < n):
 * even image about each wall. */
static double tap_h(const double *a, int nx, int ny, int nz, int axis, int i, int j, int k)
{
    int *q = axis == 0 ? &i : axis == 1 ? &j : &k;
    const int n = axis == 0 ? nx : axis == 1 ? ny : nz;
    if (*q < 0)
        *q = -1 - *q;
    else if (*q > n - 1)
        *q = 2 * n - 1 - *q;
    return AT(a, i, j, k);
}

/* D of E component a along axis at the half-cell position (index + 1/2) of (i, j, k). */
static double d4_e(const double *a, int nx, int ny, int nz, int axis, int i, int j, int k, double c1, double c2)
{
    const int di = axis == 0, dj = axis == 1, dk = axis == 2;
    const double p1 = tap_e(a, nx, ny, nz, axis, i + di, j + dj, k + dk);
    const double m1 = tap_e(a, nx, ny, nz, axis, i, j, k);
    const double p3 = tap_e(a, nx, ny, nz, axis, i + 2 * di, j + 2 * dj, k + 2 * dk);
    const double m3 = tap_e(a, nx, ny, nz, axis, i - di, j - dj, k - dk);
    return c1 * (p1 - m1) + c2 * (p3 - m3);
}

/* D of H component a along axis at the node position (index) of (i, j, k). */
static double d4_h(const double *a, int nx, int ny, int nz, int axis, int i, int j, int k, double c1, double c2)
{
    const int di = axis == 0, dj = axis == 1, dk = axis == 2;
    const double p1 = tap_h(a, nx, ny, nz, axis, i, j, k);
    const double m1 = tap_h(a, nx, ny, nz, axis, i - di, j - dj, k - dk);
    const double p3 = tap_h(a, nx, ny, nz, axis, i + di, j + dj, k + dk);
    const double m3 = tap_h(a, nx, ny, nz, axis, i - 2 * di, j - 2 * dj, k - 2 * dk);
    return c1 * (p1 - m1) + c2 * (p3 - m3);
}

/* H^{n+1/2} = H^{n-1/2} - ch * curl4 E^n over each H component's extent. */
void oracle_update_h4(int nx, int ny, int nz,
                      double *hx, double *hy, double *hz,
                      const double *ex, const double *ey, const double *ez,
                      const double *chx, const double *chy, const double *chz, double c1, double c2)
{
    int i, j, k;
#pragma omp parallel for private(i, j)
    for (k = 0; k < nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 0; i <= nx; ++i) {
                double c = d4_e(ez, nx, ny, nz, 1, i, j, k, c1, c2) - d4_e(ey, nx, ny, nz, 2, i, j, k, c1, c2);
                AT(hx, i, j, k) -= AT(chx, i, j, k) * c;
            }
#pragma omp parallel for private(i, j)
    for (k = 0; k < nz; ++k)
        for (j = 0; j <= ny; ++j)
            for (i = 0; i < nx; ++i) {
                double c = d4_e(ex, nx, ny, nz, 2, i, j, k, c1, c2) - d4_e(ez, nx, ny, nz, 0, i, j, k, c1, c2);
                AT(hy, i, j, k) -= AT(chy, i, j, k) * c;
            }
#pragma omp parallel for private(i, j)
    for (k = 0; k <= nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 0; i < nx; ++i) {
                double c = d4_e(ey, nx, ny, nz, 0, i, j, k, c1, c2) - d4_e(ex, nx, ny, nz, 1, i, j, k, c1, c2);
                AT(hz, i, j, k) -= AT(chz, i, j, k) * c;
            }
}

/* E^{n+1} = E^n + ce * curl4 H^{n+1/2} over each E component's non-tangential entries. */
void oracle_update_e4(int nx, int ny, int nz,
                      double *ex, double *ey, double *ez,
                      const double *hx, const double *hy, const double *hz,
                      const double *cex, const double *cey, const double *cez, double c1, double c2)
{
    int i, j, k;
#pragma omp parallel for private(i, j)
    for (k = 1; k < nz; ++k)
        for (j = 1; j < ny; ++j)
            for (i = 0; i < nx; ++i) {
                double c = d4_h(hz, nx, ny, nz, 1, i, j, k, c1, c2) - d4_h(hy, nx, ny, nz, 2, i, j, k, c1, c2);
                AT(ex, i, j, k) += AT(cex, i, j, k) * c;
            }
#pragma omp parallel for private(i, j)
    for (k = 1; k < nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 1; i < nx; ++i) {
                double c = d4_h(hx, nx, ny, nz, 2, i, j, k, c1, c2) - d4_h(hz, nx, ny, nz, 0, i, j, k, c1, c2);
                AT(ey, i, j, k) += AT(cey, i, j, k) * c;
            }
#pragma omp parallel for private(i, j)
    for (k = 0; k < nz; ++k)
        for (j = 1; j < ny; ++j)
            for (i = 1; i < nx; ++i) {
                double c = d4_h(hy, nx, ny, nz, 0, i, j, k, c1, c2) - d4_h(hx, nx, ny, nz, 1, i, j, k, c1, c2);
                AT(ez, i, j, k) += AT(cez, i, j, k) * c;
            }
}

/* nsteps steps of the fourth-order scheme, in the order of oracle_step; with nsrc > 0 the point
 * currents of oracle_step_sources are added after each E update. */
void oracle_step4(int nx, int ny, int nz, double *const f[6],
                  const double *const ce[3], const double *const ch[3], int nsteps, double c1, double c2,
                  int n0, int nsrc, const int *comp, const int *si, const int *sj, const int *sk,
                  const double *wave, int wave_len, double dx)
{
    for (int n = 0; n < nsteps; ++n) {
        oracle_update_h4(nx, ny, nz, f[3], f[4], f[5], f[0], f[1], f[2], ch[0], ch[1], ch[2], c1, c2);
        oracle_update_e4(nx, ny, nz, f[0], f[1], f[2], f[3], f[4], f[5], ce[0], ce[1], ce[2], c1, c2);
        const int t = n0 + n;
        for (int q = 0; q < nsrc; ++q) {
            const double J = t < wave_len ? wave[(size_t)q * wave_len + t] : 0.0;
            const int c = comp[q];
            AT(f[c], si[q], sj[q], sk[q]) -= AT(ce[c], si[q], sj[q], sk[q]) * dx * J;
        }
        oracle_pec_e(nx, ny, nz, f[0], f[1], f[2]);
    }
}

/* oracle_energy with the fourth-order curl in the virtual H^{n+1/2}: the invariant of the (2,4)
 * leapfrog (its curl operators are each other's negative transpose under the image closure). */
double oracle_energy4(int nx, int ny, int nz, const double *const f[6],
                      const double *const ce[3], const double *const ch[3], double dt_over_dx, double c1, double c2)
{
    const double *ex = f[0], *ey = f[1], *ez = f[2], *hx = f[3], *hy = f[4], *hz = f[5];
    double we = 0.0, wh = 0.0;
    int i, j, k;
    for (k = 0; k <= nz; ++k)
        for (j = 0; j <= ny; ++j)
            for (i = 0; i <= nx; ++i) {
                if (i < nx) we += AT(ex, i, j, k) * AT(ex, i, j, k) / AT(ce[0], i, j, k);
                if (j < ny) we += AT(ey, i, j, k) * AT(ey, i, j, k) / AT(ce[1], i, j, k);
                if (k < nz) we += AT(ez, i, j, k) * AT(ez, i, j, k) / AT(ce[2], i, j, k);
                if (j < ny && k < nz) {
                    double c = d4_e(ez, nx, ny, nz, 1, i, j, k, c1, c2) - d4_e(ey, nx, ny, nz, 2, i, j, k, c1, c2);
                    double h = AT(hx, i, j, k), cc = AT(ch[0], i, j, k);
                    wh += h * (h - cc * c) / cc;
                }
                if (i < nx && k < nz) {
                    double c = d4_e(ex, nx, ny, nz, 2, i, j, k, c1, c2) - d4_e(ez, nx, ny, nz, 0, i, j, k, c1, c2);
                    double h = AT(hy, i, j, k), cc = AT(ch[1], i, j, k);
                    wh += h * (h - cc * c) / cc;
                }
                if (i < nx && j < ny) {
                    double c = d4_e(ey, nx, ny, nz, 0, i, j, k, c1, c2) - d4_e(ex, nx, ny, nz, 1, i, j, k, c1, c2);
                    double h = AT(hz, i, j, k), cc = AT(ch[2], i, j, k);
                    wh += h * (h - cc * c) / cc;
                }
            }
    return 0.5 * dt_over_dx * (we + wh);
}

/* Flux density B_a = H_a / ch_a (normal to the walls across axis a, node-aligned along it) at an
 * index that may lie one past a wall: odd image, as its changes (-curl E, whose normal component
 * is odd about a PEC wall) are. */
static double tap_b(const double *h, const double *ch, int nx, int ny, int nz, int axis, int i, int j, int k)
{
    int *q = axis == 0 ? &i : axis == 1 ? &j : &k;
    const int n = axis == 0 ? nx : axis == 1 ? ny : nz;
    double s = 1.0;
    if (*q < 0) {
        *q = -*q;
        s = -1.0;
    } else if (*q > n) {
        *q = 2 * n - *q;
        s = -1.0;
    }
    return s * AT(h, i, j, k) / AT(ch, i, j, k);
}

/* Displacement D_a = E_a / ce_a (normal to the walls across axis a, half-cell aligned along it):
 * even image, as curl H's normal component is. */
static double tap_d(const double *e, const double *ce, int nx, int ny, int nz, int axis, int i, int j, int k)
{
    int *q = axis == 0 ? &i : axis == 1 ? &j : &k;
    const int n = axis == 0 ? nx : axis == 1 ? ny : nz;
    if (*q < 0)
        *q = -1 - *q;
    else if (*q > n - 1)
        *q = 2 * n - 1 - *q;
    return AT(e, i, j, k) / AT(ce, i, j, k);
}

/* oracle_divergence with fourth-order differences and the images above; both stay invariant under
 * oracle_step4 (the difference operators of different axes commute on the image-extended grid). */
void oracle_divergence4(int nx, int ny, int nz, const double *const f[6],
                        const double *const ce[3], const double *const ch[3],
                        double *out_e, double *out_h, double c1, double c2)
{
    int i, j, k;
    for (k = 0; k <= nz; ++k)
        for (j = 0; j <= ny; ++j)
            for (i = 0; i <= nx; ++i) {
                double d = 0.0;
                if (i >= 1 && i < nx && j >= 1 && j < ny && k >= 1 && k < nz) {
                    for (int a = 0; a < 3; ++a) {
                        const int di = a == 0, dj = a == 1, dk = a == 2;
                        const double *e = f[a], *c = ce[a];
                        d += c1 * (tap_d(e, c, nx, ny, nz, a, i, j, k) - tap_d(e, c, nx, ny, nz, a, i - di, j - dj, k - dk))
                           + c2 * (tap_d(e, c, nx, ny, nz, a, i + di, j + dj, k + dk)
                                   - tap_d(e, c, nx, ny, nz, a, i - 2 * di, j - 2 * dj, k - 2 * dk));
                    }
                }
                AT(out_e, i, j, k) = d;
            }
    for (k = 0; k < nz; ++k)
        for (j = 0; j < ny; ++j)
            for (i = 0; i < nx; ++i) {
                double d = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const int di = a == 0, dj = a == 1, dk = a == 2;
                    const double *h = f[3 + a], *c = ch[a];
                    d += c1 * (tap_b(h, c, nx, ny, nz, a, i + di, j + dj, k + dk) - tap_b(h, c, nx, ny, nz, a, i, j, k))
                       + c2 * (tap_b(h, c, nx, ny, nz, a, i + 2 * di, j + 2 * dj, k + 2 * dk)
                               - tap_b(h, c, nx, ny, nz, a, i - di, j - dj, k - dk));
                }
                out_h[((size_t)k * (size_t)ny + (size_t)j) * (size_t)nx + (size_t)i] = d;
            }
}
