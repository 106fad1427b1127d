/* Potential-flow fixture on the host CPU (input generation for large oracle runs; not
 * part of the state-of-charge solver and not called by it).
 *
 * The same discrete problem as the GPU fixture (synth_flow.cu): phi = 1 on inlet faces
 * (low-z face of plane 0), phi = 0 on outlet faces (high-z face of plane nz-1), no flux
 * through fiber faces and side walls, cell-to-cell conductance 1, cell-to-face 2. The
 * unknown is psi = phi - phi_lin with phi_lin = 1 - (k + 1/2)/nz, so the rounding floor
 * of the face differences is set by |psi| << 1. Jacobi-preconditioned CG in FP64.
 *
 * Sums are formed per z-plane and the plane sums added in plane order, so the result
 * does not depend on the number of threads; with -ffp-contract=off it is the same on
 * every IEEE-754 host. Face velocities u = -grad(phi) are scaled so that the mean of W
 * over fluid z-faces (inlet and outlet faces included) equals u_mean.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* neighbour bits of a fluid cell: fluid -x, +x, -y, +y, -z, +z; inlet, outlet plane */
enum { NXM = 1, NXP = 2, NYM = 4, NYP = 8, NZM = 16, NZP = 32, NIN = 64, NOUT = 128 };

typedef struct {
    int nx, ny, nz;
    int64_t nxny, N;
    const uint8_t* nb;   /* per cell: neighbour bits (0 for a solid cell) */
    const uint8_t* solid;
} Grid;

static double diag_of(unsigned m) {
    double d = 0.0;
    for (int b = 0; b < 6; ++b)
        if (m & (1u << b)) d += 1.0;
    if (m & NIN) d += 2.0;
    if (m & NOUT) d += 2.0;
    return d;
}

/* (A x)_c of a fluid cell */
static double apply_row(const Grid* g, const double* x, int64_t c, unsigned m) {
    const double xc = x[c];
    double a = 0.0;
    if (m & NXM) a += xc - x[c - 1];
    if (m & NXP) a += xc - x[c + 1];
    if (m & NYM) a += xc - x[c - g->nx];
    if (m & NYP) a += xc - x[c + g->nx];
    if (m & NZM) a += xc - x[c - g->nxny];
    if (m & NZP) a += xc - x[c + g->nxny];
    if (m & NIN) a += 2.0 * xc;
    if (m & NOUT) a += 2.0 * xc;
    return a;
}

/* b - A phi_lin, exactly (phi_lin differs by 1/nz between z neighbours and by 1/(2 nz)
 * from the inlet value 1 and the outlet value 0) */
static double rhs_lin(const Grid* g, unsigned m) {
    double t = 0.0;
    if (m & NZM) t += 1.0;
    if (m & NZP) t -= 1.0;
    if (m & NIN) t += 1.0;
    if (m & NOUT) t -= 1.0;
    return t / g->nz;
}

static double sum_planes(const double* ps, int nz) {
    double s = 0.0;
    for (int k = 0; k < nz; ++k) s += ps[k];
    return s;
}

static double max_planes(const double* ps, int nz) {
    double s = 0.0;
    for (int k = 0; k < nz; ++k) s = fmax(s, ps[k]);
    return s;
}

/* unscaled face values (psi differences, in units of phi per cell) into U, V, W; the
 * plane sums of W over fluid z-faces and their counts into ps / pc (nz + 1 planes) */
static void faces(const Grid* g, const double* x, double* U, double* V, double* W, double* ps,
                  double* pc) {
    const int nx = g->nx, ny = g->ny, nz = g->nz;
    const double dl = 1.0 / nz;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        for (int j = 0; j < ny; ++j)
            for (int a = 0; a <= nx; ++a) {
                double v = 0.0;
                if (a > 0 && a < nx) {
                    const int64_t c0 = (a - 1) + (int64_t)nx * j + g->nxny * k;
                    if (!g->solid[c0] && !g->solid[c0 + 1]) v = -(x[c0 + 1] - x[c0]);
                }
                U[a + (int64_t)(nx + 1) * (j + (int64_t)ny * k)] = v;
            }
        for (int b = 0; b <= ny; ++b)
            for (int i = 0; i < nx; ++i) {
                double v = 0.0;
                if (b > 0 && b < ny) {
                    const int64_t c0 = i + (int64_t)nx * (b - 1) + g->nxny * k;
                    if (!g->solid[c0] && !g->solid[c0 + nx]) v = -(x[c0 + nx] - x[c0]);
                }
                V[i + (int64_t)nx * (b + (int64_t)(ny + 1) * k)] = v;
            }
    }
#pragma omp parallel for schedule(static)
    for (int k = 0; k <= nz; ++k) {
        double sw = 0.0, cnt = 0.0;
        for (int64_t ij = 0; ij < g->nxny; ++ij) {
            double v = 0.0;
            int face = 0;
            if (k == 0) {
                /* phi <= 1 in the exact solution, so inflow is >= 0 */
                if (!g->solid[ij]) { v = fmax(dl - 2.0 * x[ij], 0.0); face = 1; }
            } else if (k == nz) {
                const int64_t c = ij + g->nxny * (nz - 1);
                if (!g->solid[c]) { v = fmax(dl + 2.0 * x[c], 0.0); face = 1; }
            } else {
                const int64_t c0 = ij + g->nxny * (k - 1);
                if (!g->solid[c0] && !g->solid[c0 + g->nxny]) {
                    v = dl - (x[c0 + g->nxny] - x[c0]);
                    face = 1;
                }
            }
            W[ij + g->nxny * k] = v;
            if (face) { sw += v; cnt += 1.0; }
        }
        ps[k] = sw;
        pc[k] = cnt;
    }
}

/* Returns 0 on success, 1 on bad arguments, 2 if memory ran out, 3 if the CG did not
 * reach the tolerance (the best fields found are still written). info (4 doubles):
 * iterations, max|div u| / u_mean, true residual / (mean unscaled W), superficial q.
 * nthreads <= 0 keeps the OpenMP default. */
int rfb_synth_potential_flow_cpu(int nx, int ny, int nz, double h, double u_mean, double tol,
                                 int max_iter, int check_every, const uint8_t* solid,
                                 double* U, double* V, double* W, double* info, int nthreads) {
    if (nx < 1 || ny < 1 || nz < 2 || !(h > 0) || !(u_mean > 0) || !solid || !U || !V || !W ||
        !info || check_every < 1)
        return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    Grid g;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.nxny = (int64_t)nx * ny;
    g.N = g.nxny * nz;
    g.solid = solid;
    const int64_t N = g.N;
    uint8_t* nb = (uint8_t*)malloc((size_t)N);
    double* rhs = (double*)malloc((size_t)N * 8);
    double* x = (double*)malloc((size_t)N * 8);
    double* r = (double*)malloc((size_t)N * 8);
    double* p = (double*)malloc((size_t)N * 8);
    double* q = (double*)malloc((size_t)N * 8);
    double* dinv = (double*)malloc((size_t)N * 8);
    double* ps = (double*)malloc((size_t)(nz + 1) * 8);
    double* pc = (double*)malloc((size_t)(nz + 1) * 8);
    int rc = 0;
    if (!nb || !rhs || !x || !r || !p || !q || !dinv || !ps || !pc) { rc = 2; goto done; }
    g.nb = nb;

    /* neighbour bits, rhs, x = 0, r = rhs, p = z = r / diag, plane sums of r.z */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double acc = 0.0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t c = i + (int64_t)nx * j + g.nxny * k;
                unsigned m = 0;
                if (!solid[c]) {
                    if (i > 0 && !solid[c - 1]) m |= NXM;
                    if (i + 1 < nx && !solid[c + 1]) m |= NXP;
                    if (j > 0 && !solid[c - nx]) m |= NYM;
                    if (j + 1 < ny && !solid[c + nx]) m |= NYP;
                    if (k > 0 && !solid[c - g.nxny]) m |= NZM;
                    if (k + 1 < nz && !solid[c + g.nxny]) m |= NZP;
                    if (k == 0) m |= NIN;
                    if (k == nz - 1) m |= NOUT;
                }
                nb[c] = (uint8_t)m;
                double rv = 0.0, di = 0.0;
                if (!solid[c]) {
                    rv = rhs_lin(&g, m);
                    const double d = diag_of(m);
                    di = d > 0 ? 1.0 / d : 0.0;
                }
                rhs[c] = rv;
                x[c] = 0.0;
                r[c] = rv;
                dinv[c] = di;
                p[c] = rv * di;
                acc += rv * (rv * di);
            }
        ps[k] = acc;
    }
    double rz = sum_planes(ps, nz);
    int it = 0;
    double best = INFINITY;
    int since_best = 0;
    int converged = 0;
    while (it < max_iter) {
        for (int s = 0; s < check_every && it < max_iter; ++s, ++it) {
            /* q = A p, plane sums of p.q */
#pragma omp parallel for schedule(static)
            for (int k = 0; k < nz; ++k) {
                double acc = 0.0;
                const int64_t c0 = g.nxny * k;
                for (int64_t c = c0; c < c0 + g.nxny; ++c) {
                    const unsigned m = nb[c];
                    const double a = solid[c] ? 0.0 : apply_row(&g, p, c, m);
                    q[c] = a;
                    acc += p[c] * a;
                }
                ps[k] = acc;
            }
            const double pq = sum_planes(ps, nz);
            const double alpha = rz / pq;
            /* x += alpha p, r -= alpha q, plane sums of r.z with z = r / diag */
#pragma omp parallel for schedule(static)
            for (int k = 0; k < nz; ++k) {
                double acc = 0.0;
                const int64_t c0 = g.nxny * k;
                for (int64_t c = c0; c < c0 + g.nxny; ++c) {
                    x[c] += alpha * p[c];
                    const double rv = r[c] - alpha * q[c];
                    r[c] = rv;
                    acc += rv * (dinv[c] * rv);
                }
                ps[k] = acc;
            }
            const double rz_new = sum_planes(ps, nz);
            const double beta = rz_new / rz;
#pragma omp parallel for schedule(static)
            for (int k = 0; k < nz; ++k) {
                const int64_t c0 = g.nxny * k;
                for (int64_t c = c0; c < c0 + g.nxny; ++c) p[c] = dinv[c] * r[c] + beta * p[c];
            }
            rz = rz_new;
        }
        /* true residual max |rhs - A x| relative to the mean unscaled W */
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; ++k) {
            double mx = 0.0;
            const int64_t c0 = g.nxny * k;
            for (int64_t c = c0; c < c0 + g.nxny; ++c)
                if (!solid[c]) mx = fmax(mx, fabs(rhs[c] - apply_row(&g, x, c, nb[c])));
            ps[k] = mx;
        }
        const double tres = max_planes(ps, nz);
        faces(&g, x, U, V, W, ps, pc);
        const double wmean = sum_planes(ps, nz + 1) / sum_planes(pc, nz + 1);
        const double achieved = tres / wmean;
        info[2] = achieved;
        if (achieved < 0.5 * tol) { converged = 1; break; }
        if (achieved < 0.7 * best) { best = achieved; since_best = 0; }
        else if (++since_best >= 20) break;   /* stagnated at the rounding floor */
    }
    info[0] = it;
    faces(&g, x, U, V, W, ps, pc);
    {
        const double sc = u_mean / (sum_planes(ps, nz + 1) / sum_planes(pc, nz + 1));
        const int64_t nU = (int64_t)(nx + 1) * ny * nz, nV = (int64_t)nx * (ny + 1) * nz,
                      nW = (int64_t)nx * ny * (nz + 1);
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < nU; ++a) U[a] *= sc;
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < nV; ++a) V[a] *= sc;
#pragma omp parallel for schedule(static)
        for (int64_t a = 0; a < nW; ++a) W[a] *= sc;
    }
    /* max over fluid cells of |sum of outward face velocities|, and the superficial q */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double mx = 0.0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t c = i + (int64_t)nx * j + g.nxny * k;
                if (solid[c]) continue;
                const int64_t u0 = i + (int64_t)(nx + 1) * (j + (int64_t)ny * k);
                const int64_t v0 = i + (int64_t)nx * (j + (int64_t)(ny + 1) * k);
                const double d = (U[u0 + 1] - U[u0]) + (V[v0 + nx] - V[v0]) +
                                 (W[c + g.nxny] - W[c]);
                mx = fmax(mx, fabs(d));
            }
        ps[k] = mx;
    }
    info[1] = max_planes(ps, nz) / u_mean;
    {
        double s = 0.0;
        for (int64_t ij = 0; ij < g.nxny; ++ij) s += W[ij];
        info[3] = s / (double)g.nxny;
    }
    if (!converged && !(info[1] < tol)) rc = 3;
done:
    free(nb); free(rhs); free(x); free(r); free(p); free(q); free(dinv); free(ps); free(pc);
    (void)h;
    return rc;
}
