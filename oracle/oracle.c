/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the short-range MD hot path
 * of MDcraft (arXiv 2511.22951).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * CUDA product path never links, calls or reads it; it shares no code,
 * header, table or constant with the CUDA sources.
 *
 * Compiled with -O2 -ffp-contract=off so that every floating-point
 * operation below is rounded exactly as written (no fused multiply-add).
 *
 * What is computed (each function cites the passage it follows):
 *   - Verlet neighbour set within r_ns = rc + skin       (Sec. "Neighbor lists
 *     construction", Eq. rhrz: r_ns = (1+beta) r_cut; absolute skin reading)
 *       * brute force over every atom and every periodic image (definition)
 *       * the paper's algorithm: bucket sort of atoms into a virtual grid of
 *         cells of size >= R, then a 3x3x3 cell stencil
 *   - Lennard-Jones energy / force / virial               (Sec. "Potentials
 *     support": f_i = sum_j V'(r_ij) r_ji / r_ji)
 *   - EAM energy / force / virial from tabulated functions (Sec. "Comparison of
 *     aluminum shock Hugoniot ...": single-element EAM read from a table; the
 *     standard embedded-atom form U = 1/2 sum phi + sum F(rho_i))
 *   - velocity-Verlet NVE integration                     (Sec. "Molecular
 *     dynamics", Eq. MD-system: m_i r_i'' = f_i = -grad_i U)
 *   - per-bin profiles of the Appendix (mass, COM velocity, temperature per
 *     degree of freedom, pressure tensor with the virial term)
 *   - the moving window's rules (Sec. "Moving window simulation")
 *   - the gradient of the EAM energy and forces with respect to the table
 *     knots, in reverse mode and (independently) forward mode
 *   - Langevin thermostat regions (Sec. "Molecular dynamics" and "Moving
 *     window simulation") with the Philox4x64-10 counter-based generator
 *   - the Behler-Parrinello potential (Sec. "Molecular dynamics with
 *     Behler-Parrinello neural networks"): symmetry functions G1-G5, the
 *     atomic network, forces by Eq. force (see the BPNN section below)
 *
 * Readings of the paper that this file fixes:
 *   * pair vector d_ij = (x_j - x_i) + n*L, rounded in that order;
 *     r^2 = (dx*dx + dy*dy) + dz*dz; a pair is a neighbour iff r^2 < r_ns^2;
 *   * the neighbour list is a full list over (j, image n) with (j,n) != (i,0);
 *   * LJ is cut at rc with an energy shift (shift_mode 1), plain truncation
 *     (0) or shifted force (2);
 *   * EAM tables are cubic Hermite splines through the knot values, knot
 *     slopes from 3-point differences (one-sided 3-point at both ends);
 *     r >= rc gives 0; rho > rho_max is extrapolated linearly and flagged;
 *   * positions of periodic dimensions are wrapped into [lo, lo+L) at every
 *     list rebuild, by whole box lengths.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* 1 eV/(Angstrom u) in Angstrom/fs^2 (e / u / 1e-10 m * 1e-20). */
static const double ORA_ACC = 9.648533212331e-3;

typedef struct {
    double lo[3];
    double L[3];
    int per[3];
} ora_box;

static ora_box make_box(const double *lo, const double *hi, const int *per) {
    ora_box b;
    for (int d = 0; d < 3; ++d) {
        b.lo[d] = lo[d];
        b.L[d] = hi[d] - lo[d];
        b.per[d] = per[d] ? 1 : 0;
    }
    return b;
}

/* ---------------------------------------------------------------------- */
/* pair geometry                                                           */
/* ---------------------------------------------------------------------- */

/* d = (xj - xi) + n*L per component; returns r^2 = (dx^2 + dy^2) + dz^2. */
static double pair_vec(const double *xi, const double *xj, const int n[3],
                       const ora_box *b, double d[3]) {
    for (int k = 0; k < 3; ++k) {
        double t = xj[k] - xi[k];
        double s = (double)n[k] * b->L[k];
        d[k] = t + s;
    }
    double r2 = d[0] * d[0];
    r2 = r2 + d[1] * d[1];
    r2 = r2 + d[2] * d[2];
    return r2;
}

/* Images n of dimension k that can bring |t + n L| below rcut (with a tiny
 * outward margin so that rounding never hides a candidate). */
static void image_range(double t, const ora_box *b, int k, double rcut,
                        int *nlo, int *nhi) {
    if (!b->per[k]) {
        *nlo = 0;
        *nhi = 0;
        return;
    }
    double L = b->L[k];
    double m = rcut * (1.0 + 1e-9) + 1e-12;
    *nlo = (int)ceil((-m - t) / L) - 1;
    *nhi = (int)floor((m - t) / L) + 1;
}

/* ---------------------------------------------------------------------- */
/* neighbour set by brute force: the definition                           */
/* ---------------------------------------------------------------------- */

/*
 * For every atom i (in input order) append every (j, n) with
 * r^2 < rns^2 and (j,n) != (i,0); j ascending, then images lexicographic.
 * offsets[N+1] always written; entries written only while < cap.
 * Returns the total number of entries.  (Sec. "Neighbor lists construction":
 * the list holds the atoms within the search radius r_ns.)
 */
int64_t ora_neighbors_brute(int64_t N, const double *x, const double *lo,
                            const double *hi, const int *per, double rns,
                            int64_t *offsets, int32_t *jout, int32_t *nout,
                            int64_t cap) {
    ora_box b = make_box(lo, hi, per);
    double r2c = rns * rns;
    int64_t cnt = 0;
    for (int64_t i = 0; i < N; ++i) {
        offsets[i] = cnt;
        const double *xi = x + 3 * i;
        for (int64_t j = 0; j < N; ++j) {
            const double *xj = x + 3 * j;
            int lo_[3], hi_[3];
            for (int k = 0; k < 3; ++k)
                image_range(xj[k] - xi[k], &b, k, rns, &lo_[k], &hi_[k]);
            int n[3];
            for (n[0] = lo_[0]; n[0] <= hi_[0]; ++n[0])
                for (n[1] = lo_[1]; n[1] <= hi_[1]; ++n[1])
                    for (n[2] = lo_[2]; n[2] <= hi_[2]; ++n[2]) {
                        if (j == i && n[0] == 0 && n[1] == 0 && n[2] == 0)
                            continue;
                        double d[3];
                        double r2 = pair_vec(xi, xj, n, &b, d);
                        if (r2 < r2c) {
                            if (cnt < cap) {
                                jout[cnt] = (int32_t)j;
                                nout[3 * cnt + 0] = n[0];
                                nout[3 * cnt + 1] = n[1];
                                nout[3 * cnt + 2] = n[2];
                            }
                            ++cnt;
                        }
                    }
        }
    }
    offsets[N] = cnt;
    return cnt;
}

/* ---------------------------------------------------------------------- */
/* wrapping and the paper's cell-list algorithm                            */
/* ---------------------------------------------------------------------- */

/* Wrap periodic coordinates into [lo, lo+L) by whole box lengths. */
void ora_wrap(int64_t N, double *x, const double *lo, const double *hi,
              const int *per) {
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) {
            if (!per[k]) continue;
            double L = hi[k] - lo[k];
            double v = x[3 * i + k];
            while (v >= hi[k]) v = v - L;
            while (v < lo[k]) v = v + L;
            if (v >= hi[k]) v = lo[k]; /* only via rounding at the upper edge */
            x[3 * i + k] = v;
        }
}

typedef struct {
    int nc[3];        /* cells per dimension                            */
    double glo[3];    /* grid origin                                    */
    double h[3];      /* cell size                                      */
    int64_t ncell;
    int64_t *start;   /* ncell + 1                                      */
    int64_t *atoms;   /* N, atom indices bucket-sorted by cell          */
} ora_grid;

/*
 * Virtual Cartesian grid of cells of size >= R over the domain, and a
 * one-pass bucket sort of the atoms into it (Sec. "Neighbor lists
 * construction").  Periodic dimensions: nc = floor(L/R) cells of size L/nc.
 * Free dimensions: the grid spans the atoms' extent at build time.
 */
static int grid_build(ora_grid *g, int64_t N, const double *x, const ora_box *b,
                      double R) {
    for (int k = 0; k < 3; ++k) {
        double glo, ext;
        if (b->per[k]) {
            glo = b->lo[k];
            ext = b->L[k];
        } else {
            double mn = INFINITY, mx = -INFINITY;
            for (int64_t i = 0; i < N; ++i) {
                double v = x[3 * i + k];
                if (v < mn) mn = v;
                if (v > mx) mx = v;
            }
            if (N == 0) { mn = 0.0; mx = 0.0; }
            glo = mn;
            ext = (mx - mn) + 1e-9;
        }
        /* the 1e-10 margin keeps h strictly above R, so that one rounding
         * of (x - lo)/h cannot separate two atoms closer than R by 2 cells */
        int nc = (int)floor(ext / (R * (1.0 + 1e-10)));
        if (nc < 1) nc = 1;
        g->nc[k] = nc;
        g->glo[k] = glo;
        g->h[k] = ext / nc;
    }
    g->ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    g->start = (int64_t *)calloc((size_t)g->ncell + 1, sizeof(int64_t));
    g->atoms = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    int64_t *cell_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
    if (!g->start || !g->atoms || !cell_of) return -1;
    for (int64_t i = 0; i < N; ++i) {
        int64_t c[3];
        for (int k = 0; k < 3; ++k) {
            int64_t ck = (int64_t)floor((x[3 * i + k] - g->glo[k]) / g->h[k]);
            if (ck < 0) ck = 0;
            if (ck >= g->nc[k]) ck = g->nc[k] - 1;
            c[k] = ck;
        }
        cell_of[i] = c[0] + (int64_t)g->nc[0] * (c[1] + (int64_t)g->nc[1] * c[2]);
        g->start[cell_of[i] + 1] += 1;
    }
    for (int64_t c = 0; c < g->ncell; ++c) g->start[c + 1] += g->start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)g->ncell);
    if (!fill) return -1;
    memcpy(fill, g->start, sizeof(int64_t) * (size_t)g->ncell);
    for (int64_t i = 0; i < N; ++i) g->atoms[fill[cell_of[i]]++] = i;
    free(fill);
    free(cell_of);
    return 0;
}

static void grid_free(ora_grid *g) {
    free(g->start);
    free(g->atoms);
    g->start = NULL;
    g->atoms = NULL;
}

/* Verlet list in CSR form: for atom i, entries [off[i], off[i+1]). */
typedef struct {
    int64_t *off;
    int32_t *j;
    int32_t *n;   /* 3 per entry */
    int64_t cap;
} ora_vlist;

static int vlist_push(ora_vlist *vl, int64_t *cnt, int32_t j, const int n[3]) {
    if (*cnt >= vl->cap) {
        int64_t nc = vl->cap ? 2 * vl->cap : 1024;
        int32_t *nj = (int32_t *)realloc(vl->j, sizeof(int32_t) * (size_t)nc);
        if (!nj) return -1;
        vl->j = nj;
        int32_t *nn = (int32_t *)realloc(vl->n, sizeof(int32_t) * 3 * (size_t)nc);
        if (!nn) return -1;
        vl->n = nn;
        vl->cap = nc;
    }
    vl->j[*cnt] = j;
    vl->n[3 * *cnt + 0] = n[0];
    vl->n[3 * *cnt + 1] = n[1];
    vl->n[3 * *cnt + 2] = n[2];
    ++*cnt;
    return 0;
}

/*
 * The paper's neighbour search: for the cell of atom i, visit the 3x3x3
 * block of cells around it and keep the atoms within r_ns.  Each stencil
 * offset s is one distinct periodic image of the visited cell, so grids with
 * fewer than 3 cells in a periodic dimension still give every (j, image)
 * exactly once (a stencil position that wraps onto the same cell is another
 * image of it).  Free dimensions skip stencil cells outside the grid.
 */
/* the list entries of atom i (appended to vl at *cnt) */
static int vlist_atom(ora_vlist *vl, int64_t *cnt, int64_t i, const double *x,
                      const ora_box *b, const ora_grid *g, double r2c) {
    const double *xi = x + 3 * i;
    int ci[3];
    for (int k = 0; k < 3; ++k) {
        int64_t ck = (int64_t)floor((xi[k] - g->glo[k]) / g->h[k]);
        if (ck < 0) ck = 0;
        if (ck >= g->nc[k]) ck = g->nc[k] - 1;
        ci[k] = (int)ck;
    }
    int s[3];
    for (s[2] = -1; s[2] <= 1; ++s[2])
        for (s[1] = -1; s[1] <= 1; ++s[1])
            for (s[0] = -1; s[0] <= 1; ++s[0]) {
                int cj[3], n[3], skip = 0;
                for (int k = 0; k < 3; ++k) {
                    int c = ci[k] + s[k];
                    if (b->per[k]) {
                        /* n = floor(c / nc); cell = c - n nc */
                        int q = (c >= 0) ? c / g->nc[k] : -((-c + g->nc[k] - 1) / g->nc[k]);
                        n[k] = q;
                        cj[k] = c - q * g->nc[k];
                    } else {
                        if (c < 0 || c >= g->nc[k]) skip = 1;
                        n[k] = 0;
                        cj[k] = c;
                    }
                }
                if (skip) continue;
                int64_t c = cj[0] + (int64_t)g->nc[0] * (cj[1] + (int64_t)g->nc[1] * cj[2]);
                /* image n of cell cj seen from ci: positions were wrapped,
                 * so the image shift in box lengths is the cell wrap count */
                for (int64_t q = g->start[c]; q < g->start[c + 1]; ++q) {
                    int64_t j = g->atoms[q];
                    if (j == i && n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
                    double d[3];
                    double r2 = pair_vec(xi, x + 3 * j, n, b, d);
                    if (r2 < r2c)
                        if (vlist_push(vl, cnt, (int32_t)j, n) != 0) return -1;
                }
            }
    return 0;
}

static int vlist_build(ora_vlist *vl, int64_t N, const double *x,
                       const ora_box *b, double rns) {
    ora_grid g;
    if (grid_build(&g, N, x, b, rns) != 0) return -1;
    double r2c = rns * rns;
    int64_t cnt = 0;
    for (int64_t i = 0; i < N; ++i) {
        vl->off[i] = cnt;
        if (vlist_atom(vl, &cnt, i, x, b, &g, r2c) != 0) {
            grid_free(&g);
            return -1;
        }
    }
    vl->off[N] = cnt;
    grid_free(&g);
    return 0;
}

/*
 * Cell-list neighbour set (the paper's algorithm) for positions that are
 * already inside the primary box on periodic dimensions.  Same output
 * format as ora_neighbors_brute (the order within a list differs).
 */
int64_t ora_neighbors_cells(int64_t N, const double *x, const double *lo,
                            const double *hi, const int *per, double rns,
                            int64_t *offsets, int32_t *jout, int32_t *nout,
                            int64_t cap) {
    ora_box b = make_box(lo, hi, per);
    for (int k = 0; k < 3; ++k)
        if (b.per[k] && b.L[k] < rns) return -1;
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = offsets;
    if (vlist_build(&vl, N, x, &b, rns) != 0) return -2;
    int64_t tot = offsets[N];
    for (int64_t q = 0; q < tot && q < cap; ++q) {
        jout[q] = vl.j[q];
        nout[3 * q + 0] = vl.n[3 * q + 0];
        nout[3 * q + 1] = vl.n[3 * q + 1];
        nout[3 * q + 2] = vl.n[3 * q + 2];
    }
    free(vl.j);
    free(vl.n);
    return tot;
}

/* ---------------------------------------------------------------------- */
/* tabulated functions: cubic Hermite spline through knot values           */
/* ---------------------------------------------------------------------- */

/* Knot slopes dy/dx from 3-point differences; one-sided 3-point at the ends. */
void ora_spline_slopes(const double *y, int n, double h, double *m) {
    if (n < 3) {
        for (int k = 0; k < n; ++k) m[k] = (n == 2) ? (y[1] - y[0]) / h : 0.0;
        return;
    }
    m[0] = (-3.0 * y[0] + 4.0 * y[1] - y[2]) / (2.0 * h);
    for (int k = 1; k < n - 1; ++k) m[k] = (y[k + 1] - y[k - 1]) / (2.0 * h);
    m[n - 1] = (3.0 * y[n - 1] - 4.0 * y[n - 2] + y[n - 3]) / (2.0 * h);
}

/*
 * Hermite evaluation on the knot grid x_k = k h, k = 0..n-1:
 *   u = x/h, k = min(floor(u), n-2), t = u - k,
 *   y = h00 y_k + h10 h m_k + h01 y_{k+1} + h11 h m_{k+1}.
 * Valid for 0 <= x <= (n-1) h; callers handle the outside.
 */
static double spline_eval(const double *y, const double *m, int n, double h,
                          double x, double *dydx) {
    double u = x / h;
    int k = (int)floor(u);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    double t = u - (double)k;
    double t2 = t * t, t3 = t2 * t;
    double h00 = 2.0 * t3 - 3.0 * t2 + 1.0;
    double h10 = t3 - 2.0 * t2 + t;
    double h01 = -2.0 * t3 + 3.0 * t2;
    double h11 = t3 - t2;
    double d00 = 6.0 * t2 - 6.0 * t;
    double d10 = 3.0 * t2 - 4.0 * t + 1.0;
    double d01 = -6.0 * t2 + 6.0 * t;
    double d11 = 3.0 * t2 - 2.0 * t;
    double yk = y[k], yk1 = y[k + 1], mk = h * m[k], mk1 = h * m[k + 1];
    if (dydx) *dydx = (d00 * yk + d10 * mk + d01 * yk1 + d11 * mk1) / h;
    return h00 * yk + h10 * mk + h01 * yk1 + h11 * mk1;
}

/* Exported for the spline pins: evaluate n_x points through ora_spline_slopes. */
void ora_spline_eval_many(const double *y, int n, double h, int64_t nx,
                          const double *xs, double *val, double *der) {
    double *m = (double *)malloc(sizeof(double) * (size_t)n);
    ora_spline_slopes(y, n, h, m);
    for (int64_t q = 0; q < nx; ++q) val[q] = spline_eval(y, m, n, h, xs[q], &der[q]);
    free(m);
}

/* A radial table on [0, rc]: value and derivative, 0 for r >= rc. */
typedef struct {
    const double *y;
    double *m;
    int n;
    double h;
    double xmax;
} ora_table;

static void table_init(ora_table *t, const double *y, int n, double xmax) {
    t->y = y;
    t->n = n;
    t->xmax = xmax;
    t->h = xmax / (double)(n - 1);
    t->m = (double *)malloc(sizeof(double) * (size_t)n);
    ora_spline_slopes(y, n, t->h, t->m);
}

static double radial(const ora_table *t, double r, double *d) {
    if (r >= t->xmax) {
        *d = 0.0;
        return 0.0;
    }
    return spline_eval(t->y, t->m, t->n, t->h, r, d);
}

/* Embedding F(rho): spline on [0, rho_max]; linear extrapolation above. */
static double embed(const ora_table *t, double rho, double *d, int *flag) {
    if (rho > t->xmax) {
        double d0;
        double f0 = spline_eval(t->y, t->m, t->n, t->h, t->xmax, &d0);
        *d = d0;
        if (flag) *flag = 1;
        return f0 + d0 * (rho - t->xmax);
    }
    return spline_eval(t->y, t->m, t->n, t->h, rho, d);
}

/* ---------------------------------------------------------------------- */
/* potentials                                                              */
/* ---------------------------------------------------------------------- */

typedef struct {
    int kind;              /* 0 = LJ, 1 = EAM, 2 = BPNN (model set separately) */
    /* LJ */
    double eps, sigma, rc;
    int shift_mode;
    double u_rc, du_rc;
    /* EAM */
    ora_table phi, rho, F;
} ora_pot;

static double lj_u(const ora_pot *p, double r, double *du) {
    double sr = p->sigma / r;
    double s2 = sr * sr;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    *du = -24.0 * p->eps * (2.0 * s12 - s6) / r;
    return 4.0 * p->eps * (s12 - s6);
}

static void pot_lj_init(ora_pot *p, double eps, double sigma, double rc, int mode) {
    memset(p, 0, sizeof(*p));
    p->kind = 0;
    p->eps = eps;
    p->sigma = sigma;
    p->rc = rc;
    p->shift_mode = mode;
    double du;
    double u = lj_u(p, rc, &du);
    p->u_rc = (mode >= 1) ? u : 0.0;
    p->du_rc = (mode == 2) ? du : 0.0;
}

/* LJ pair term with its truncation: value and dV/dr for r < rc. */
static double lj_pair(const ora_pot *p, double r, double *dv) {
    double du;
    double u = lj_u(p, r, &du);
    *dv = du - p->du_rc;
    return u - p->u_rc - (r - p->rc) * p->du_rc;
}

static void pot_eam_init(ora_pot *p, int nr, double rc, const double *phi,
                         const double *rho, int nrho, double rho_max,
                         const double *F) {
    memset(p, 0, sizeof(*p));
    p->kind = 1;
    p->rc = rc;
    table_init(&p->phi, phi, nr, rc);
    table_init(&p->rho, rho, nr, rc);
    table_init(&p->F, F, nrho, rho_max);
}

static double bpnn_rc(void);

/* BPNN: only the cutoff lives here; the model is the one set last */
static void pot_bpnn_init(ora_pot *p) {
    memset(p, 0, sizeof(*p));
    p->kind = 2;
    p->rc = bpnn_rc();
}

static void pot_free(ora_pot *p) {
    if (p->kind == 1) {
        free(p->phi.m);
        free(p->rho.m);
        free(p->F.m);
    }
}

/*
 * Energy, forces and virial from an explicit pair list (CSR over atoms,
 * entries (j, n)).  f_i = sum_j V'(r_ij) d_ij / r_ij with d_ij = r_j - r_i
 * (Sec. "Potentials support"); virial W^{ab} = 1/2 sum_i sum_j r_ij^a f_ij^b
 * with r_ij = r_i - r_j and f_ij the force on i from j (Appendix, read with
 * the pair force).  EAM: rho_i = sum_j rho(r_ij), U = 1/2 sum phi + sum F(rho_i),
 * f_i = sum_j [phi'(r) + (F'(rho_i) + F'(rho_j)) rho'(r)] d_ij / r.
 * Per-atom outputs may be NULL.  Returns a bitmask: 1 = rho above the F table.
 */
static int bpnn_from_list(int64_t N, const double *x, const ora_box *b, const int64_t *off,
                          const int32_t *jl, const int32_t *nl, double *E, double *F,
                          double *W, double *Ea, double *Wa, double *G_out,
                          double *dEdG_out);

/* EAM pass 1 for atom i: rho_i = sum_j rho(r_ij); returns F(rho_i), sets
 * *dF = F'(rho_i) and *fl (1: rho above the F table) */
static double eam_embed_atom(const ora_pot *p, int64_t i, const double *x, const ora_box *b,
                             const int64_t *off, const int32_t *jl, const int32_t *nl,
                             double *rho_out, double *dF, int *fl) {
    double rc2 = p->rc * p->rc;
    double rho_i = 0.0;
    for (int64_t q = off[i]; q < off[i + 1]; ++q) {
        double d[3];
        double r2 = pair_vec(x + 3 * i, x + 3 * (int64_t)jl[q], nl + 3 * q, b, d);
        if (r2 < rc2) {
            double dr;
            rho_i += radial(&p->rho, sqrt(r2), &dr);
        }
    }
    *fl = 0;
    *rho_out = rho_i;
    return embed(&p->F, rho_i, dF, fl);
}

/* the pair sums of atom i: force fi, energy ei (half of each pair), virial wi */
static void pair_atom(const ora_pot *p, int64_t i, const double *x, const ora_box *b,
                      const int64_t *off, const int32_t *jl, const int32_t *nl,
                      const double *fp, double fi[3], double *ei_out, double wi[6]) {
    double rc2 = p->rc * p->rc;
    double ei = 0.0;
    fi[0] = fi[1] = fi[2] = 0.0;
    for (int c = 0; c < 6; ++c) wi[c] = 0.0;
    for (int64_t q = off[i]; q < off[i + 1]; ++q) {
        int64_t j = jl[q];
        double d[3];
        double r2 = pair_vec(x + 3 * i, x + 3 * j, nl + 3 * q, b, d);
        if (!(r2 < rc2)) continue;
        double r = sqrt(r2);
        double v, dv;
        if (p->kind == 0) {
            v = lj_pair(p, r, &dv);
        } else {
            double dphi, drho;
            v = radial(&p->phi, r, &dphi);
            radial(&p->rho, r, &drho);
            dv = dphi + (fp[i] + fp[j]) * drho;
        }
        ei += 0.5 * v;
        double s = dv / r;
        double f[3] = {s * d[0], s * d[1], s * d[2]};
        fi[0] += f[0];
        fi[1] += f[1];
        fi[2] += f[2];
        /* r_ij = -d */
        wi[0] += 0.5 * (-d[0]) * f[0];
        wi[1] += 0.5 * (-d[1]) * f[1];
        wi[2] += 0.5 * (-d[2]) * f[2];
        wi[3] += 0.5 * (-d[0]) * f[1];
        wi[4] += 0.5 * (-d[0]) * f[2];
        wi[5] += 0.5 * (-d[1]) * f[2];
    }
    *ei_out = ei;
}

static int forces_from_list(const ora_pot *p, int64_t N, const double *x,
                            const ora_box *b, const int64_t *off,
                            const int32_t *jl, const int32_t *nl, double *E,
                            double *F, double *W, double *Ea, double *Wa,
                            double *rho_out, double *fp_out) {
    if (p->kind == 2)   /* BPNN: the model set by ora_bpnn_set_model */
        return bpnn_from_list(N, x, b, off, jl, nl, E, F, W, Ea, Wa, NULL, NULL);
    int flag = 0;
    double Etot = 0.0;
    double Wt[6] = {0, 0, 0, 0, 0, 0};
    double *fp = NULL;
    if (p->kind == 1) {
        fp = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
        /* pass 1: densities, embedding energy and F'(rho_i) */
        for (int64_t i = 0; i < N; ++i) {
            int fl;
            double rho_i, dF;
            double Fi = eam_embed_atom(p, i, x, b, off, jl, nl, &rho_i, &dF, &fl);
            flag |= fl;
            fp[i] = dF;
            if (rho_out) rho_out[i] = rho_i;
            if (fp_out) fp_out[i] = dF;
            if (Ea) Ea[i] = Fi;
            Etot += Fi;
        }
    }
    for (int64_t i = 0; i < N; ++i) {
        double fi[3], ei, wi[6];
        pair_atom(p, i, x, b, off, jl, nl, fp, fi, &ei, wi);
        if (F) {
            F[3 * i + 0] = fi[0];
            F[3 * i + 1] = fi[1];
            F[3 * i + 2] = fi[2];
        }
        if (Ea) Ea[i] = (p->kind == 1 ? Ea[i] : 0.0) + ei;
        if (Wa)
            for (int c = 0; c < 6; ++c) Wa[6 * i + c] = wi[c];
        Etot += ei;
        for (int c = 0; c < 6; ++c) Wt[c] += wi[c];
    }
    if (E) *E = Etot;
    if (W)
        for (int c = 0; c < 6; ++c) W[c] = Wt[c];
    free(fp);
    return flag;
}

/* full brute-force list (helper for the all-pairs evaluations) */
static int brute_list(int64_t N, const double *x, const ora_box *b, double rcut,
                      ora_vlist *vl) {
    double r2c = rcut * rcut;
    int64_t cnt = 0;
    for (int64_t i = 0; i < N; ++i) {
        vl->off[i] = cnt;
        for (int64_t j = 0; j < N; ++j) {
            int lo_[3], hi_[3];
            for (int k = 0; k < 3; ++k)
                image_range(x[3 * j + k] - x[3 * i + k], b, k, rcut, &lo_[k], &hi_[k]);
            int n[3];
            for (n[0] = lo_[0]; n[0] <= hi_[0]; ++n[0])
                for (n[1] = lo_[1]; n[1] <= hi_[1]; ++n[1])
                    for (n[2] = lo_[2]; n[2] <= hi_[2]; ++n[2]) {
                        if (j == i && n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
                        double d[3];
                        if (pair_vec(x + 3 * i, x + 3 * j, n, b, d) < r2c)
                            if (vlist_push(vl, &cnt, (int32_t)j, n) != 0) return -1;
                    }
        }
    }
    vl->off[N] = cnt;
    return 0;
}

/* LJ by brute force over all pairs and images (the definition). */
int ora_lj(int64_t N, const double *x, const double *lo, const double *hi,
           const int *per, double eps, double sigma, double rc, int shift_mode,
           double *E, double *F, double *W, double *Ea, double *Wa) {
    ora_box b = make_box(lo, hi, per);
    ora_pot p;
    pot_lj_init(&p, eps, sigma, rc, shift_mode);
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (brute_list(N, x, &b, rc, &vl) != 0) return -1;
    int fl = forces_from_list(&p, N, x, &b, vl.off, vl.j, vl.n, E, F, W, Ea, Wa, NULL, NULL);
    free(vl.off);
    free(vl.j);
    free(vl.n);
    return fl;
}

/* EAM by brute force over all pairs and images (the definition). */
int ora_eam(int64_t N, const double *x, const double *lo, const double *hi,
            const int *per, int nr, double rc, const double *phi,
            const double *rho, int nrho, double rho_max, const double *Ftab,
            double *E, double *F, double *W, double *Ea, double *Wa,
            double *rho_out, double *fp_out) {
    ora_box b = make_box(lo, hi, per);
    ora_pot p;
    pot_eam_init(&p, nr, rc, phi, rho, nrho, rho_max, Ftab);
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (brute_list(N, x, &b, rc, &vl) != 0) return -1;
    int fl = forces_from_list(&p, N, x, &b, vl.off, vl.j, vl.n, E, F, W, Ea, Wa,
                              rho_out, fp_out);
    free(vl.off);
    free(vl.j);
    free(vl.n);
    pot_free(&p);
    return fl;
}

/*
 * Force and energy of selected atoms only, by brute force over all j and
 * images (for parity spot checks on systems too large for all pairs).
 * kind 0 = LJ (params: eps, sigma, rc, shift_mode); kind 1 = EAM.
 * For EAM, rho of the selected atom and of each of its neighbours is itself
 * summed over all atoms.
 */
int ora_sampled(int kind, int64_t N, const double *x, const double *lo,
                const double *hi, const int *per, const double *lj_par,
                int nr, double rc_eam, const double *phi, const double *rho,
                int nrho, double rho_max, const double *Ftab, int64_t nsel,
                const int64_t *sel, double *Fsel, double *Esel) {
    ora_box b = make_box(lo, hi, per);
    ora_pot p;
    if (kind == 0)
        pot_lj_init(&p, lj_par[0], lj_par[1], lj_par[2], (int)lj_par[3]);
    else
        pot_eam_init(&p, nr, rc_eam, phi, rho, nrho, rho_max, Ftab);
    double rc = p.rc, rc2 = rc * rc;
    int flag = 0;
    /* collect the (j, n) within rc of one atom */
    int64_t cap = 4096;
    int32_t *js = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t *ns = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)cap);
    for (int64_t q = 0; q < nsel; ++q) {
        int64_t i = sel[q];
        const double *xi = x + 3 * i;
        int64_t cnt = 0;
        for (int64_t j = 0; j < N; ++j) {
            int lo_[3], hi_[3];
            for (int k = 0; k < 3; ++k)
                image_range(x[3 * j + k] - xi[k], &b, k, rc, &lo_[k], &hi_[k]);
            int n[3];
            for (n[0] = lo_[0]; n[0] <= hi_[0]; ++n[0])
                for (n[1] = lo_[1]; n[1] <= hi_[1]; ++n[1])
                    for (n[2] = lo_[2]; n[2] <= hi_[2]; ++n[2]) {
                        if (j == i && n[0] == 0 && n[1] == 0 && n[2] == 0) continue;
                        double d[3];
                        if (pair_vec(xi, x + 3 * j, n, &b, d) < rc2) {
                            if (cnt == cap) {
                                cap *= 2;
                                js = (int32_t *)realloc(js, sizeof(int32_t) * (size_t)cap);
                                ns = (int32_t *)realloc(ns, sizeof(int32_t) * 3 * (size_t)cap);
                            }
                            js[cnt] = (int32_t)j;
                            ns[3 * cnt] = n[0];
                            ns[3 * cnt + 1] = n[1];
                            ns[3 * cnt + 2] = n[2];
                            ++cnt;
                        }
                    }
        }
        double fpi = 0.0, Fi_emb = 0.0;
        double *fpj = NULL;
        if (kind == 1) {
            /* rho_i, then rho_j of every neighbour j by its own all-atom sum */
            double rho_i = 0.0;
            for (int64_t c = 0; c < cnt; ++c) {
                double d[3], dr;
                double r2 = pair_vec(xi, x + 3 * (int64_t)js[c], ns + 3 * c, &b, d);
                rho_i += radial(&p.rho, sqrt(r2), &dr);
            }
            int fl = 0;
            Fi_emb = embed(&p.F, rho_i, &fpi, &fl);
            flag |= fl;
            fpj = (double *)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
            for (int64_t c = 0; c < cnt; ++c) {
                const double *xj = x + 3 * (int64_t)js[c];
                double rho_j = 0.0;
                for (int64_t k2 = 0; k2 < N; ++k2) {
                    int lo2[3], hi2[3];
                    for (int k = 0; k < 3; ++k)
                        image_range(x[3 * k2 + k] - xj[k], &b, k, rc, &lo2[k], &hi2[k]);
                    int n[3];
                    for (n[0] = lo2[0]; n[0] <= hi2[0]; ++n[0])
                        for (n[1] = lo2[1]; n[1] <= hi2[1]; ++n[1])
                            for (n[2] = lo2[2]; n[2] <= hi2[2]; ++n[2]) {
                                if (k2 == js[c] && n[0] == 0 && n[1] == 0 && n[2] == 0)
                                    continue;
                                double d[3], dr;
                                double r2 = pair_vec(xj, x + 3 * k2, n, &b, d);
                                if (r2 < rc2) rho_j += radial(&p.rho, sqrt(r2), &dr);
                            }
                }
                int fl2 = 0;
                embed(&p.F, rho_j, &fpj[c], &fl2);
                flag |= fl2;
            }
        }
        double fi[3] = {0, 0, 0}, ei = 0.0;
        for (int64_t c = 0; c < cnt; ++c) {
            double d[3];
            double r2 = pair_vec(xi, x + 3 * (int64_t)js[c], ns + 3 * c, &b, d);
            double r = sqrt(r2), v, dv;
            if (kind == 0) {
                v = lj_pair(&p, r, &dv);
            } else {
                double dphi, drho;
                v = radial(&p.phi, r, &dphi);
                radial(&p.rho, r, &drho);
                dv = dphi + (fpi + fpj[c]) * drho;
            }
            ei += 0.5 * v;
            double s = dv / r;
            fi[0] += s * d[0];
            fi[1] += s * d[1];
            fi[2] += s * d[2];
        }
        free(fpj);
        Fsel[3 * q + 0] = fi[0];
        Fsel[3 * q + 1] = fi[1];
        Fsel[3 * q + 2] = fi[2];
        if (Esel) Esel[q] = ei + Fi_emb;
    }
    free(js);
    free(ns);
    pot_free(&p);
    return flag;
}

/* ---------------------------------------------------------------------- */
/* velocity-Verlet MD with Verlet lists (the paper's algorithm)            */
/* ---------------------------------------------------------------------- */

/*
 * NVE integration (Sec. "Molecular dynamics": conventional Verlet, here in
 * velocity form):  v += dt/2 a;  x += dt v;  [rebuild list if needed];
 * a = f/m;  v += dt/2 a.   Accelerations a = f/m * ORA_ACC (Angstrom/fs^2).
 *
 * The Verlet list (search radius rc + skin) is rebuilt when the largest
 * displacement since the last build exceeds skin/2 (rebuild_every = 0), or
 * every rebuild_every steps.  Every rebuild wraps periodic coordinates into
 * the primary box and bins the atoms into cells of size >= rc + skin (Sec.
 * "Neighbor lists construction").
 *
 * Piston atoms (piston[i] != 0, may be NULL) move rigidly: v = (u_p, 0, 0)
 * and x += u_p dt; they ignore forces (reading of the piston boundary of the
 * shock problems).
 *
 * thermo (may be NULL) receives per step: K, U, W_xx+W_yy+W_zz.
 * Returns the number of list builds (>= 1) or a negative error code.
 */
/* ---------------------------------------------------------------------- */
/* Langevin thermostat (Sec. "Molecular dynamics": a Langevin force added to  */
/* the right-hand side of Eq. MD-system gives NVT; Sec. "Moving window        */
/* simulation": thermostats with a target temperature, a target mean         */
/* velocity and a stiffness beta, acting in regions along x)                  */
/* ---------------------------------------------------------------------- */

/*
 * Philox4x64-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten rounds of
 * two 64x64 -> 128-bit multiplications on the counter, the key bumped by
 * the Weyl constants between rounds.
 */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void ora_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static const double ORA_KB = 8.617333262e-5; /* eV/K */

/*
 * Regions along x, each with a target temperature T, a target mean velocity
 * u and a stiffness beta (1/fs).  Reading (the paper gives no formula): at
 * every force evaluation of a step, an atom in a region (first r with
 * x_lo <= x < x_hi at the new positions, piston atoms excluded) gets
 *   F += -beta m (v - u) / A  +  sigma (xi - 1/2),
 *   sigma = sqrt(24 beta m k_B T / (dt A))
 * per component, with v its half-step velocity, A = ORA_ACC, and xi uniform
 * on [0, 1): output d of Philox4x64-10 with counter (atom id, step, 0, 0)
 * and key (seed, 0), xi = (out >> 11) 2^-53.  (Uniform noise with the
 * variance 2 beta m k_B T / (dt A) of the Gaussian one.)  For a free
 * particle this velocity-Verlet discretisation leaves the full-step
 * velocities with variance exactly k_B T A / m.
 */
typedef struct {
    int n;
    double xlo[8], xhi[8], T[8], u[8][3], beta[8];
    uint64_t seed;
    int64_t step0;
    const int64_t *ids;
} ora_langevin;

static void langevin_forces(const ora_langevin *lg, int64_t N, const double *x,
                            const double *v, const double *mass, const uint8_t *piston,
                            double dt, int64_t step, double *F) {
    for (int64_t i = 0; i < N; ++i) {
        if (piston && piston[i]) continue;
        int r = -1;
        for (int q = 0; q < lg->n && r < 0; ++q)
            if (x[3 * i] >= lg->xlo[q] && x[3 * i] < lg->xhi[q]) r = q;
        if (r < 0) continue;
        uint64_t ctr[4] = {(uint64_t)lg->ids[i], (uint64_t)step, 0, 0};
        uint64_t key[2] = {lg->seed, 0};
        uint64_t out[4];
        ora_philox4x64(ctr, key, out);
        double m = mass[i], beta = lg->beta[r];
        double kT = ORA_KB * lg->T[r];
        double sigma = sqrt(24.0 * beta * m * kT / (dt * ORA_ACC));
        for (int k = 0; k < 3; ++k) {
            double xi = (double)(out[k] >> 11) * 0x1.0p-53;
            double fr = -beta * m * (v[3 * i + k] - lg->u[r][k]) / ORA_ACC;
            double fn = sigma * (xi - 0.5);
            F[3 * i + k] = F[3 * i + k] + fr + fn;
        }
    }
}

static int64_t md_run_impl(int64_t N, double *x, double *v, const double *mass,
                           const double *lo, const double *hi, const int *per,
                           int kind, const double *lj_par, int nr, double rc_eam,
                           const double *phi, const double *rho, int nrho,
                           double rho_max, const double *Ftab, double skin, double dt,
                           int64_t nsteps, int rebuild_every, const uint8_t *piston,
                           double u_p, double *thermo, double *F_out,
                           const ora_langevin *lg) {
    ora_box b = make_box(lo, hi, per);
    ora_pot p;
    if (kind == 0)
        pot_lj_init(&p, lj_par[0], lj_par[1], lj_par[2], (int)lj_par[3]);
    else if (kind == 2)
        pot_bpnn_init(&p);
    else
        pot_eam_init(&p, nr, rc_eam, phi, rho, nrho, rho_max, Ftab);
    if (kind == 2 && !(p.rc > 0.0)) return -3;
    double rns = p.rc + skin;
    for (int k = 0; k < 3; ++k)
        if (b.per[k] && b.L[k] < rns) return -1;
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    double *xref = (double *)malloc(sizeof(double) * 3 * (size_t)(N > 0 ? N : 1));
    int64_t nbuild = 0;
    double half_skin2 = 0.25 * skin * skin;

    ora_wrap(N, x, lo, hi, per);
    if (vlist_build(&vl, N, x, &b, rns) != 0) return -2;
    memcpy(xref, x, sizeof(double) * 3 * (size_t)N);
    ++nbuild;
    double E, W[6];
    forces_from_list(&p, N, x, &b, vl.off, vl.j, vl.n, &E, F, W, NULL, NULL, NULL, NULL);

    for (int64_t step = 0; step < nsteps; ++step) {
        for (int64_t i = 0; i < N; ++i) {
            if (piston && piston[i]) {
                v[3 * i + 0] = u_p;
                v[3 * i + 1] = 0.0;
                v[3 * i + 2] = 0.0;
            } else {
                double c = 0.5 * dt * ORA_ACC / mass[i];
                for (int k = 0; k < 3; ++k) v[3 * i + k] += c * F[3 * i + k];
            }
            for (int k = 0; k < 3; ++k) x[3 * i + k] += dt * v[3 * i + k];
        }
        int rebuild = 0;
        if (rebuild_every > 0) {
            rebuild = ((step + 1) % rebuild_every) == 0;
        } else {
            for (int64_t i = 0; i < N && !rebuild; ++i) {
                double dx = x[3 * i] - xref[3 * i];
                double dy = x[3 * i + 1] - xref[3 * i + 1];
                double dz = x[3 * i + 2] - xref[3 * i + 2];
                double d2 = dx * dx;
                d2 = d2 + dy * dy;
                d2 = d2 + dz * dz;
                if (d2 > half_skin2) rebuild = 1;
            }
        }
        if (rebuild) {
            ora_wrap(N, x, lo, hi, per);
            if (vlist_build(&vl, N, x, &b, rns) != 0) return -2;
            memcpy(xref, x, sizeof(double) * 3 * (size_t)N);
            ++nbuild;
        }
        forces_from_list(&p, N, x, &b, vl.off, vl.j, vl.n, &E, F, W, NULL, NULL, NULL, NULL);
        if (lg) langevin_forces(lg, N, x, v, mass, piston, dt, lg->step0 + step + 1, F);
        double K = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            if (!(piston && piston[i])) {
                double c = 0.5 * dt * ORA_ACC / mass[i];
                for (int k = 0; k < 3; ++k) v[3 * i + k] += c * F[3 * i + k];
            }
            double v2 = v[3 * i] * v[3 * i];
            v2 = v2 + v[3 * i + 1] * v[3 * i + 1];
            v2 = v2 + v[3 * i + 2] * v[3 * i + 2];
            K += 0.5 * mass[i] * v2 / ORA_ACC;
        }
        if (thermo) {
            thermo[3 * step + 0] = K;
            thermo[3 * step + 1] = E;
            thermo[3 * step + 2] = W[0] + W[1] + W[2];
        }
    }
    if (F_out) memcpy(F_out, F, sizeof(double) * 3 * (size_t)N);
    free(vl.off);
    free(vl.j);
    free(vl.n);
    free(F);
    free(xref);
    pot_free(&p);
    return nbuild;
}

/* Velocity-Verlet NVE (Sec. "Molecular dynamics"); see md_run_impl. */
int64_t ora_md_run(int64_t N, double *x, double *v, const double *mass,
                   const double *lo, const double *hi, const int *per,
                   int kind, const double *lj_par, int nr, double rc_eam,
                   const double *phi, const double *rho, int nrho,
                   double rho_max, const double *Ftab, double skin, double dt,
                   int64_t nsteps, int rebuild_every, const uint8_t *piston,
                   double u_p, double *thermo, double *F_out) {
    return md_run_impl(N, x, v, mass, lo, hi, per, kind, lj_par, nr, rc_eam, phi, rho, nrho,
                       rho_max, Ftab, skin, dt, nsteps, rebuild_every, piston, u_p, thermo,
                       F_out, NULL);
}

/*
 * The same with the Langevin regions (see langevin_forces).  lang_par =
 * [n, then per region x_lo, x_hi, T, u_x, u_y, u_z, beta]; ids = permanent
 * atom ids (the generator's counter); step0 = steps done before this run.
 */
int64_t ora_md_langevin(int64_t N, double *x, double *v, const double *mass,
                        const double *lo, const double *hi, const int *per,
                        int kind, const double *lj_par, int nr, double rc_eam,
                        const double *phi, const double *rho, int nrho,
                        double rho_max, const double *Ftab, double skin, double dt,
                        int64_t nsteps, int rebuild_every, const uint8_t *piston,
                        double u_p, double *thermo, double *F_out,
                        const double *lang_par, const int64_t *ids, uint64_t seed,
                        int64_t step0) {
    ora_langevin lg;
    memset(&lg, 0, sizeof(lg));
    lg.n = (int)lang_par[0];
    if (lg.n < 0 || lg.n > 8) return -3;
    for (int q = 0; q < lg.n; ++q) {
        const double *r = lang_par + 1 + 7 * q;
        lg.xlo[q] = r[0];
        lg.xhi[q] = r[1];
        lg.T[q] = r[2];
        lg.u[q][0] = r[3];
        lg.u[q][1] = r[4];
        lg.u[q][2] = r[5];
        lg.beta[q] = r[6];
    }
    lg.seed = seed;
    lg.step0 = step0;
    lg.ids = ids;
    return md_run_impl(N, x, v, mass, lo, hi, per, kind, lj_par, nr, rc_eam, phi, rho, nrho,
                       rho_max, Ftab, skin, dt, nsteps, rebuild_every, piston, u_p, thermo,
                       F_out, &lg);
}

/* ---------------------------------------------------------------------- */
/* Threaded driver for the timed CPU baseline                             */
/* ---------------------------------------------------------------------- */

/*
 * ora_md_run_threads: the velocity-Verlet run of ora_md_run (LJ or EAM, no
 * piston or thermostat) with the per-atom work -- list search, EAM density
 * pass, pair sums, kicks and drifts, displacement test -- split into
 * contiguous atom ranges over nthreads POSIX threads.  Every per-atom value is
 * computed by the same helpers as the serial run and every total is summed in
 * the serial order, so the result equals ora_md_run bit for bit; only the
 * wall time changes.  It exists to time the oracle on all host cores.
 */
typedef struct {
    int64_t N, i0, i1;
    int phase;
    const ora_pot *p;
    const ora_box *b;
    const ora_grid *g;
    double r2c, dt, half_skin2;
    double *x, *v, *F, *xref;
    const double *mass;
    const ora_vlist *vl;
    ora_vlist lv;           /* this range's list entries (phase 1) */
    int64_t *loff;          /* this range's list offsets, local */
    double *fp, *rho, *Fi, *ei, *wi;
    int flag, trig, err;
} ora_work;

enum { PH_KICK_DRIFT = 0, PH_LIST = 1, PH_EMBED = 2, PH_PAIR = 3, PH_KICK = 4 };

static void *ora_work_run(void *arg) {
    ora_work *w = (ora_work *)arg;
    const int64_t i0 = w->i0, i1 = w->i1;
    if (w->phase == PH_KICK_DRIFT) {
        w->trig = 0;
        for (int64_t i = i0; i < i1; ++i) {
            double c = 0.5 * w->dt * ORA_ACC / w->mass[i];
            for (int k = 0; k < 3; ++k) w->v[3 * i + k] += c * w->F[3 * i + k];
            for (int k = 0; k < 3; ++k) w->x[3 * i + k] += w->dt * w->v[3 * i + k];
            double dx = w->x[3 * i] - w->xref[3 * i];
            double dy = w->x[3 * i + 1] - w->xref[3 * i + 1];
            double dz = w->x[3 * i + 2] - w->xref[3 * i + 2];
            double d2 = dx * dx;
            d2 = d2 + dy * dy;
            d2 = d2 + dz * dz;
            if (d2 > w->half_skin2) w->trig = 1;
        }
    } else if (w->phase == PH_LIST) {
        int64_t cnt = 0;
        w->err = 0;
        for (int64_t i = i0; i < i1 && !w->err; ++i) {
            w->loff[i - i0] = cnt;
            if (vlist_atom(&w->lv, &cnt, i, w->x, w->b, w->g, w->r2c) != 0) w->err = 1;
        }
        w->loff[i1 - i0] = cnt;
    } else if (w->phase == PH_EMBED) {
        w->flag = 0;
        for (int64_t i = i0; i < i1; ++i) {
            int fl;
            double rho_i, dF;
            w->Fi[i] = eam_embed_atom(w->p, i, w->x, w->b, w->vl->off, w->vl->j, w->vl->n,
                                      &rho_i, &dF, &fl);
            w->flag |= fl;
            w->fp[i] = dF;
        }
    } else if (w->phase == PH_PAIR) {
        for (int64_t i = i0; i < i1; ++i)
            pair_atom(w->p, i, w->x, w->b, w->vl->off, w->vl->j, w->vl->n, w->fp,
                      w->F + 3 * i, w->ei + i, w->wi + 6 * i);
    } else {  /* PH_KICK */
        for (int64_t i = i0; i < i1; ++i) {
            double c = 0.5 * w->dt * ORA_ACC / w->mass[i];
            for (int k = 0; k < 3; ++k) w->v[3 * i + k] += c * w->F[3 * i + k];
        }
    }
    return NULL;
}

static void ora_parallel(ora_work *w, int nt, int phase) {
    pthread_t th[256];
    for (int t = 0; t < nt; ++t) {
        w[t].phase = phase;
        if (t > 0 && pthread_create(&th[t], NULL, ora_work_run, &w[t]) != 0) {
            ora_work_run(&w[t]);
            th[t] = 0;
        }
    }
    ora_work_run(&w[0]);
    for (int t = 1; t < nt; ++t)
        if (th[t]) pthread_join(th[t], NULL);
}

/* the Verlet list of all atoms, the ranges' local lists concatenated in atom
 * order (so it equals vlist_build's) */
static int vlist_build_threads(ora_vlist *vl, ora_work *w, int nt, int64_t N, double *x,
                               const ora_box *b, double rns) {
    ora_grid g;
    if (grid_build(&g, N, x, b, rns) != 0) return -1;
    for (int t = 0; t < nt; ++t) {
        w[t].g = &g;
        w[t].x = x;
        w[t].r2c = rns * rns;
    }
    ora_parallel(w, nt, PH_LIST);
    grid_free(&g);
    int64_t tot = 0;
    for (int t = 0; t < nt; ++t) {
        if (w[t].err) return -1;
        tot += w[t].loff[w[t].i1 - w[t].i0];
    }
    if (tot > vl->cap) {
        int32_t *nj = (int32_t *)realloc(vl->j, sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
        int32_t *nn = (int32_t *)realloc(vl->n, sizeof(int32_t) * 3 * (size_t)(tot > 0 ? tot : 1));
        if (!nj || !nn) return -1;
        vl->j = nj;
        vl->n = nn;
        vl->cap = tot;
    }
    int64_t base = 0;
    for (int t = 0; t < nt; ++t) {
        const int64_t m = w[t].loff[w[t].i1 - w[t].i0];
        for (int64_t i = w[t].i0; i < w[t].i1; ++i) vl->off[i] = base + w[t].loff[i - w[t].i0];
        if (m > 0) {
            memcpy(vl->j + base, w[t].lv.j, sizeof(int32_t) * (size_t)m);
            memcpy(vl->n + 3 * base, w[t].lv.n, sizeof(int32_t) * 3 * (size_t)m);
        }
        base += m;
    }
    vl->off[N] = base;
    return 0;
}

/* forces, energy and virial as forces_from_list (same order of the sums) */
static int forces_threads(ora_work *w, int nt, const ora_pot *p, int64_t N, double *E,
                          double *W, double *Fi, double *ei, double *wi) {
    int flag = 0;
    double Etot = 0.0;
    double Wt[6] = {0, 0, 0, 0, 0, 0};
    if (p->kind == 1) {
        ora_parallel(w, nt, PH_EMBED);
        for (int t = 0; t < nt; ++t) flag |= w[t].flag;
        for (int64_t i = 0; i < N; ++i) Etot += Fi[i];
    }
    ora_parallel(w, nt, PH_PAIR);
    for (int64_t i = 0; i < N; ++i) {
        Etot += ei[i];
        for (int c = 0; c < 6; ++c) Wt[c] += wi[6 * i + c];
    }
    *E = Etot;
    for (int c = 0; c < 6; ++c) W[c] = Wt[c];
    return flag;
}

int64_t ora_md_run_threads(int64_t N, double *x, double *v, const double *mass,
                           const double *lo, const double *hi, const int *per,
                           int kind, const double *lj_par, int nr, double rc_eam,
                           const double *phi, const double *rho, int nrho,
                           double rho_max, const double *Ftab, double skin, double dt,
                           int64_t nsteps, int nthreads, double *thermo) {
    if (kind != 0 && kind != 1) return -3;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (N < nthreads) nthreads = N > 0 ? (int)N : 1;
    ora_box b = make_box(lo, hi, per);
    ora_pot p;
    if (kind == 0)
        pot_lj_init(&p, lj_par[0], lj_par[1], lj_par[2], (int)lj_par[3]);
    else
        pot_eam_init(&p, nr, rc_eam, phi, rho, nrho, rho_max, Ftab);
    double rns = p.rc + skin;
    for (int k = 0; k < 3; ++k)
        if (b.per[k] && b.L[k] < rns) return -1;
    const size_t n1 = (size_t)(N > 0 ? N : 1);
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = (int64_t *)malloc(sizeof(int64_t) * (n1 + 1));
    double *F = (double *)malloc(sizeof(double) * 3 * n1);
    double *xref = (double *)malloc(sizeof(double) * 3 * n1);
    double *fp = (double *)malloc(sizeof(double) * n1);
    double *Fi = (double *)malloc(sizeof(double) * n1);
    double *ei = (double *)malloc(sizeof(double) * n1);
    double *wi = (double *)malloc(sizeof(double) * 6 * n1);
    ora_work *w = (ora_work *)calloc((size_t)nthreads, sizeof(ora_work));
    int64_t nbuild = -2;
    if (!vl.off || !F || !xref || !fp || !Fi || !ei || !wi || !w) goto done;
    for (int t = 0; t < nthreads; ++t) {
        ora_work *q = &w[t];
        q->N = N;
        q->i0 = N * t / nthreads;
        q->i1 = N * (t + 1) / nthreads;
        q->p = &p;
        q->b = &b;
        q->dt = dt;
        q->half_skin2 = 0.25 * skin * skin;
        q->x = x;
        q->v = v;
        q->F = F;
        q->xref = xref;
        q->mass = mass;
        q->vl = &vl;
        q->loff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(q->i1 - q->i0 + 1));
        q->fp = fp;
        q->Fi = Fi;
        q->ei = ei;
        q->wi = wi;
        if (!q->loff) goto done;
    }
    nbuild = 0;
    ora_wrap(N, x, lo, hi, per);
    if (vlist_build_threads(&vl, w, nthreads, N, x, &b, rns) != 0) { nbuild = -2; goto done; }
    memcpy(xref, x, sizeof(double) * 3 * (size_t)N);
    ++nbuild;
    double E, W[6];
    forces_threads(w, nthreads, &p, N, &E, W, Fi, ei, wi);
    for (int64_t step = 0; step < nsteps; ++step) {
        ora_parallel(w, nthreads, PH_KICK_DRIFT);
        int rebuild = 0;
        for (int t = 0; t < nthreads; ++t) rebuild |= w[t].trig;
        if (rebuild) {
            ora_wrap(N, x, lo, hi, per);
            if (vlist_build_threads(&vl, w, nthreads, N, x, &b, rns) != 0) { nbuild = -2; goto done; }
            memcpy(xref, x, sizeof(double) * 3 * (size_t)N);
            ++nbuild;
        }
        forces_threads(w, nthreads, &p, N, &E, W, Fi, ei, wi);
        ora_parallel(w, nthreads, PH_KICK);
        double K = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double v2 = v[3 * i] * v[3 * i];
            v2 = v2 + v[3 * i + 1] * v[3 * i + 1];
            v2 = v2 + v[3 * i + 2] * v[3 * i + 2];
            K += 0.5 * mass[i] * v2 / ORA_ACC;
        }
        if (thermo) {
            thermo[3 * step + 0] = K;
            thermo[3 * step + 1] = E;
            thermo[3 * step + 2] = W[0] + W[1] + W[2];
        }
    }
done:
    if (w)
        for (int t = 0; t < nthreads; ++t) {
            free(w[t].loff);
            free(w[t].lv.j);
            free(w[t].lv.n);
        }
    free(w);
    free(vl.off);
    free(vl.j);
    free(vl.n);
    free(F);
    free(xref);
    free(fp);
    free(Fi);
    free(ei);
    free(wi);
    pot_free(&p);
    return nbuild;
}

/* ---------------------------------------------------------------------- */
/* Appendix: per-bin statistics                                            */
/* ---------------------------------------------------------------------- */

/*
 * Bins of width w along `axis` starting at origin (bin l covers
 * [origin + l w, origin + (l+1) w)); atoms outside [0, nbins) are ignored.
 * Output per bin, 17 values:
 *   [0] N_l  [1] M_l  [2..4] u_l (COM velocity)  [5..7] T^x, T^y, T^z
 *   [8] E_pot,l (sum of per-atom U_i)
 *   [9..14] P^{xx,yy,zz,xy,xz,yz} = (sum m du du + W_l) / V_l
 *   [15] E_kin,l (peculiar, eV)  [16] V_l
 * Temperatures: T^a = 2 E^a_kin / (k_B N_l) per degree of freedom.
 * W_l = sum over the bin's atoms of the per-atom virial Wa (6 per atom).
 * (Appendix "Analysis of MD simulation results"; virial read with the pair
 * force, see the file header.)
 */
void ora_profiles(int64_t N, const double *x, const double *v, const double *mass,
                  const double *Ua, const double *Wa, int axis, double origin,
                  double w, int nbins, double cross_area, double *out) {
    const double KB = 8.617333262e-5;
    memset(out, 0, sizeof(double) * 17 * (size_t)nbins);
    int *bin = (int *)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) {
        double u = (x[3 * i + axis] - origin) / w;
        int l = (int)floor(u);
        bin[i] = (l >= 0 && l < nbins) ? l : -1;
    }
    /* mass and momentum */
    for (int64_t i = 0; i < N; ++i) {
        int l = bin[i];
        if (l < 0) continue;
        double *o = out + 17 * l;
        o[0] += 1.0;
        o[1] += mass[i];
        for (int k = 0; k < 3; ++k) o[2 + k] += mass[i] * v[3 * i + k];
        if (Ua) o[8] += Ua[i];
    }
    for (int l = 0; l < nbins; ++l) {
        double *o = out + 17 * l;
        for (int k = 0; k < 3; ++k) o[2 + k] = (o[1] > 0.0) ? o[2 + k] / o[1] : 0.0;
        o[16] = w * cross_area;
    }
    /* peculiar kinetic tensor and virial */
    double *kt = (double *)calloc(6 * (size_t)nbins, sizeof(double));
    for (int64_t i = 0; i < N; ++i) {
        int l = bin[i];
        if (l < 0) continue;
        double *o = out + 17 * l;
        double du[3];
        for (int k = 0; k < 3; ++k) du[k] = v[3 * i + k] - o[2 + k];
        double m = mass[i] / ORA_ACC; /* u Angstrom^2/fs^2 -> eV */
        double *t = kt + 6 * l;
        t[0] += m * du[0] * du[0];
        t[1] += m * du[1] * du[1];
        t[2] += m * du[2] * du[2];
        t[3] += m * du[0] * du[1];
        t[4] += m * du[0] * du[2];
        t[5] += m * du[1] * du[2];
        if (Wa)
            for (int c = 0; c < 6; ++c) o[9 + c] += Wa[6 * i + c];
    }
    for (int l = 0; l < nbins; ++l) {
        double *o = out + 17 * l, *t = kt + 6 * l;
        double nl = o[0];
        for (int k = 0; k < 3; ++k) o[5 + k] = (nl > 0.0) ? t[k] / (KB * nl) : 0.0;
        o[15] = 0.5 * (t[0] + t[1] + t[2]);
        for (int c = 0; c < 6; ++c) o[9 + c] = (t[c] + o[9 + c]) / o[16];
    }
    free(kt);
    free(bin);
}

/* ---------------------------------------------------------------------- */
/* moving window (Sec. "Moving window simulation")                          */
/* ---------------------------------------------------------------------- */

/*
 * The window rules applied at a list build (reading of the paper's moving
 * window for a piston-driven shock along x):
 *   the shock front is found from bins of width w along x, b = floor((x -
 *   x_lo) / w) clamped to [0, nb - 1], nb = max(1, ceil((x_hi - x_lo) / w)):
 *   a bin is shocked when its mean v_x exceeds u_p / 2, decided exactly on
 *   velocities rounded to multiples of 2^-40 Angstrom/fs:
 *   2 * sum_i q(v_x,i) > n_b * q(u_p), q(v) = rint(v * 2^40);
 *   x_front = x_lo + (b* + 1) w for the largest shocked bin b* (none: no
 *   window action);
 *   atoms with x < x_front - L_behind are deleted (order of the rest kept);
 *   while the leading edge x_max < x_front + L_ahead, copies of a fresh slab
 *   are appended: copy c at x offset (x_max + gap) + c * slab_lx, velocities
 *   slab_v, ids next_id, next_id + 1, ...; k = ceil((x_front + L_ahead -
 *   x_max) / slab_lx) copies, at most floor(((x_hi - x_max) - gap) /
 *   slab_lx) (no copy starts past the box) and as many atoms as the
 *   capacity allows;
 *   atoms with x < x_min + piston_depth (x_min over the atoms left) become
 *   piston atoms.
 * With a finite fixed_front the front is that x instead (the paper's
 * stationary-shock window: outflow deletion at fixed_front - L_behind and
 * inflow layers up to fixed_front + L_ahead, whatever the velocities).
 * Returns the new atom count.
 */
int64_t ora_window_apply(int64_t N, int64_t cap, double *x, double *v, double *mass,
                         uint8_t *piston, int64_t *ids, int64_t *next_id, double x_lo,
                         double x_hi, double front_bin, double fixed_front, double u_p,
                         double L_behind,
                         double L_ahead, const double *slab_x, const double *slab_v,
                         int64_t n_slab, double slab_lx, double slab_gap, double slab_mass,
                         double piston_depth) {
    const double two40 = 1099511627776.0;
    int64_t nb = (int64_t)ceil((x_hi - x_lo) / front_bin);
    if (nb < 1) nb = 1;
    long long *S = (long long *)calloc((size_t)nb, sizeof(long long));
    long long *cnt = (long long *)calloc((size_t)nb, sizeof(long long));
    double x_max = -INFINITY;
    for (int64_t i = 0; i < N; ++i) {
        double xi = x[3 * i], vi = v[3 * i];
        if (xi > x_max) x_max = xi;
        if (!isfinite(xi) || !isfinite(vi)) continue;
        double u = floor((xi - x_lo) / front_bin);
        int64_t b = u < 0.0 ? 0 : (u > (double)(nb - 1) ? nb - 1 : (int64_t)u);
        S[b] += llrint(vi * two40);
        cnt[b] += 1;
    }
    long long q_up = llrint(u_p * two40);
    int64_t bf = -1;
    for (int64_t b = nb - 1; b >= 0; --b)
        if (cnt[b] > 0 && 2 * S[b] > cnt[b] * q_up) {
            bf = b;
            break;
        }
    free(S);
    free(cnt);
    double x_front;
    if (isfinite(fixed_front)) {
        x_front = fixed_front;  /* stationary window: boundaries fixed in the box */
    } else {
        if (bf < 0) return N;
        x_front = x_lo + (double)(bf + 1) * front_bin;
    }
    double cut = x_front - L_behind;
    int64_t n = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (x[3 * i] < cut) continue;
        if (n != i) {
            for (int k = 0; k < 3; ++k) {
                x[3 * n + k] = x[3 * i + k];
                v[3 * n + k] = v[3 * i + k];
            }
            mass[n] = mass[i];
            piston[n] = piston[i];
            ids[n] = ids[i];
        }
        ++n;
    }
    double need = x_front + L_ahead - x_max;
    int64_t copies = need > 0.0 ? (int64_t)ceil(need / slab_lx) : 0;
    double room = floor(((x_hi - x_max) - slab_gap) / slab_lx);
    int64_t fit = room > 0.0 ? (int64_t)room : 0;
    if (copies > fit) copies = fit;
    for (int64_t c = 0; c < copies; ++c) {
        double x0 = (x_max + slab_gap) + (double)c * slab_lx;
        for (int64_t q = 0; q < n_slab && n < cap; ++q) {
            x[3 * n] = slab_x[3 * q] + x0;
            x[3 * n + 1] = slab_x[3 * q + 1];
            x[3 * n + 2] = slab_x[3 * q + 2];
            for (int k = 0; k < 3; ++k) v[3 * n + k] = slab_v[3 * q + k];
            mass[n] = slab_mass;
            piston[n] = 0;
            ids[n] = (*next_id)++;
            ++n;
        }
    }
    double x_min = INFINITY;
    for (int64_t i = 0; i < n; ++i)
        if (x[3 * i] < x_min) x_min = x[3 * i];
    for (int64_t i = 0; i < n; ++i)
        if (x[3 * i] < x_min + piston_depth) piston[i] = 1;
    return n;
}

/*
 * Velocity-Verlet MD with a rigid piston and the moving window: as
 * ora_md_run with rebuilds every rebuild_every steps, the window rules
 * applied before every rebuild after the first build.  Arrays have room for
 * cap atoms; *n_io is the atom count in and out.  Returns the number of
 * builds or a negative error code.
 */
int64_t ora_md_window(int64_t *n_io, int64_t cap, double *x, double *v, double *mass,
                      uint8_t *piston, int64_t *ids, int64_t *next_id, const double *lo,
                      const double *hi, const int *per, int nr, double rc_eam,
                      const double *phi, const double *rho, int nrho, double rho_max,
                      const double *Ftab, double skin, double dt, int64_t nsteps,
                      int rebuild_every, double u_p, double front_bin, double fixed_front,
                      double L_behind, double L_ahead, const double *slab_x,
                      const double *slab_v, int64_t n_slab, double slab_lx, double slab_gap,
                      double slab_mass, double piston_depth, const double *lang_par,
                      uint64_t seed) {
    int64_t N = *n_io;
    ora_langevin lg;
    memset(&lg, 0, sizeof(lg));
    const ora_langevin *lgp = NULL;
    if (lang_par) {
        lg.n = (int)lang_par[0];
        if (lg.n < 0 || lg.n > 8) return -3;
        for (int q = 0; q < lg.n; ++q) {
            const double *r = lang_par + 1 + 7 * q;
            lg.xlo[q] = r[0];
            lg.xhi[q] = r[1];
            lg.T[q] = r[2];
            lg.u[q][0] = r[3];
            lg.u[q][1] = r[4];
            lg.u[q][2] = r[5];
            lg.beta[q] = r[6];
        }
        lg.seed = seed;
        lg.ids = ids;
        lgp = &lg;
    }
    ora_box b = make_box(lo, hi, per);
    ora_pot p;
    pot_eam_init(&p, nr, rc_eam, phi, rho, nrho, rho_max, Ftab);
    double rns = p.rc + skin;
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cap + 1));
    double *F = (double *)calloc(3 * (size_t)(cap > 0 ? cap : 1), sizeof(double));
    int64_t nbuild = 0;
    ora_wrap(N, x, lo, hi, per);
    if (vlist_build(&vl, N, x, &b, rns) != 0) return -2;
    ++nbuild;
    double E, W[6];
    forces_from_list(&p, N, x, &b, vl.off, vl.j, vl.n, &E, F, W, NULL, NULL, NULL, NULL);
    for (int64_t step = 0; step < nsteps; ++step) {
        for (int64_t i = 0; i < N; ++i) {
            if (piston[i]) {
                v[3 * i] = u_p;
                v[3 * i + 1] = 0.0;
                v[3 * i + 2] = 0.0;
            } else {
                double c = 0.5 * dt * ORA_ACC / mass[i];
                for (int k = 0; k < 3; ++k) v[3 * i + k] += c * F[3 * i + k];
            }
            for (int k = 0; k < 3; ++k) x[3 * i + k] += dt * v[3 * i + k];
        }
        if (((step + 1) % rebuild_every) == 0) {
            N = ora_window_apply(N, cap, x, v, mass, piston, ids, next_id, lo[0], hi[0],
                                 front_bin, fixed_front, u_p, L_behind, L_ahead, slab_x,
                                 slab_v, n_slab, slab_lx, slab_gap, slab_mass, piston_depth);
            ora_wrap(N, x, lo, hi, per);
            if (vlist_build(&vl, N, x, &b, rns) != 0) return -2;
            ++nbuild;
        }
        forces_from_list(&p, N, x, &b, vl.off, vl.j, vl.n, &E, F, W, NULL, NULL, NULL, NULL);
        if (lgp) langevin_forces(lgp, N, x, v, mass, piston, dt, step + 1, F);
        for (int64_t i = 0; i < N; ++i) {
            if (piston[i]) continue;
            double c = 0.5 * dt * ORA_ACC / mass[i];
            for (int k = 0; k < 3; ++k) v[3 * i + k] += c * F[3 * i + k];
        }
    }
    *n_io = N;
    free(vl.off);
    free(vl.j);
    free(vl.n);
    free(F);
    pot_free(&p);
    return nbuild;
}

/* ---------------------------------------------------------------------- */
/* adjoint of the tabulated EAM with respect to the knot values            */
/* ---------------------------------------------------------------------- */

/*
 * Loss L = gE * E + sum_i gF_i . F_i for one periodic/free system, as a
 * function of the knots theta = (phi knots, rho knots, F knots).  The spline
 * of ora_spline_eval is linear in the knot values y and the scaled slopes
 * M_k = h m_k, and M is a fixed linear map of y; derivatives with respect to
 * (y, M) are collected first and M's transpose is applied at the end.
 */

/* Hermite basis weights of value (w) and x-derivative (dw, per unit x) on
 * the interval of x: coefficients of y_k, M_k, y_{k+1}, M_{k+1}. */
static int herm_weights(int n, double h, double x, double w[4], double dw[4], double ddw[4]) {
    double u = x / h;
    int k = (int)floor(u);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    double t = u - (double)k, t2 = t * t, t3 = t2 * t;
    w[0] = 2.0 * t3 - 3.0 * t2 + 1.0;
    w[1] = t3 - 2.0 * t2 + t;
    w[2] = -2.0 * t3 + 3.0 * t2;
    w[3] = t3 - t2;
    dw[0] = (6.0 * t2 - 6.0 * t) / h;
    dw[1] = (3.0 * t2 - 4.0 * t + 1.0) / h;
    dw[2] = (-6.0 * t2 + 6.0 * t) / h;
    dw[3] = (3.0 * t2 - 2.0 * t) / h;
    if (ddw) {
        ddw[0] = (12.0 * t - 6.0) / (h * h);
        ddw[1] = (6.0 * t - 4.0) / (h * h);
        ddw[2] = (-12.0 * t + 6.0) / (h * h);
        ddw[3] = (6.0 * t - 2.0) / (h * h);
    }
    return k;
}

/* add c_v * (d value / d (y, M)) + c_d * (d derivative / d (y, M)) at x */
static void scatter_knots(int n, double h, double x, double cv, double cd, double *gy,
                          double *gM) {
    double w[4], dw[4];
    int k = herm_weights(n, h, x, w, dw, NULL);
    gy[k] += cv * w[0] + cd * dw[0];
    gM[k] += cv * w[1] + cd * dw[1];
    gy[k + 1] += cv * w[2] + cd * dw[2];
    gM[k + 1] += cv * w[3] + cd * dw[3];
}

/* transpose of M(y): interior M_k = (y_{k+1} - y_{k-1})/2, one-sided ends */
static void slope_map_T(int n, const double *gM, double *gy) {
    gy[0] += -1.5 * gM[0];
    gy[1] += 2.0 * gM[0];
    gy[2] += -0.5 * gM[0];
    for (int k = 1; k < n - 1; ++k) {
        gy[k + 1] += 0.5 * gM[k];
        gy[k - 1] -= 0.5 * gM[k];
    }
    gy[n - 1] += 1.5 * gM[n - 1];
    gy[n - 2] -= 2.0 * gM[n - 1];
    gy[n - 3] += 0.5 * gM[n - 1];
}

/* second derivative of the F spline at rho (0 beyond rho_max: linear there) */
static double embed_dd(const ora_table *t, double rho) {
    if (rho > t->xmax) return 0.0;
    double w[4], dw[4], ddw[4];
    int k = herm_weights(t->n, t->h, rho, w, dw, ddw);
    return ddw[0] * t->y[k] + ddw[1] * t->h * t->m[k] + ddw[2] * t->y[k + 1] +
           ddw[3] * t->h * t->m[k + 1];
}

/*
 * Reverse mode, written out from the chain rule with f_i = sum_j V'(r_ij) d^_ij,
 * V'(r) = phi'(r) + (F'(rho_i) + F'(rho_j)) rho'(r):
 *   phi knots: per directed pair  1/2 gE d phi(r) + (gF_i . d^_ij) d phi'(r)
 *   c_i = sum_j [(gF_i - gF_j) . d^_ij] rho'(r_ij)
 *   F knots:   per atom  gE d F(rho_i) + c_i d F'(rho_i)
 *   lambda_i = gE F'(rho_i) + c_i F''(rho_i)
 *   rho knots: per directed pair  lambda_i d rho(r) + (gF_i . d^_ij)(F'_i + F'_j) d rho'(r)
 * dtheta [nr + nr + nrho] = (phi, rho, F) knot gradients.
 */
int ora_eam_vjp(int64_t N, const double *x, const double *lo, const double *hi, const int *per,
                int nr, double rc, const double *phi, const double *rho, int nrho,
                double rho_max, const double *Ftab, double gE, const double *gF,
                double *dtheta) {
    ora_box b = make_box(lo, hi, per);
    ora_pot p;
    pot_eam_init(&p, nr, rc, phi, rho, nrho, rho_max, Ftab);
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (brute_list(N, x, &b, rc, &vl) != 0) return -1;
    double rc2 = rc * rc;
    double *rho_i = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double *fp = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double *ci = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double *gyp = (double *)calloc((size_t)nr, sizeof(double));
    double *gMp = (double *)calloc((size_t)nr, sizeof(double));
    double *gyr = (double *)calloc((size_t)nr, sizeof(double));
    double *gMr = (double *)calloc((size_t)nr, sizeof(double));
    double *gyF = (double *)calloc((size_t)nrho, sizeof(double));
    double *gMF = (double *)calloc((size_t)nrho, sizeof(double));
    /* forward: densities and F'(rho_i) */
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t q = vl.off[i]; q < vl.off[i + 1]; ++q) {
            double d[3];
            double r2 = pair_vec(x + 3 * i, x + 3 * (int64_t)vl.j[q], vl.n + 3 * q, &b, d);
            if (r2 < rc2) {
                double dr;
                rho_i[i] += radial(&p.rho, sqrt(r2), &dr);
            }
        }
        double dF;
        embed(&p.F, rho_i[i], &dF, NULL);
        fp[i] = dF;
    }
    /* c_i */
    for (int64_t i = 0; i < N; ++i)
        for (int64_t q = vl.off[i]; q < vl.off[i + 1]; ++q) {
            int64_t j = vl.j[q];
            double d[3];
            double r2 = pair_vec(x + 3 * i, x + 3 * j, vl.n + 3 * q, &b, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2), drho;
            radial(&p.rho, r, &drho);
            double g = 0.0;
            for (int k = 0; k < 3; ++k) g += (gF[3 * i + k] - gF[3 * j + k]) * d[k] / r;
            ci[i] += g * drho;
        }
    /* F knots, and lambda_i */
    double *lam = (double *)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    for (int64_t i = 0; i < N; ++i) {
        double rh = rho_i[i];
        if (rh > rho_max) {
            /* F = y_{n-1} + (M_{n-1}/h)(rho - rho_max), F' = M_{n-1}/h */
            double h = p.F.h;
            gyF[nrho - 1] += gE;
            gMF[nrho - 1] += gE * (rh - rho_max) / h + ci[i] / h;
        } else {
            scatter_knots(nrho, p.F.h, rh, gE, ci[i], gyF, gMF);
        }
        lam[i] = gE * fp[i] + ci[i] * embed_dd(&p.F, rh);
    }
    /* phi and rho knots over directed pairs */
    for (int64_t i = 0; i < N; ++i)
        for (int64_t q = vl.off[i]; q < vl.off[i + 1]; ++q) {
            int64_t j = vl.j[q];
            double d[3];
            double r2 = pair_vec(x + 3 * i, x + 3 * j, vl.n + 3 * q, &b, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            if (r >= rc) continue; /* the radial tables are 0 from rc on */
            double gd = 0.0;
            for (int k = 0; k < 3; ++k) gd += gF[3 * i + k] * d[k] / r;
            scatter_knots(nr, p.phi.h, r, 0.5 * gE, gd, gyp, gMp);
            scatter_knots(nr, p.rho.h, r, lam[i], gd * (fp[i] + fp[j]), gyr, gMr);
        }
    slope_map_T(nr, gMp, gyp);
    slope_map_T(nr, gMr, gyr);
    slope_map_T(nrho, gMF, gyF);
    memcpy(dtheta, gyp, sizeof(double) * (size_t)nr);
    memcpy(dtheta + nr, gyr, sizeof(double) * (size_t)nr);
    memcpy(dtheta + 2 * nr, gyF, sizeof(double) * (size_t)nrho);
    free(rho_i); free(fp); free(ci); free(lam);
    free(gyp); free(gMp); free(gyr); free(gMr); free(gyF); free(gMF);
    free(vl.off); free(vl.j); free(vl.n);
    pot_free(&p);
    return 0;
}

/* ---- forward mode (dual numbers): an independent derivative ----------- */

typedef struct {
    double v, d;
} dual;

static dual dmk(double v, double d) { dual r = {v, d}; return r; }
static dual dadd(dual a, dual b) { return dmk(a.v + b.v, a.d + b.d); }
static dual dmul(dual a, dual b) { return dmk(a.v * b.v, a.v * b.d + a.d * b.v); }
static dual dscale(dual a, double s) { return dmk(a.v * s, a.d * s); }

/* spline value and x-derivative with tangent knots dy: both duals (x fixed,
 * or x a dual for rho_i) */
static void dual_spline(const double *y, const double *dy, int n, double h, dual x, dual *val,
                        dual *der) {
    /* slopes of y and of dy by the same 3-point rule */
    double u = x.v / h;
    int k = (int)floor(u);
    if (k > n - 2) k = n - 2;
    if (k < 0) k = 0;
    dual t = dscale(x, 1.0 / h);
    t.v -= (double)k;
    double Mv[2], Md[2];
    for (int q = 0; q < 2; ++q) {
        int kk = k + q;
        if (kk == 0) {
            Mv[q] = 0.5 * (-3.0 * y[0] + 4.0 * y[1] - y[2]);
            Md[q] = 0.5 * (-3.0 * dy[0] + 4.0 * dy[1] - dy[2]);
        } else if (kk == n - 1) {
            Mv[q] = 0.5 * (3.0 * y[n - 1] - 4.0 * y[n - 2] + y[n - 3]);
            Md[q] = 0.5 * (3.0 * dy[n - 1] - 4.0 * dy[n - 2] + dy[n - 3]);
        } else {
            Mv[q] = 0.5 * (y[kk + 1] - y[kk - 1]);
            Md[q] = 0.5 * (dy[kk + 1] - dy[kk - 1]);
        }
    }
    dual y0 = dmk(y[k], dy[k]), y1 = dmk(y[k + 1], dy[k + 1]);
    dual M0 = dmk(Mv[0], Md[0]), M1 = dmk(Mv[1], Md[1]);
    dual t2 = dmul(t, t), t3 = dmul(t2, t);
    dual h00 = dadd(dadd(dscale(t3, 2.0), dscale(t2, -3.0)), dmk(1.0, 0.0));
    dual h10 = dadd(dadd(t3, dscale(t2, -2.0)), t);
    dual h01 = dadd(dscale(t3, -2.0), dscale(t2, 3.0));
    dual h11 = dadd(t3, dscale(t2, -1.0));
    *val = dadd(dadd(dmul(h00, y0), dmul(h10, M0)), dadd(dmul(h01, y1), dmul(h11, M1)));
    dual d00 = dadd(dscale(t2, 6.0), dscale(t, -6.0));
    dual d10 = dadd(dadd(dscale(t2, 3.0), dscale(t, -4.0)), dmk(1.0, 0.0));
    dual d01 = dadd(dscale(t2, -6.0), dscale(t, 6.0));
    dual d11 = dadd(dscale(t2, 3.0), dscale(t, -2.0));
    *der = dscale(dadd(dadd(dmul(d00, y0), dmul(d10, M0)), dadd(dmul(d01, y1), dmul(d11, M1))),
                  1.0 / h);
}

/*
 * Directional derivative of L = gE E + sum_i gF_i . F_i along the knot
 * tangent (dphi, drho, dF), by forward mode through the whole evaluation
 * (densities, embedding, forces).  Independent of ora_eam_vjp.  Requires
 * every rho_i <= rho_max.
 */
int ora_eam_jvp(int64_t N, const double *x, const double *lo, const double *hi, const int *per,
                int nr, double rc, const double *phi, const double *rho, int nrho,
                double rho_max, const double *Ftab, const double *dphi, const double *drho,
                const double *dF, double gE, const double *gF, double *out) {
    ora_box b = make_box(lo, hi, per);
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (brute_list(N, x, &b, rc, &vl) != 0) return -1;
    double rc2 = rc * rc, hr = rc / (double)(nr - 1), hF = rho_max / (double)(nrho - 1);
    dual *rh = (dual *)calloc((size_t)(N > 0 ? N : 1), sizeof(dual));
    dual *Fp = (dual *)calloc((size_t)(N > 0 ? N : 1), sizeof(dual));
    dual L = dmk(0.0, 0.0);
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t q = vl.off[i]; q < vl.off[i + 1]; ++q) {
            double d[3];
            double r2 = pair_vec(x + 3 * i, x + 3 * (int64_t)vl.j[q], vl.n + 3 * q, &b, d);
            if (!(r2 < rc2) || sqrt(r2) >= rc) continue;
            dual v, dv;
            dual_spline(rho, drho, nr, hr, dmk(sqrt(r2), 0.0), &v, &dv);
            rh[i] = dadd(rh[i], v);
        }
        if (rh[i].v > rho_max) return -2;
        dual Fv, dFv;
        dual_spline(Ftab, dF, nrho, hF, rh[i], &Fv, &dFv);
        Fp[i] = dFv;
        L = dadd(L, dscale(Fv, gE));
    }
    for (int64_t i = 0; i < N; ++i)
        for (int64_t q = vl.off[i]; q < vl.off[i + 1]; ++q) {
            int64_t j = vl.j[q];
            double d[3];
            double r2 = pair_vec(x + 3 * i, x + 3 * j, vl.n + 3 * q, &b, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            if (r >= rc) continue;
            dual pv, pd, rv, rd;
            dual_spline(phi, dphi, nr, hr, dmk(r, 0.0), &pv, &pd);
            dual_spline(rho, drho, nr, hr, dmk(r, 0.0), &rv, &rd);
            L = dadd(L, dscale(pv, 0.5 * gE));
            dual s = dadd(pd, dmul(dadd(Fp[i], Fp[j]), rd));  /* V'(r) */
            double gd = 0.0;
            for (int k = 0; k < 3; ++k) gd += gF[3 * i + k] * d[k] / r;
            L = dadd(L, dscale(s, gd));
        }
    out[0] = L.v;
    out[1] = L.d;
    free(rh);
    free(Fp);
    free(vl.off);
    free(vl.j);
    free(vl.n);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Behler-Parrinello neural-network potential (Sec. "Molecular dynamics   */
/* with Behler-Parrinello neural networks")                               */
/* ---------------------------------------------------------------------- */
/*
 * E = sum_i E_i (Eq. E_as_sum).  Atom i's input layer is a set of symmetry
 * functions of its neighbourhood N(i) (atoms, with their periodic images,
 * closer than R_c), cut off smoothly by
 *     f_c(R) = 1/2 [cos(pi R / R_c) + 1]  for R <= R_c,  0 beyond
 * (the printed form puts the "+ 1" inside the cosine; read as the standard
 * cutoff, which is the only reading with f_c(R_c) = 0).
 * Radial functions (Eqs. G1-G3):
 *     G1 = sum_j f_c(R_ij)
 *     G2 = sum_j exp(-eta (R_ij - R_s)^2) f_c(R_ij)   (read with the square of
 *          the Gaussian the paper says it takes from Behler; without it R_s
 *          would only rescale the function)
 *     G3 = sum_j cos(kappa R_ij) f_c(R_ij)
 * Angular functions (Eqs. G4, G5), over the unordered pairs {j, k} of
 * distinct neighbours of i (each angle once):
 *     G4 = 2^(1-zeta) sum (1 + lambda cos theta_ijk)^zeta
 *          exp(-eta (R_ij^2 + R_ik^2 + R_jk^2)) f_c(R_ij) f_c(R_ik) f_c(R_jk)
 *     G5 = the same without the R_jk terms.
 * Atomic network (Eq. AtomicNN, with the activations as the text states them:
 * tanh on both hidden layers, the output linear):
 *     h1 = tanh(b1 + G W01),  h2 = tanh(b2 + h1 W12),  E_i = b3 + h2 . w23.
 * Forces (Eq. force): F_k = -sum_i sum_mu dE_i/dG_mu(i) dG_mu(i)/dR_k, with
 * dE_i/dG from the network's reverse pass and dG/dR analytic.
 * Virial: atom i carries the virial of its own energy, W_i = -sum_j r_ij (x)
 * dE_i/dR_j over its neighbours j (r_ij = R_j + image - R_i), which for a
 * pair energy E_i = 1/2 sum V reduces to the pair virial used for LJ/EAM.
 */
typedef struct {
    int set;
    double rc;
    int n_rad, n_ang, H1, H2;
    int rad_kind[64];
    double rad_par[128];   /* G2: (eta, R_s); G3: (kappa, 0); G1: unused */
    int ang_kind[128];
    double ang_par[384];   /* (zeta, lambda, eta) */
    double *W01, *b1, *W12, *b2, *w23;
    double b3;
} ora_bpnn_model;

static ora_bpnn_model g_bp;

static double bpnn_rc(void) { return g_bp.set ? g_bp.rc : 0.0; }

int ora_bpnn_set_model(double rc, int n_rad, const int *rad_kind, const double *rad_par,
                       int n_ang, const int *ang_kind, const double *ang_par, int H1, int H2,
                       const double *W01, const double *b1, const double *W12,
                       const double *b2, const double *w23, double b3) {
    if (!(rc > 0.0) || n_rad < 0 || n_rad > 64 || n_ang < 0 || n_ang > 128 ||
        n_rad + n_ang < 1 || H1 < 1 || H2 < 1)
        return -1;
    free(g_bp.W01);
    free(g_bp.b1);
    free(g_bp.W12);
    free(g_bp.b2);
    free(g_bp.w23);
    memset(&g_bp, 0, sizeof(g_bp));
    int G = n_rad + n_ang;
    g_bp.rc = rc;
    g_bp.n_rad = n_rad;
    g_bp.n_ang = n_ang;
    g_bp.H1 = H1;
    g_bp.H2 = H2;
    for (int m = 0; m < n_rad; ++m) {
        g_bp.rad_kind[m] = rad_kind[m];
        g_bp.rad_par[2 * m] = rad_par[2 * m];
        g_bp.rad_par[2 * m + 1] = rad_par[2 * m + 1];
    }
    for (int m = 0; m < n_ang; ++m) {
        g_bp.ang_kind[m] = ang_kind[m];
        for (int c = 0; c < 3; ++c) g_bp.ang_par[3 * m + c] = ang_par[3 * m + c];
    }
    g_bp.W01 = (double *)malloc(sizeof(double) * (size_t)(G * H1));
    g_bp.b1 = (double *)malloc(sizeof(double) * (size_t)H1);
    g_bp.W12 = (double *)malloc(sizeof(double) * (size_t)(H1 * H2));
    g_bp.b2 = (double *)malloc(sizeof(double) * (size_t)H2);
    g_bp.w23 = (double *)malloc(sizeof(double) * (size_t)H2);
    memcpy(g_bp.W01, W01, sizeof(double) * (size_t)(G * H1));
    memcpy(g_bp.b1, b1, sizeof(double) * (size_t)H1);
    memcpy(g_bp.W12, W12, sizeof(double) * (size_t)(H1 * H2));
    memcpy(g_bp.b2, b2, sizeof(double) * (size_t)H2);
    memcpy(g_bp.w23, w23, sizeof(double) * (size_t)H2);
    g_bp.b3 = b3;
    g_bp.set = 1;
    return 0;
}

static const double ORA_PI = 3.14159265358979323846;

/* f_c(R) and its derivative */
static double bp_fc(double R, double rc, double *d) {
    if (R >= rc) {
        *d = 0.0;
        return 0.0;
    }
    double a = ORA_PI / rc;
    *d = -0.5 * a * sin(a * R);
    return 0.5 * (cos(a * R) + 1.0);
}

/* radial symmetry function m of one neighbour at R: value, derivative */
static double bp_radial(int m, double R, double *d) {
    double fd, f = bp_fc(R, g_bp.rc, &fd);
    int kind = g_bp.rad_kind[m];
    double p0 = g_bp.rad_par[2 * m], p1 = g_bp.rad_par[2 * m + 1];
    if (kind == 1) {
        *d = fd;
        return f;
    }
    if (kind == 2) {
        double t = R - p1;
        double e = exp(-p0 * t * t);
        *d = e * (-2.0 * p0 * t * f + fd);
        return e * f;
    }
    /* kind 3 */
    double c = cos(p0 * R), s = sin(p0 * R);
    *d = -p0 * s * f + c * fd;
    return c * f;
}

/*
 * Angular term of function m for the neighbours u, w of atom i (vectors
 * from i) and s = w - u: value, and the gradients with respect to u, w.
 */
static double bp_angular(int m, const double u[3], const double w[3], double gu[3],
                         double gw[3]) {
    double zeta = g_bp.ang_par[3 * m], lam = g_bp.ang_par[3 * m + 1];
    double eta = g_bp.ang_par[3 * m + 2];
    int kind = g_bp.ang_kind[m];
    double s[3] = {w[0] - u[0], w[1] - u[1], w[2] - u[2]};
    double Ru = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double Rw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double Rs = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    double dot = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
    double c = dot / (Ru * Rw);
    double base = 1.0 + lam * c;
    double A = pow(base, zeta);
    double dA = zeta * lam * pow(base, zeta - 1.0);   /* dA/dc */
    double coef = pow(2.0, 1.0 - zeta);
    double fud, fu = bp_fc(Ru, g_bp.rc, &fud);
    double fwd, fw = bp_fc(Rw, g_bp.rc, &fwd);
    double fsd = 0.0, fs = 1.0;
    double r2sum = Ru * Ru + Rw * Rw;
    if (kind == 4) {
        fs = bp_fc(Rs, g_bp.rc, &fsd);
        r2sum += Rs * Rs;
    }
    double e = exp(-eta * r2sum);
    double Y = e * fu * fw * fs;
    /* dY/dR_u, dY/dR_w, dY/dR_s (scalar, along each length) */
    double Yu = e * fw * fs * (-2.0 * eta * Ru * fu + fud);
    double Yw = e * fu * fs * (-2.0 * eta * Rw * fw + fwd);
    double Ys = kind == 4 ? e * fu * fw * (-2.0 * eta * Rs * fs + fsd) : 0.0;
    for (int k = 0; k < 3; ++k) {
        double dc_du = w[k] / (Ru * Rw) - c * u[k] / (Ru * Ru);
        double dc_dw = u[k] / (Ru * Rw) - c * w[k] / (Rw * Rw);
        double ds = kind == 4 ? Ys * s[k] / Rs : 0.0;   /* dY/ds along s */
        /* s = w - u: d/du picks -ds, d/dw picks +ds */
        gu[k] = coef * (dA * dc_du * Y + A * (Yu * u[k] / Ru - ds));
        gw[k] = coef * (dA * dc_dw * Y + A * (Yw * w[k] / Rw + ds));
    }
    return coef * A * Y;
}

/*
 * Energies, forces and virials from a CSR list of (j, image) entries (any
 * list that contains every neighbour closer than R_c; entries beyond R_c are
 * skipped).  G_out [N][G] and dEdG_out [N][G] may be NULL.
 */
static int bpnn_from_list(int64_t N, const double *x, const ora_box *b, const int64_t *off,
                          const int32_t *jl, const int32_t *nl, double *E, double *F,
                          double *W, double *Ea, double *Wa, double *G_out,
                          double *dEdG_out) {
    if (!g_bp.set) return -1;
    const int G = g_bp.n_rad + g_bp.n_ang, H1 = g_bp.H1, H2 = g_bp.H2;
    const double rc = g_bp.rc, rc2 = rc * rc;
    double Etot = 0.0, Wt[6] = {0, 0, 0, 0, 0, 0};
    if (F) memset(F, 0, sizeof(double) * 3 * (size_t)N);
    double *Gv = (double *)malloc(sizeof(double) * (size_t)G);
    double *dG = (double *)malloc(sizeof(double) * (size_t)G);
    double *h1 = (double *)malloc(sizeof(double) * (size_t)H1);
    double *h2 = (double *)malloc(sizeof(double) * (size_t)H2);
    double *d1 = (double *)malloc(sizeof(double) * (size_t)H1);
    double *d2 = (double *)malloc(sizeof(double) * (size_t)H2);
    int64_t cap = 256;
    double *u = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
    int64_t *js = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    double *g = (double *)malloc(sizeof(double) * 3 * (size_t)cap);
    for (int64_t i = 0; i < N; ++i) {
        /* the neighbourhood N(i) */
        int64_t n = 0;
        for (int64_t q = off[i]; q < off[i + 1]; ++q) {
            double d[3];
            double r2 = pair_vec(x + 3 * i, x + 3 * (int64_t)jl[q], nl + 3 * q, b, d);
            if (!(r2 < rc2)) continue;
            if (n == cap) {
                cap *= 2;
                u = (double *)realloc(u, sizeof(double) * 3 * (size_t)cap);
                js = (int64_t *)realloc(js, sizeof(int64_t) * (size_t)cap);
                g = (double *)realloc(g, sizeof(double) * 3 * (size_t)cap);
            }
            for (int k = 0; k < 3; ++k) u[3 * n + k] = d[k];
            js[n] = jl[q];
            ++n;
        }
        /* symmetry functions */
        for (int m = 0; m < G; ++m) Gv[m] = 0.0;
        for (int64_t a = 0; a < n; ++a) {
            double R = sqrt(u[3 * a] * u[3 * a] + u[3 * a + 1] * u[3 * a + 1] +
                            u[3 * a + 2] * u[3 * a + 2]);
            for (int m = 0; m < g_bp.n_rad; ++m) {
                double dd;
                Gv[m] += bp_radial(m, R, &dd);
            }
        }
        for (int64_t a = 0; a < n; ++a)
            for (int64_t c = a + 1; c < n; ++c)
                for (int m = 0; m < g_bp.n_ang; ++m) {
                    double gu[3], gw[3];
                    Gv[g_bp.n_rad + m] += bp_angular(m, u + 3 * a, u + 3 * c, gu, gw);
                }
        /* atomic network: forward, then the reverse pass to dE_i/dG */
        for (int j = 0; j < H1; ++j) {
            double z = g_bp.b1[j];
            for (int m = 0; m < G; ++m) z += Gv[m] * g_bp.W01[m * H1 + j];
            h1[j] = tanh(z);
        }
        for (int k = 0; k < H2; ++k) {
            double z = g_bp.b2[k];
            for (int j = 0; j < H1; ++j) z += h1[j] * g_bp.W12[j * H2 + k];
            h2[k] = tanh(z);
        }
        double Ei = g_bp.b3;
        for (int k = 0; k < H2; ++k) Ei += h2[k] * g_bp.w23[k];
        for (int k = 0; k < H2; ++k) d2[k] = g_bp.w23[k] * (1.0 - h2[k] * h2[k]);
        for (int j = 0; j < H1; ++j) {
            double t = 0.0;
            for (int k = 0; k < H2; ++k) t += g_bp.W12[j * H2 + k] * d2[k];
            d1[j] = t * (1.0 - h1[j] * h1[j]);
        }
        for (int m = 0; m < G; ++m) {
            double t = 0.0;
            for (int j = 0; j < H1; ++j) t += g_bp.W01[m * H1 + j] * d1[j];
            dG[m] = t;
        }
        if (G_out) memcpy(G_out + (size_t)i * G, Gv, sizeof(double) * (size_t)G);
        if (dEdG_out) memcpy(dEdG_out + (size_t)i * G, dG, sizeof(double) * (size_t)G);
        /* g_a = dE_i/dR_(j_a), Eq. force */
        for (int64_t a = 0; a < 3 * n; ++a) g[a] = 0.0;
        for (int64_t a = 0; a < n; ++a) {
            double R = sqrt(u[3 * a] * u[3 * a] + u[3 * a + 1] * u[3 * a + 1] +
                            u[3 * a + 2] * u[3 * a + 2]);
            double s = 0.0;
            for (int m = 0; m < g_bp.n_rad; ++m) {
                double dd;
                bp_radial(m, R, &dd);
                s += dG[m] * dd;
            }
            for (int k = 0; k < 3; ++k) g[3 * a + k] += s * u[3 * a + k] / R;
        }
        for (int64_t a = 0; a < n; ++a)
            for (int64_t c = a + 1; c < n; ++c)
                for (int m = 0; m < g_bp.n_ang; ++m) {
                    double gu[3], gw[3];
                    bp_angular(m, u + 3 * a, u + 3 * c, gu, gw);
                    for (int k = 0; k < 3; ++k) {
                        g[3 * a + k] += dG[g_bp.n_rad + m] * gu[k];
                        g[3 * c + k] += dG[g_bp.n_rad + m] * gw[k];
                    }
                }
        double wi[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t a = 0; a < n; ++a) {
            const double *ga = g + 3 * a, *ua = u + 3 * a;
            if (F)
                for (int k = 0; k < 3; ++k) {
                    F[3 * js[a] + k] -= ga[k];   /* -dE_i/dR_j */
                    F[3 * i + k] += ga[k];       /* dE_i/dR_i = -sum_a g_a */
                }
            wi[0] -= ua[0] * ga[0];
            wi[1] -= ua[1] * ga[1];
            wi[2] -= ua[2] * ga[2];
            wi[3] -= ua[0] * ga[1];
            wi[4] -= ua[0] * ga[2];
            wi[5] -= ua[1] * ga[2];
        }
        if (Ea) Ea[i] = Ei;
        if (Wa)
            for (int c = 0; c < 6; ++c) Wa[6 * i + c] = wi[c];
        Etot += Ei;
        for (int c = 0; c < 6; ++c) Wt[c] += wi[c];
    }
    if (E) *E = Etot;
    if (W)
        for (int c = 0; c < 6; ++c) W[c] = Wt[c];
    free(Gv);
    free(dG);
    free(h1);
    free(h2);
    free(d1);
    free(d2);
    free(u);
    free(js);
    free(g);
    return 0;
}

/* BPNN by brute force over all atoms and images within R_c (the definition). */
int ora_bpnn(int64_t N, const double *x, const double *lo, const double *hi, const int *per,
             double *E, double *F, double *W, double *Ea, double *Wa, double *G_out,
             double *dEdG_out) {
    if (!g_bp.set) return -1;
    ora_box b = make_box(lo, hi, per);
    ora_vlist vl;
    memset(&vl, 0, sizeof(vl));
    vl.off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (brute_list(N, x, &b, g_bp.rc, &vl) != 0) return -2;
    int r = bpnn_from_list(N, x, &b, vl.off, vl.j, vl.n, E, F, W, Ea, Wa, G_out, dEdG_out);
    free(vl.off);
    free(vl.j);
    free(vl.n);
    return r;
}
