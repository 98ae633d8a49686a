/*
 * vbc_oracle.c -- plain FP64 CPU oracle for the valency-bounding correction (VBC).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: it exists so that the tests, the smoke check and the CPU
 * baseline of the benchmark can compare the CUDA path against a slow,
 * obviously correct restatement of the paper's definitions.  It shares no
 * code, header or constant table with the CUDA library.
 *
 * What it computes (paper "Valency-bounding correction potential for
 * coarse-grained molecular dynamics simulations", Sec. 2):
 *   - smooth step omega(x; x1, x2)                        Eq. (omega)
 *   - smoothed neighbour count n_i = sum_j omega(r_ij; r_l, r_h)   Eq. (counter)
 *   - switching factor s_i = omega(n_i; f - delta, f - delta + 1),
 *     Psi_ij = s_i s_j                                     Eqs. (Psi), (Psidelta)
 *   - corrected pair energy V_r + Psi V_a, U = sum_{i<j}   Eq. (Vhat)
 *   - polynomial soft core V_r and quartic well V_a        Eq. (softcore)
 *   - forces F = -grad U.  The paper defers the explicit force to its
 *     supplement, which is not available; the chain rule is written out here:
 *       A_i  = dU/dn_i = s'_i * sum_{j != i} s_j V_a(r_ij)
 *       g_ij = V_r'(r) + s_i s_j V_a'(r) + (A_i + A_j) omega'(r; r_l, r_h)
 *       F_i  = -sum_{j != i} g_ij (x_i - x_j) / r_ij       (minimum image)
 *     virial W = sum_{i<j} -g_ij r_ij.
 *   - one Langevin step in the BAOAB splitting (the paper uses Langevin
 *     dynamics, Sec. 2 "simulation parameters", without naming the scheme)
 *     with Gaussian noise from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the
 *     Box-Muller transform.
 *
 * Two evaluation modes: mode 0 visits all N(N-1) ordered pairs (the
 * definition); mode 1 visits the same pairs through a cell list of edge
 * >= the interaction range, only so that the CPU baseline can be timed at
 * large N.  Both produce the same sums up to rounding order; a test checks
 * mode 1 against mode 0.
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, finite differences, invariants, published Philox test vectors);
 * the multi-type evaluation also by its reduction to the single-type one.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double r_r, r_a, r_l, r_h, E_r, E_a, f, delta;
} orc_params;

/* ---------------------------------------------------------------- Eq. omega */
/* 1 for x <= x1, (1 - ((x - x1)/(x2 - x1))^2)^2 between, 0 for x >= x2. */
double orc_omega(double x, double x1, double x2)
{
    if (x <= x1) return 1.0;
    if (x >= x2) return 0.0;
    double t = (x - x1) / (x2 - x1);
    double q = 1.0 - t * t;
    return q * q;
}

/* d omega / dx: -4 t (1 - t^2) / (x2 - x1) inside the window, 0 outside. */
double orc_domega(double x, double x1, double x2)
{
    if (x <= x1 || x >= x2) return 0.0;
    double w = x2 - x1;
    double t = (x - x1) / w;
    return -4.0 * t * (1.0 - t * t) / w;
}

/* ------------------------------------------------------------ Eq. softcore */
/* V_r = E_r (1 - (r/r_r)^2)^2 for r < r_r. */
double orc_Vr(double r, const orc_params* p)
{
    if (r >= p->r_r) return 0.0;
    double q = 1.0 - (r / p->r_r) * (r / p->r_r);
    return p->E_r * q * q;
}

/* dV_r/dr = -4 E_r (r / r_r^2) (1 - (r/r_r)^2). */
double orc_dVr(double r, const orc_params* p)
{
    if (r >= p->r_r) return 0.0;
    double q = 1.0 - (r / p->r_r) * (r / p->r_r);
    return -4.0 * p->E_r * (r / (p->r_r * p->r_r)) * q;
}

/* V_a = -E_a (1 - u^2)^2, u = (r - (r_a + r_r)/2) / ((r_a - r_r)/2), r_r < r < r_a. */
double orc_Va(double r, const orc_params* p)
{
    if (r <= p->r_r || r >= p->r_a) return 0.0;
    double h = 0.5 * (p->r_a - p->r_r);
    double u = (r - 0.5 * (p->r_a + p->r_r)) / h;
    double q = 1.0 - u * u;
    return -p->E_a * q * q;
}

/* dV_a/dr = 4 E_a u (1 - u^2) / h. */
double orc_dVa(double r, const orc_params* p)
{
    if (r <= p->r_r || r >= p->r_a) return 0.0;
    double h = 0.5 * (p->r_a - p->r_r);
    double u = (r - 0.5 * (p->r_a + p->r_r)) / h;
    return 4.0 * p->E_a * u * (1.0 - u * u) / h;
}

static double orc_rcut(const orc_params* p)
{
    double c = p->r_r;
    if (p->r_a > c) c = p->r_a;
    if (p->r_h > c) c = p->r_h;
    return c;
}

/* Minimum-image separation d = x_i - x_j in a periodic orthorhombic box. */
static void orc_sep(const double* xi, const double* xj, const double box[3], double d[3])
{
    for (int a = 0; a < 3; ++a) {
        double v = xi[a] - xj[a];
        v -= box[a] * nearbyint(v / box[a]);
        d[a] = v;
    }
}

/* ------------------------------------------------------------- pair visitor */
/* The cell list of mode 1: particle indices grouped by cell. */
typedef struct {
    int nc[3];
    int64_t ncell;
    int64_t* start; /* ncell + 1 */
    int64_t* idx;   /* n */
    int* cell_of;   /* n */
} orc_cells;

static int orc_cells_build(int64_t n, const double box[3], const double* pos, double rc, orc_cells* c)
{
    for (int a = 0; a < 3; ++a) {
        c->nc[a] = (int)floor(box[a] / rc);
        if (c->nc[a] < 3) return -1;
    }
    c->ncell = (int64_t)c->nc[0] * c->nc[1] * c->nc[2];
    c->start = (int64_t*)calloc((size_t)c->ncell + 1, sizeof(int64_t));
    c->idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    c->cell_of = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            double w = pos[3 * i + a] - box[a] * floor(pos[3 * i + a] / box[a]);
            int k = (int)floor(w / box[a] * c->nc[a]);
            if (k < 0) k = 0;
            if (k >= c->nc[a]) k = c->nc[a] - 1;
            ci[a] = k;
        }
        int cell = (ci[2] * c->nc[1] + ci[1]) * c->nc[0] + ci[0];
        c->cell_of[i] = cell;
        c->start[cell + 1]++;
    }
    for (int64_t k = 0; k < c->ncell; ++k) c->start[k + 1] += c->start[k];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->ncell);
    memcpy(fill, c->start, sizeof(int64_t) * (size_t)c->ncell);
    for (int64_t i = 0; i < n; ++i) c->idx[fill[c->cell_of[i]]++] = i;
    free(fill);
    return 0;
}

static void orc_cells_free(orc_cells* c)
{
    free(c->start);
    free(c->idx);
    free(c->cell_of);
}

/* Calls visit(i, j, d, r, ctx) for every j != i with r_ij < rc. */
typedef void (*orc_visit_fn)(int64_t i, int64_t j, const double d[3], double r, void* ctx);

static void orc_for_neighbours(int64_t i, int64_t n, const double box[3], const double* pos,
                               double rc, const orc_cells* cells, orc_visit_fn visit, void* ctx)
{
    double d[3];
    if (!cells) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            orc_sep(pos + 3 * i, pos + 3 * j, box, d);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r < rc) visit(i, j, d, r, ctx);
        }
        return;
    }
    int cell = cells->cell_of[i];
    int cx = cell % cells->nc[0];
    int cy = (cell / cells->nc[0]) % cells->nc[1];
    int cz = cell / (cells->nc[0] * cells->nc[1]);
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = (cx + dx + cells->nc[0]) % cells->nc[0];
                int y = (cy + dy + cells->nc[1]) % cells->nc[1];
                int z = (cz + dz + cells->nc[2]) % cells->nc[2];
                int c2 = (z * cells->nc[1] + y) * cells->nc[0] + x;
                for (int64_t k = cells->start[c2]; k < cells->start[c2 + 1]; ++k) {
                    int64_t j = cells->idx[k];
                    if (j == i) continue;
                    orc_sep(pos + 3 * i, pos + 3 * j, box, d);
                    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    if (r < rc) visit(i, j, d, r, ctx);
                }
            }
}

/* ------------------------------------------------------------ the three sums */
typedef struct {
    const orc_params* p;
    const double* s;
    const double* A;
    double acc;      /* scalar accumulator */
    double vec[3];   /* force accumulator */
    double e, w;     /* half pair energy and half virial of particle i */
} orc_ctx;

static void visit_count(int64_t i, int64_t j, const double d[3], double r, void* vctx)
{
    (void)i; (void)j; (void)d;
    orc_ctx* c = (orc_ctx*)vctx;
    c->acc += orc_omega(r, c->p->r_l, c->p->r_h);
}

static void visit_chain(int64_t i, int64_t j, const double d[3], double r, void* vctx)
{
    (void)i; (void)d;
    orc_ctx* c = (orc_ctx*)vctx;
    c->acc += c->s[j] * orc_Va(r, c->p);
}

static void visit_force(int64_t i, int64_t j, const double d[3], double r, void* vctx)
{
    orc_ctx* c = (orc_ctx*)vctx;
    const orc_params* p = c->p;
    double g = orc_dVr(r, p) + c->s[i] * c->s[j] * orc_dVa(r, p)
             + (c->A[i] + c->A[j]) * orc_domega(r, p->r_l, p->r_h);
    if (r > 0.0) {
        for (int a = 0; a < 3; ++a) c->vec[a] -= g * d[a] / r;
    }
    /* each unordered pair is visited twice (from i and from j): take half */
    c->e += 0.5 * (orc_Vr(r, p) + c->s[i] * c->s[j] * orc_Va(r, p));
    c->w += 0.5 * (-g * r);
}

/*
 * Full evaluation.  Outputs (each may be NULL): counts n_i, s_i, s'_i, A_i,
 * F (n*3, row-major), per-particle energy e_i (half of each pair, so that
 * sum e_i = U), U, W.  mode 0 = all pairs, mode 1 = cell list (returns -1 if
 * the box holds fewer than 3 cells per axis).  Returns 0 on success.
 */
int orc_eval(int64_t n, const double* box, const double* pos, const orc_params* p, int mode,
             double* counts, double* s_out, double* ds_out, double* A_out, double* F,
             double* e_out, double* U, double* W)
{
    double rc = orc_rcut(p);
    orc_cells cells;
    orc_cells* cp = NULL;
    if (mode == 1) {
        if (orc_cells_build(n, box, pos, rc, &cells) != 0) return -1;
        cp = &cells;
    }
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* nn = (double*)malloc(sz);
    double* s = (double*)malloc(sz);
    double* ds = (double*)malloc(sz);
    double* A = (double*)malloc(sz);
    double* e = (double*)malloc(sz);
    double* w = (double*)malloc(sz);
    double lo = p->f - p->delta, hi = p->f - p->delta + 1.0;

    /* pass 1: counts, then the switching factor and its derivative (Eqs. counter, Psidelta) */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        orc_ctx c = {p, NULL, NULL, 0.0, {0, 0, 0}, 0, 0};
        orc_for_neighbours(i, n, box, pos, rc, cp, visit_count, &c);
        nn[i] = c.acc;
        s[i] = orc_omega(nn[i], lo, hi);
        ds[i] = orc_domega(nn[i], lo, hi);
    }
    /* chain-rule coefficient A_i = dU/dn_i */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        if (ds[i] == 0.0) {
            A[i] = 0.0;
            continue;
        }
        orc_ctx c = {p, s, NULL, 0.0, {0, 0, 0}, 0, 0};
        orc_for_neighbours(i, n, box, pos, rc, cp, visit_chain, &c);
        A[i] = ds[i] * c.acc;
    }
    /* pass 2: forces, pair energies, virial (Eq. Vhat) */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        orc_ctx c = {p, s, A, 0.0, {0, 0, 0}, 0, 0};
        orc_for_neighbours(i, n, box, pos, rc, cp, visit_force, &c);
        if (F) {
            F[3 * i + 0] = c.vec[0];
            F[3 * i + 1] = c.vec[1];
            F[3 * i + 2] = c.vec[2];
        }
        e[i] = c.e;
        w[i] = c.w;
    }
    double Usum = 0.0, Wsum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        Usum += e[i];
        Wsum += w[i];
    }
    if (counts) memcpy(counts, nn, sizeof(double) * (size_t)n);
    if (s_out) memcpy(s_out, s, sizeof(double) * (size_t)n);
    if (ds_out) memcpy(ds_out, ds, sizeof(double) * (size_t)n);
    if (A_out) memcpy(A_out, A, sizeof(double) * (size_t)n);
    if (e_out) memcpy(e_out, e, sizeof(double) * (size_t)n);
    if (U) *U = Usum;
    if (W) *W = Wsum;
    free(nn); free(s); free(ds); free(A); free(e); free(w);
    if (cp) orc_cells_free(cp);
    return 0;
}

/* ------------------------------------------ several particle types and bonds */
/*
 * Multi-type VBC with harmonic bonds: the count of a particle restricted to
 * selected neighbour types (Sec. 2, where the counter may run over chosen
 * types only) and the bead-spring sticker chains of Sec. 4.  Type t_i is in
 * [0, ntypes).  The pair (i, j) uses the potential parameters
 * P[t_i][t_j] (r_r, r_a, r_l, r_h, E_r, E_a; P symmetric), a type's
 * valency and threshold shift are P[t][t].f and P[t][t].delta, and the
 * count of i takes the pair only if cmask[t_i][t_j] != 0:
 *   n_i  = sum_{j != i, cmask[t_i][t_j]} omega(r_ij; r_l^{ij}, r_h^{ij})
 *   s_i  = omega(n_i; f_{t_i} - delta_{t_i}, f_{t_i} - delta_{t_i} + 1)
 *   U    = sum_{i<j} [V_r^{ij} + s_i s_j V_a^{ij}] + sum_bonds k_b/2 (r - r_0)^2
 *   A_i  = dU/dn_i = s'_i sum_{j != i} s_j V_a^{ij}
 *   g_ij = V_r' + s_i s_j V_a' + (cmask[t_i][t_j] A_i + cmask[t_j][t_i] A_j) omega'^{ij}
 * (A_i enters through n_i, which holds the pair only when cmask[t_i][t_j]
 * is set.)  A bond (i, j) adds k_b (r - r_0) to g_ij; bonded pairs keep
 * their non-bonded terms.  With one type, cmask = 1 and no bonds this is
 * orc_eval.
 */
typedef struct {
    const orc_params* P; /* [ntypes][ntypes] */
    const int* cmask;    /* [ntypes][ntypes] */
    const int32_t* type;
    int ntypes;
    const double* s;
    const double* A;
    double acc;
    double vec[3];
    double e, w;
} orc_tctx;

static const orc_params* orc_pair(const orc_tctx* c, int64_t i, int64_t j)
{
    return c->P + (size_t)c->type[i] * c->ntypes + c->type[j];
}

static int orc_counts_pair(const orc_tctx* c, int64_t i, int64_t j)
{
    return c->cmask[(size_t)c->type[i] * c->ntypes + c->type[j]] != 0;
}

static void tvisit_count(int64_t i, int64_t j, const double d[3], double r, void* vctx)
{
    (void)d;
    orc_tctx* c = (orc_tctx*)vctx;
    if (!orc_counts_pair(c, i, j)) return;
    const orc_params* p = orc_pair(c, i, j);
    c->acc += orc_omega(r, p->r_l, p->r_h);
}

static void tvisit_chain(int64_t i, int64_t j, const double d[3], double r, void* vctx)
{
    (void)d;
    orc_tctx* c = (orc_tctx*)vctx;
    c->acc += c->s[j] * orc_Va(r, orc_pair(c, i, j));
}

static void tvisit_force(int64_t i, int64_t j, const double d[3], double r, void* vctx)
{
    orc_tctx* c = (orc_tctx*)vctx;
    const orc_params* p = orc_pair(c, i, j);
    double chain = (orc_counts_pair(c, i, j) ? c->A[i] : 0.0) + (orc_counts_pair(c, j, i) ? c->A[j] : 0.0);
    double g = orc_dVr(r, p) + c->s[i] * c->s[j] * orc_dVa(r, p) + chain * orc_domega(r, p->r_l, p->r_h);
    if (r > 0.0) {
        for (int a = 0; a < 3; ++a) c->vec[a] -= g * d[a] / r;
    }
    c->e += 0.5 * (orc_Vr(r, p) + c->s[i] * c->s[j] * orc_Va(r, p));
    c->w += 0.5 * (-g * r);
}

/*
 * Full typed evaluation.  type [n], P and cmask [ntypes * ntypes] row-major,
 * bonds [nbonds][2] particle indices (each bond once), k_b and r_0 the
 * harmonic bond constants.  Outputs as in orc_eval (each may be NULL).
 * Returns 0, -1 if the cell list does not fit the box (mode 1), -2 for a type
 * or bond index out of range.
 */
int orc_eval_typed(int64_t n, const double* box, const double* pos, const int32_t* type, int ntypes,
                   const orc_params* P, const int* cmask, int64_t nbonds, const int64_t* bonds,
                   double k_b, double r_0, int mode, double* counts, double* s_out, double* ds_out,
                   double* A_out, double* F, double* e_out, double* U, double* W)
{
    if (ntypes < 1) return -2;
    for (int64_t i = 0; i < n; ++i)
        if (type[i] < 0 || type[i] >= ntypes) return -2;
    for (int64_t b = 0; b < 2 * nbonds; ++b)
        if (bonds[b] < 0 || bonds[b] >= n) return -2;
    double rc = 0.0;
    for (int k = 0; k < ntypes * ntypes; ++k) {
        double c = orc_rcut(P + k);
        if (c > rc) rc = c;
    }
    orc_cells cells;
    orc_cells* cp = NULL;
    if (mode == 1) {
        if (orc_cells_build(n, box, pos, rc, &cells) != 0) return -1;
        cp = &cells;
    }
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* nn = (double*)malloc(sz);
    double* s = (double*)malloc(sz);
    double* ds = (double*)malloc(sz);
    double* A = (double*)malloc(sz);
    double* e = (double*)malloc(sz);
    double* w = (double*)malloc(sz);
    double* Fl = (double*)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));

    /* counts over the selected neighbour types, then each particle's own switch */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        orc_tctx c = {P, cmask, type, ntypes, NULL, NULL, 0.0, {0, 0, 0}, 0, 0};
        orc_for_neighbours(i, n, box, pos, rc, cp, tvisit_count, &c);
        const orc_params* own = P + (size_t)type[i] * ntypes + type[i];
        double lo = own->f - own->delta;
        nn[i] = c.acc;
        s[i] = orc_omega(nn[i], lo, lo + 1.0);
        ds[i] = orc_domega(nn[i], lo, lo + 1.0);
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        if (ds[i] == 0.0) {
            A[i] = 0.0;
            continue;
        }
        orc_tctx c = {P, cmask, type, ntypes, s, NULL, 0.0, {0, 0, 0}, 0, 0};
        orc_for_neighbours(i, n, box, pos, rc, cp, tvisit_chain, &c);
        A[i] = ds[i] * c.acc;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        orc_tctx c = {P, cmask, type, ntypes, s, A, 0.0, {0, 0, 0}, 0, 0};
        orc_for_neighbours(i, n, box, pos, rc, cp, tvisit_force, &c);
        for (int a = 0; a < 3; ++a) Fl[3 * i + a] = c.vec[a];
        e[i] = c.e;
        w[i] = c.w;
    }
    /* harmonic bonds, one after another: each gives -k_b (r - r_0) d / r to i and the opposite to j */
    for (int64_t b = 0; b < nbonds; ++b) {
        int64_t i = bonds[2 * b], j = bonds[2 * b + 1];
        double d[3];
        orc_sep(pos + 3 * i, pos + 3 * j, box, d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double g = k_b * (r - r_0);
        if (r > 0.0) {
            for (int a = 0; a < 3; ++a) {
                Fl[3 * i + a] -= g * d[a] / r;
                Fl[3 * j + a] += g * d[a] / r;
            }
        }
        double eb = 0.5 * k_b * (r - r_0) * (r - r_0);
        e[i] += 0.5 * eb;
        e[j] += 0.5 * eb;
        w[i] += 0.5 * (-g * r);
        w[j] += 0.5 * (-g * r);
    }
    double Usum = 0.0, Wsum = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        Usum += e[i];
        Wsum += w[i];
    }
    if (F) memcpy(F, Fl, 3 * sizeof(double) * (size_t)n);
    if (counts) memcpy(counts, nn, sizeof(double) * (size_t)n);
    if (s_out) memcpy(s_out, s, sizeof(double) * (size_t)n);
    if (ds_out) memcpy(ds_out, ds, sizeof(double) * (size_t)n);
    if (A_out) memcpy(A_out, A, sizeof(double) * (size_t)n);
    if (e_out) memcpy(e_out, e, sizeof(double) * (size_t)n);
    if (U) *U = Usum;
    if (W) *W = Wsum;
    free(nn); free(s); free(ds); free(A); free(e); free(w); free(Fl);
    if (cp) orc_cells_free(cp);
    return 0;
}

/* All unordered pairs (i < j) closer than rcut, brute force.  Writes up to
 * cap pairs into pairs[2*k], returns the total number found. */
int64_t orc_pairs_within(int64_t n, const double* box, const double* pos, double rcut,
                         int64_t* pairs, int64_t cap)
{
    int64_t found = 0;
    double d[3];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            orc_sep(pos + 3 * i, pos + 3 * j, box, d);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < rcut * rcut) {
                if (found < cap) {
                    pairs[2 * found] = i;
                    pairs[2 * found + 1] = j;
                }
                ++found;
            }
        }
    return found;
}

/* ------------------------------------------------------- Philox4x32-10 (SC'11) */
/* One round: two 32x32->64 products of counter words 0 and 2 with the
 * round multipliers; the high halves are mixed with the other counter words
 * and the key, the low halves pass through. */
static void orc_philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

/* Ten rounds; the key is advanced by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        orc_philox_round(c, k);
    }
    memcpy(out, c, sizeof(c));
}

/*
 * Three standard normals for particle `id` at step `step` under `seed`:
 * counter (step lo, step hi, id, 0), key (seed lo, seed hi); each 32-bit word
 * x becomes u = ((x >> 9) + 1/2) / 2^23 in (0, 1) (exact in binary32 and
 * binary64), and Box-Muller maps (u0, u1) -> (z0, z1), (u2, u3) -> z2.
 */
void orc_normals(uint64_t seed, uint64_t step, uint32_t id, double z[3])
{
    uint32_t ctr[4] = {(uint32_t)step, (uint32_t)(step >> 32), id, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u[4];
    for (int a = 0; a < 4; ++a) u[a] = ((double)(x[a] >> 9) + 0.5) / 8388608.0;
    const double two_pi = 6.283185307179586476925286766559;
    double r0 = sqrt(-2.0 * log(u[0]));
    double r1 = sqrt(-2.0 * log(u[2]));
    z[0] = r0 * cos(two_pi * u[1]);
    z[1] = r0 * sin(two_pi * u[1]);
    z[2] = r1 * cos(two_pi * u[3]);
}

/*
 * BAOAB Langevin steps (unit mass): B half kick, A half drift, O exact
 * Ornstein-Uhlenbeck update v <- c1 v + sqrt((1 - c1^2) kT) xi with
 * c1 = exp(-gamma dt), A half drift, new force, B half kick.  The noise of
 * the step taken from state counter `step` uses that counter; `step` is
 * advanced by nsteps.  pos/vel are n*3 row-major, unwrapped positions.
 */
int orc_baoab(int64_t n, const double* box, double* pos, double* vel, const orc_params* p,
              int mode, int64_t nsteps, double dt, double kT, double gamma, uint64_t seed,
              int64_t* step)
{
    double* F = (double*)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (orc_eval(n, box, pos, p, mode, NULL, NULL, NULL, NULL, F, NULL, NULL, NULL) != 0) {
        free(F);
        return -1;
    }
    double c1 = exp(-gamma * dt);
    double c2 = sqrt((1.0 - c1 * c1) * kT);
    for (int64_t k = 0; k < nsteps; ++k) {
        for (int64_t i = 0; i < n; ++i) {
            double z[3];
            orc_normals(seed, (uint64_t)*step, (uint32_t)i, z);
            for (int a = 0; a < 3; ++a) {
                double v = vel[3 * i + a] + 0.5 * dt * F[3 * i + a];
                double x = pos[3 * i + a] + 0.5 * dt * v;
                v = c1 * v + c2 * z[a];
                x += 0.5 * dt * v;
                vel[3 * i + a] = v;
                pos[3 * i + a] = x;
            }
        }
        if (orc_eval(n, box, pos, p, mode, NULL, NULL, NULL, NULL, F, NULL, NULL, NULL) != 0) {
            free(F);
            return -1;
        }
        for (int64_t i = 0; i < 3 * n; ++i) vel[i] += 0.5 * dt * F[i];
        *step += 1;
    }
    free(F);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
