/*
 * fdw_oracle.c -- plain FP64 CPU oracle for the damped acoustic wave equation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference
 * that the CUDA library is checked against.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library, and the library never calls it.
 *
 * What it computes (paper: "Devito: Towards a generic Finite Difference DSL using
 * Symbolic Python", arXiv 1609.03361):
 *   m u_tt + eta u_t - lap(u) = q                       (Sec. 5, Eq. 3)
 * discretised with central differences of order p in space (Sec. 3.1, the
 * `dx2` / `laplace` shorthands) and second order in time (Sec. 3.1, the `dt2`
 * expansion of `m*u.dt2 = u.laplace`), marched forward in time (Sec. 5.1,
 * Listing 6), its adjoint marched backward (Sec. 5.1, Listing 7), sparse
 * point-to-grid injection and grid-to-point interpolation (Sec. 5.2,
 * Listing 8) and the exact discrete FWI gradient of the forward map
 * (Sec. 5.4 "gradient test").
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *  - u_t of the damping term is the centred difference (u+ - u-)/(2 dt);
 *  - u^{-1} = u^0 = 0; step n (0..nt-2) makes u^{n+1} and then adds q^n into it;
 *    receivers record rec^n = P_r u^n for n = 0..nt-1;
 *  - injection adds dt^2 w q / (m + eta dt/2) (no 1/h^d factor);
 *  - interpolation is multilinear; the cell index is floor(x/h) clamped to
 *    [0, N-2] in physical indices (a point on the last grid line gets f = 1);
 *  - eta = sum over axes of eta_max,a (d_a/nbl)^2 with
 *    eta_max,a = 3 ln(1000) / (2 nbl h_a vmax), d_a = distance in cells into
 *    the layer along axis a;
 *  - the model is extended into the layer by repeating its edge value;
 *  - the zero halo: u = 0 outside the computational grid.
 *
 * Layout: row-major, the last axis contiguous.  3D fields are [nx][ny][nz];
 * 2D fields are [nx][nz].  Point coordinates are [npts][ndim] in metres,
 * relative to the physical origin, in the same axis order.
 *
 * Everything is double precision.  OpenMP (when compiled with -fopenmp)
 * parallelises the outermost spatial loop only; each point is computed the
 * same way for any thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int ndim;            /* 2 or 3 */
    int64_t shape[3];    /* physical points per axis (first ndim entries used) */
    double spacing[3];   /* grid spacing per axis, metres */
    int space_order;     /* p: even, 2..16 */
    int nbl;             /* absorbing-layer points added on every side */
    double dt;           /* time step, ms */
    int nt;              /* number of time samples */
} orc_setup;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_ORDER = 2, ORC_ERR_DOMAIN = 3, ORC_ERR_MEM = 4 };

/* ------------------------------------------------------------------------- */
/* Finite-difference weights                                                  */
/* ------------------------------------------------------------------------- */

static double factorial(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/*
 * Central second-derivative weights of order p (Sec. 3.1: the order of the
 * `dx2` expansion is a parameter of the symbol; for p = 2 the paper prints
 * f(x-h) - 2 f(x) + f(x+h) over h^2).  The closed form of the central weights
 * for a 2r+1 point stencil, r = p/2:
 *   c_j = 2 (-1)^(j+1) (r!)^2 / ( j^2 (r-j)! (r+j)! ),  j = 1..r
 *   c_0 = -2 sum_{j>=1} c_j      (the stencil annihilates constants)
 * c must hold r+1 doubles.  Returns ORC_ERR_ORDER for odd p or p outside 2..16.
 */
int orc_fd_weights(int p, double *c)
{
    if (p < 2 || p > 16 || (p % 2) != 0 || c == NULL) return ORC_ERR_ORDER;
    int r = p / 2;
    double rf2 = factorial(r) * factorial(r);
    double s = 0.0;
    for (int j = 1; j <= r; ++j) {
        double sign = (j % 2 == 1) ? 1.0 : -1.0;
        c[j] = 2.0 * sign * rf2 / ((double)j * (double)j * factorial(r - j) * factorial(r + j));
        s += c[j];
    }
    c[0] = -2.0 * s;
    return ORC_OK;
}

/*
 * Largest magnitude of the symbol of the 1-D second-derivative stencil
 * (times h^2), reached at the Nyquist wavenumber:
 *   S = | c_0 + 2 sum_j (-1)^j c_j |
 */
double orc_stability_sum(int p)
{
    double c[9];
    if (orc_fd_weights(p, c) != ORC_OK) return -1.0;
    double s = c[0];
    for (int j = 1; j <= p / 2; ++j) s += 2.0 * ((j % 2 == 0) ? 1.0 : -1.0) * c[j];
    return fabs(s);
}

/*
 * Leapfrog stability limit for m u_tt = lap u with the order-p Laplacian:
 *   dt_max = 2 / ( vmax sqrt( sum_a S / h_a^2 ) )
 * (von Neumann analysis of the three-level scheme of Sec. 3.1 / Sec. 5.1).
 * Returns -1 on bad arguments.
 */
double orc_dt_max(int ndim, const double *spacing, int p, double vmax)
{
    if ((ndim != 2 && ndim != 3) || spacing == NULL || vmax <= 0.0) return -1.0;
    double S = orc_stability_sum(p);
    if (S <= 0.0) return -1.0;
    double acc = 0.0;
    for (int a = 0; a < ndim; ++a) {
        if (spacing[a] <= 0.0) return -1.0;
        acc += S / (spacing[a] * spacing[a]);
    }
    return 2.0 / (vmax * sqrt(acc));
}

/* ------------------------------------------------------------------------- */
/* Grid helpers                                                               */
/* ------------------------------------------------------------------------- */

static void comp_shape(const orc_setup *s, int64_t n[3])
{
    for (int a = 0; a < 3; ++a) n[a] = 1;
    for (int a = 0; a < s->ndim; ++a) n[a] = s->shape[a] + 2 * (int64_t)s->nbl;
}

static int64_t comp_points(const orc_setup *s)
{
    int64_t n[3];
    comp_shape(s, n);
    return n[0] * n[1] * n[2];
}

static int check_setup(const orc_setup *s)
{
    if (s == NULL || (s->ndim != 2 && s->ndim != 3)) return ORC_ERR_ARG;
    if (s->space_order < 2 || s->space_order > 16 || s->space_order % 2) return ORC_ERR_ORDER;
    if (s->nbl < 0 || s->nt < 1 || !(s->dt > 0.0)) return ORC_ERR_ARG;
    for (int a = 0; a < s->ndim; ++a)
        if (s->shape[a] < 2 || !(s->spacing[a] > 0.0)) return ORC_ERR_ARG;
    return ORC_OK;
}

/* Unravel a flat index into ndim coordinates of the computational grid. */
static void unravel(int ndim, const int64_t n[3], int64_t idx, int64_t i[3])
{
    if (ndim == 3) {
        i[2] = idx % n[2]; idx /= n[2];
        i[1] = idx % n[1]; idx /= n[1];
        i[0] = idx;
    } else {
        i[1] = idx % n[1]; idx /= n[1];
        i[0] = idx;
        i[2] = 0;
    }
}

/*
 * Extend a physical-shape model into the computational grid by repeating the
 * nearest physical value (each computational index is clamped into the
 * physical range).  m_comp has the computational shape.
 */
int orc_extend_model(const orc_setup *s, const double *m_phys, double *m_comp)
{
    if (check_setup(s) != ORC_OK || !m_phys || !m_comp) return ORC_ERR_ARG;
    int64_t n[3];
    comp_shape(s, n);
    int64_t np[3] = {1, 1, 1};
    for (int a = 0; a < s->ndim; ++a) np[a] = s->shape[a];
    int64_t total = n[0] * n[1] * n[2];
    int nd = s->ndim;
    for (int64_t idx = 0; idx < total; ++idx) {
        int64_t i[3];
        unravel(nd, n, idx, i);
        int64_t src = 0;
        for (int a = 0; a < nd; ++a) {
            int64_t k = i[a] - s->nbl;
            if (k < 0) k = 0;
            if (k > np[a] - 1) k = np[a] - 1;
            src = src * np[a] + k;
        }
        m_comp[idx] = m_phys[src];
    }
    return ORC_OK;
}

/*
 * Adjoint of orc_extend_model (the gradient with respect to the physical
 * model): every computational point adds its value into the physical point
 * whose value the extension repeats there, so that for any m_phys and g_comp
 *   <extend(m_phys), g_comp> = <m_phys, fold(g_comp)>.
 * g_phys has the physical shape and is overwritten.
 */
int orc_fold_model(const orc_setup *s, const double *g_comp, double *g_phys)
{
    if (check_setup(s) != ORC_OK || !g_comp || !g_phys) return ORC_ERR_ARG;
    int64_t n[3];
    comp_shape(s, n);
    int64_t np[3] = {1, 1, 1};
    for (int a = 0; a < s->ndim; ++a) np[a] = s->shape[a];
    int64_t total = n[0] * n[1] * n[2];
    memset(g_phys, 0, sizeof(double) * (size_t)(np[0] * np[1] * np[2]));
    int nd = s->ndim;
    for (int64_t idx = 0; idx < total; ++idx) {
        int64_t i[3];
        unravel(nd, n, idx, i);
        int64_t dst = 0;
        for (int a = 0; a < nd; ++a) {
            int64_t k = i[a] - s->nbl;
            if (k < 0) k = 0;
            if (k > np[a] - 1) k = np[a] - 1;
            dst = dst * np[a] + k;
        }
        g_phys[dst] += g_comp[idx];
    }
    return ORC_OK;
}

/*
 * Damping field eta of the absorbing layer (Sec. 5, Eq. 3: "spatially varying
 * dampening factor"; Sec. 5.4: 40 layer points on each side).  Quadratic
 * profile, one term per axis, zero in the physical domain.
 */
int orc_damping(const orc_setup *s, double vmax, double *eta)
{
    if (check_setup(s) != ORC_OK || !eta || !(vmax > 0.0)) return ORC_ERR_ARG;
    int64_t n[3];
    comp_shape(s, n);
    int64_t total = n[0] * n[1] * n[2];
    int nd = s->ndim;
    for (int64_t idx = 0; idx < total; ++idx) {
        int64_t i[3];
        unravel(nd, n, idx, i);
        double e = 0.0;
        if (s->nbl > 0) {
            for (int a = 0; a < nd; ++a) {
                int64_t lo = s->nbl - i[a];                          /* cells before the first physical point */
                int64_t hi = i[a] - (s->nbl + s->shape[a] - 1);      /* cells past the last physical point */
                int64_t d = lo > 0 ? lo : (hi > 0 ? hi : 0);
                double emax = 3.0 * log(1000.0) / (2.0 * s->nbl * s->spacing[a] * vmax);
                double f = (double)d / (double)s->nbl;
                e += emax * f * f;
            }
        }
        eta[idx] = e;
    }
    return ORC_OK;
}

/*
 * Multilinear weights of sparse points (Sec. 5.2, Listing 8: a value is spread
 * over the nodes enclosing the point; the grid-to-point direction uses the same
 * nodes and weights).  For each point and each of the 2^ndim corners: the flat
 * computational index and the weight.  Corner bit order: x is the most
 * significant bit, the last axis the least.  Returns ORC_ERR_DOMAIN when a
 * coordinate lies outside [0, (N-1) h] of its axis.
 */
int orc_interp(const orc_setup *s, int npts, const double *coords, int64_t *idx, double *w)
{
    if (check_setup(s) != ORC_OK || npts < 0 || (npts > 0 && (!coords || !idx || !w))) return ORC_ERR_ARG;
    int nd = s->ndim;
    int nc = 1 << nd;
    int64_t n[3];
    comp_shape(s, n);
    for (int p = 0; p < npts; ++p) {
        int64_t base[3];
        double f[3];
        for (int a = 0; a < nd; ++a) {
            double x = coords[(int64_t)p * nd + a];
            double top = (double)(s->shape[a] - 1) * s->spacing[a];
            if (!(x >= 0.0) || !(x <= top)) return ORC_ERR_DOMAIN;
            double xi = x / s->spacing[a];
            int64_t i = (int64_t)floor(xi);
            if (i < 0) i = 0;
            if (i > s->shape[a] - 2) i = s->shape[a] - 2;
            base[a] = i + s->nbl;
            f[a] = xi - (double)i;
        }
        for (int c = 0; c < nc; ++c) {
            double wt = 1.0;
            int64_t flat = 0;
            for (int a = 0; a < nd; ++a) {
                int bit = (c >> (nd - 1 - a)) & 1;
                wt *= bit ? f[a] : (1.0 - f[a]);
                flat = flat * n[a] + base[a] + bit;
            }
            idx[(int64_t)p * nc + c] = flat;
            w[(int64_t)p * nc + c] = wt;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Time stepping                                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    int nd;
    int r;
    int64_t n[3];       /* computational shape (unused axes = 1) */
    int64_t total;
    double w[3][9];     /* per-axis weights c_k / h_a^2 */
    double dt;
    const double *m;
    const double *eta;
} stepper;

static int make_stepper(const orc_setup *s, const double *m, const double *eta, stepper *st)
{
    int rc = check_setup(s);
    if (rc != ORC_OK) return rc;
    if (!m || !eta) return ORC_ERR_ARG;
    st->nd = s->ndim;
    st->r = s->space_order / 2;
    comp_shape(s, st->n);
    st->total = st->n[0] * st->n[1] * st->n[2];
    double c[9];
    orc_fd_weights(s->space_order, c);
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 9; ++k)
            st->w[a][k] = (a < s->ndim && k <= st->r) ? c[k] / (s->spacing[a] * s->spacing[a]) : 0.0;
    st->dt = s->dt;
    st->m = m;
    st->eta = eta;
    return ORC_OK;
}

/* Value of a field at integer coordinates; zero outside the grid (zero halo). */
static double at(const stepper *st, const double *u, int64_t x, int64_t y, int64_t z)
{
    if (x < 0 || x >= st->n[0]) return 0.0;
    if (st->nd == 3) {
        if (y < 0 || y >= st->n[1] || z < 0 || z >= st->n[2]) return 0.0;
        return u[(x * st->n[1] + y) * st->n[2] + z];
    }
    if (z < 0 || z >= st->n[1]) return 0.0;
    return u[x * st->n[1] + z];
}

/*
 * Order-p Laplacian at one point: the sum over axes of the 1-D second
 * derivatives (Sec. 3.1: `laplace` expands to dx2 + dy2 (+ dz2)).
 */
static double laplacian(const stepper *st, const double *u, int64_t x, int64_t y, int64_t z)
{
    double acc = 0.0;
    for (int k = -st->r; k <= st->r; ++k) {
        int kk = k < 0 ? -k : k;
        acc += st->w[0][kk] * at(st, u, x + k, y, z);
        if (st->nd == 3) {
            acc += st->w[1][kk] * at(st, u, x, y + k, z);
            acc += st->w[2][kk] * at(st, u, x, y, z + k);
        } else {
            acc += st->w[1][kk] * at(st, u, x, y, z + k);
        }
    }
    return acc;
}

/*
 * One explicit step of Eq. 3 solved for the newest time level (Sec. 5.1):
 *   m (u+ - 2u + u-)/dt^2 + eta (u+ - u-)/(2 dt) - lap(u) = 0
 *   =>  u+ = [ 2m u - (m - eta dt/2) u- + dt^2 lap(u) ] / (m + eta dt/2)
 * `cur` is u, `older` is u-, the result goes to `out` (a distinct buffer).
 * The same algebra, with the damping sign reversed and solved for the oldest
 * level, is the adjoint step of Listing 7 (see orc_adjoint).
 */
static void step_all(const stepper *st, const double *cur, const double *older, double *out)
{
    const double dt = st->dt, dt2 = dt * dt;
    int64_t n0 = st->n[0];
    int64_t plane = st->total / n0;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < n0; ++x) {
        for (int64_t q = 0; q < plane; ++q) {
            int64_t idx = x * plane + q;
            int64_t y, z;
            if (st->nd == 3) { y = q / st->n[2]; z = q % st->n[2]; }
            else { y = 0; z = q; }
            double m = st->m[idx], e = st->eta[idx];
            double lap = laplacian(st, cur, x, y, z);
            out[idx] = (2.0 * m * cur[idx] - (m - 0.5 * e * dt) * older[idx] + dt2 * lap) / (m + 0.5 * e * dt);
        }
    }
}

/* Point-to-grid: field += dt^2 w v / (m + eta dt/2) at every corner (Listing 8). */
static void inject(const stepper *st, int npts, int nc, const int64_t *idx, const double *w,
                   const double *vals, double *field)
{
    const double dt = st->dt, dt2 = dt * dt;
    for (int p = 0; p < npts; ++p)
        for (int c = 0; c < nc; ++c) {
            int64_t i = idx[(int64_t)p * nc + c];
            field[i] += dt2 * w[(int64_t)p * nc + c] * vals[p] / (st->m[i] + 0.5 * st->eta[i] * dt);
        }
}

/* Grid-to-point: out[p] = sum over corners of w * field (Sec. 5.2). */
static void sample(int npts, int nc, const int64_t *idx, const double *w, const double *field, double *out)
{
    for (int p = 0; p < npts; ++p) {
        double acc = 0.0;
        for (int c = 0; c < nc; ++c) acc += w[(int64_t)p * nc + c] * field[idx[(int64_t)p * nc + c]];
        out[p] = acc;
    }
}

typedef struct {
    int npts, nc;
    int64_t *idx;
    double *w;
} points;

static int make_points(const orc_setup *s, int npts, const double *coords, points *pt)
{
    pt->npts = npts;
    pt->nc = 1 << s->ndim;
    pt->idx = NULL;
    pt->w = NULL;
    if (npts == 0) return ORC_OK;
    pt->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)npts * pt->nc);
    pt->w = (double *)malloc(sizeof(double) * (size_t)npts * pt->nc);
    if (!pt->idx || !pt->w) return ORC_ERR_MEM;
    return orc_interp(s, npts, coords, pt->idx, pt->w);
}

static void free_points(points *pt)
{
    free(pt->idx);
    free(pt->w);
}

/*
 * Forward modelling (Sec. 5.1, Listing 6, with the source injection and the
 * receiver interpolation of Sec. 5.2).  m and eta have the computational shape;
 * q is [nt][nsrc]; rec (out) is [nt][nrec]; u_hist (optional, may be NULL) is
 * [nt][points] and receives u^0..u^{nt-1}; u_final (optional) receives u^{nt-1}.
 */
int orc_forward(const orc_setup *s, const double *m, const double *eta,
                int nsrc, const double *src_xyz, const double *q,
                int nrec, const double *rec_xyz, double *rec,
                double *u_hist, double *u_final)
{
    stepper st;
    int rc = make_stepper(s, m, eta, &st);
    if (rc != ORC_OK) return rc;
    if (nsrc < 0 || nrec < 0 || (nsrc > 0 && !q) || (nrec > 0 && !rec)) return ORC_ERR_ARG;
    points ps, pr;
    rc = make_points(s, nsrc, src_xyz, &ps);
    if (rc == ORC_OK) rc = make_points(s, nrec, rec_xyz, &pr);
    else pr.idx = NULL, pr.w = NULL;
    double *a = NULL, *b = NULL, *c = NULL;
    if (rc == ORC_OK) {
        a = (double *)calloc((size_t)st.total, sizeof(double));   /* u^{n-1} */
        b = (double *)calloc((size_t)st.total, sizeof(double));   /* u^n     */
        c = (double *)calloc((size_t)st.total, sizeof(double));   /* u^{n+1} */
        if (!a || !b || !c) rc = ORC_ERR_MEM;
    }
    if (rc == ORC_OK) {
        for (int n = 0; n < s->nt; ++n) {
            if (nrec > 0) sample(nrec, pr.nc, pr.idx, pr.w, b, rec + (int64_t)n * nrec);
            if (u_hist) memcpy(u_hist + (int64_t)n * st.total, b, sizeof(double) * (size_t)st.total);
            if (n == s->nt - 1) break;
            step_all(&st, b, a, c);
            if (nsrc > 0) inject(&st, nsrc, ps.nc, ps.idx, ps.w, q + (int64_t)n * nsrc, c);
            double *t = a; a = b; b = c; c = t;
        }
        if (u_final) memcpy(u_final, b, sizeof(double) * (size_t)st.total);
    }
    free(a); free(b); free(c);
    free_points(&ps); free_points(&pr);
    return rc;
}

/*
 * Adjoint modelling (Sec. 5.1, Listing 7): Eq. 3 with the damping term
 * subtracted, solved for the oldest time level and marched backward:
 *   m (v+ - 2v + v-)/dt^2 - eta (v+ - v-)/(2 dt) - lap(v) = P_r^T d
 *   =>  v- = [ 2m v - (m - eta dt/2) v+ + dt^2 lap(v) ] / (m + eta dt/2)
 * with v^{nt} = v^{nt+1} = 0.  Step k (nt-1..1) makes v^k and adds d^k into it
 * (the receivers become sources, Sec. 5.2); the sources sample
 * qadj^k = P_s v^{k+1} (qadj^{nt-1} = 0).  d is [nt][nrec], qadj (out) is
 * [nt][nsrc], v_hist (optional) is [nt][points] and receives v^1..v^{nt-1} in
 * rows 1..nt-1 (row 0 is zero).
 */
int orc_adjoint(const orc_setup *s, const double *m, const double *eta,
                int nrec, const double *rec_xyz, const double *d,
                int nsrc, const double *src_xyz, double *qadj, double *v_hist)
{
    stepper st;
    int rc = make_stepper(s, m, eta, &st);
    if (rc != ORC_OK) return rc;
    if (nsrc < 0 || nrec < 0 || (nrec > 0 && !d) || (nsrc > 0 && !qadj)) return ORC_ERR_ARG;
    points ps, pr;
    rc = make_points(s, nsrc, src_xyz, &ps);
    if (rc == ORC_OK) rc = make_points(s, nrec, rec_xyz, &pr);
    else pr.idx = NULL, pr.w = NULL;
    double *vp2 = NULL, *vp1 = NULL, *v = NULL;
    if (rc == ORC_OK) {
        vp2 = (double *)calloc((size_t)st.total, sizeof(double));  /* v^{k+2} */
        vp1 = (double *)calloc((size_t)st.total, sizeof(double));  /* v^{k+1} */
        v = (double *)calloc((size_t)st.total, sizeof(double));    /* v^k     */
        if (!vp2 || !vp1 || !v) rc = ORC_ERR_MEM;
    }
    if (rc == ORC_OK) {
        if (v_hist) memset(v_hist, 0, sizeof(double) * (size_t)st.total);
        for (int k = s->nt - 1; k >= 1; --k) {
            if (nsrc > 0) sample(nsrc, ps.nc, ps.idx, ps.w, vp1, qadj + (int64_t)k * nsrc);
            step_all(&st, vp1, vp2, v);
            if (nrec > 0) inject(&st, nrec, pr.nc, pr.idx, pr.w, d + (int64_t)k * nrec, v);
            if (v_hist) memcpy(v_hist + (int64_t)k * st.total, v, sizeof(double) * (size_t)st.total);
            double *t = vp2; vp2 = vp1; vp1 = v; v = t;
        }
        if (nsrc > 0) sample(nsrc, ps.nc, ps.idx, ps.w, vp1, qadj);  /* qadj^0 = P_s v^1 */
    }
    free(vp2); free(vp1); free(v);
    free_points(&ps); free_points(&pr);
    return rc;
}

/*
 * FWI gradient (Sec. 5.4 "gradient test with forward and adjoint operators").
 * For the forward map above and a cotangent r on the receivers (r = rec - d for
 * the misfit J = 1/2 sum_n |P_r u^n - d^n|^2), the exact derivative of
 * sum_n <r^n, P_r u^n> with respect to m is
 *   grad = - sum_{k=1}^{nt-1} v^k * (u^k - 2 u^{k-1} + u^{k-2}) / dt^2
 * where v is the adjoint field of orc_adjoint driven by r, and u^{-1} = 0.
 * This follows from differentiating each forward step of Eq. 3 in m: step n
 * contains m (u^{n+1} - 2u^n + u^{n-1}) and the adjoint multiplier of that
 * step is v^{n+1} / dt^2.  The full forward history is kept (small cases only).
 * grad has the computational shape.
 */
int orc_gradient(const orc_setup *s, const double *m, const double *eta,
                 int nsrc, const double *src_xyz, const double *q,
                 int nrec, const double *rec_xyz, const double *resid, double *grad)
{
    stepper st;
    int rc = make_stepper(s, m, eta, &st);
    if (rc != ORC_OK) return rc;
    if (!grad || (nrec > 0 && !resid)) return ORC_ERR_ARG;
    int64_t tot = st.total;
    double *hist = (double *)malloc(sizeof(double) * (size_t)tot * (size_t)s->nt);
    if (!hist) return ORC_ERR_MEM;
    rc = orc_forward(s, m, eta, nsrc, src_xyz, q, 0, NULL, NULL, hist, NULL);
    points pr;
    pr.idx = NULL; pr.w = NULL;
    if (rc == ORC_OK) rc = make_points(s, nrec, rec_xyz, &pr);
    double *vp2 = NULL, *vp1 = NULL, *v = NULL;
    if (rc == ORC_OK) {
        vp2 = (double *)calloc((size_t)tot, sizeof(double));
        vp1 = (double *)calloc((size_t)tot, sizeof(double));
        v = (double *)calloc((size_t)tot, sizeof(double));
        if (!vp2 || !vp1 || !v) rc = ORC_ERR_MEM;
    }
    if (rc == ORC_OK) {
        const double dt2 = s->dt * s->dt;
        memset(grad, 0, sizeof(double) * (size_t)tot);
        for (int k = s->nt - 1; k >= 1; --k) {
            step_all(&st, vp1, vp2, v);
            if (nrec > 0) inject(&st, nrec, pr.nc, pr.idx, pr.w, resid + (int64_t)k * nrec, v);
            const double *uk = hist + (int64_t)k * tot;
            const double *uk1 = hist + (int64_t)(k - 1) * tot;
            const double *uk2 = (k >= 2) ? hist + (int64_t)(k - 2) * tot : NULL;
            for (int64_t i = 0; i < tot; ++i) {
                double d2 = uk[i] - 2.0 * uk1[i] + (uk2 ? uk2[i] : 0.0);
                grad[i] -= v[i] * d2 / dt2;
            }
            double *t = vp2; vp2 = vp1; vp1 = v; v = t;
        }
    }
    free(vp2); free(vp1); free(v);
    free_points(&pr);
    free(hist);
    return rc;
}

/* Number of computational points of a setup (helper for the Python wrapper). */
int64_t orc_points(const orc_setup *s)
{
    if (check_setup(s) != ORC_OK) return -1;
    return comp_points(s);
}

/* ------------------------------------------------------------------------- */
/* 2D diffusion (Sec. 4, Eq. 1 and Eq. 2)                                     */
/* ------------------------------------------------------------------------- */

/*
 * Forward-Euler diffusion u_t = alpha lap(u) on an [nx][ny] grid with the
 * boundary rows and columns held fixed (Sec. 4.1: only interior points are
 * updated).  Second-order 3-point stencils per axis.  `u` holds the initial
 * field on entry and the field after `steps` steps on return.
 */
int orc_diffusion(int64_t nx, int64_t ny, double dx, double dy, double alpha, double dt,
                  int steps, double *u)
{
    if (nx < 3 || ny < 3 || !u || steps < 0 || !(dx > 0) || !(dy > 0)) return ORC_ERR_ARG;
    double *v = (double *)malloc(sizeof(double) * (size_t)(nx * ny));
    if (!v) return ORC_ERR_MEM;
    memcpy(v, u, sizeof(double) * (size_t)(nx * ny));
    double *cur = u, *nxt = v;
    for (int t = 0; t < steps; ++t) {
        for (int64_t i = 1; i < nx - 1; ++i)
            for (int64_t j = 1; j < ny - 1; ++j) {
                double c = cur[i * ny + j];
                double uxx = (cur[(i + 1) * ny + j] - 2.0 * c + cur[(i - 1) * ny + j]) / (dx * dx);
                double uyy = (cur[i * ny + j + 1] - 2.0 * c + cur[i * ny + j - 1]) / (dy * dy);
                nxt[i * ny + j] = c + dt * alpha * (uxx + uyy);
            }
        double *t2 = cur; cur = nxt; nxt = t2;
    }
    if (cur != u) memcpy(u, cur, sizeof(double) * (size_t)(nx * ny));
    free(v);
    return ORC_OK;
}
