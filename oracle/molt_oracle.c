/*
 * molt_oracle.c -- plain FP64 CPU oracle for the MOL^T recursive-convolution
 * wave solver of Causley & Christlieb, "Higher order A-stable schemes for the
 * wave equation using a recursive convolution approach" (arXiv:1308.3214).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the library itself never calls it and
 * shares no code, header, table or constant generator with it.
 *
 * Everything is computed in double precision, in the order the paper states
 * it, without blocking, fusion or algebraic re-arrangement:
 *
 *   - the convolution L^{-1} of eq. (L_Inverse), split into the left- and
 *     right-going parts I^L, I^R and evaluated with the exponential
 *     recurrences of Sec. 2, the increments integrated exactly against the
 *     local quadratic (or linear) interpolant, plus the homogeneous boundary
 *     terms A e^{-alpha(x-a)} + B e^{-alpha(b-x)} (Sec. 2, Sec. 3.2);
 *   - D = 1 - L^{-1} (eq. D_def_1d);
 *   - the 1D update of order 2P, eq. (update_P) with the coefficients A_p;
 *   - the 2D/3D ADI operators C (eqs. C_def_ADI, C_def_ADI_3) and
 *     D (eqs. D_def_ADI, D_def_ADI_3), combined as in eq. (Full_2D) with the
 *     terms built in the order of Table 3 (Sec. 4.2);
 *   - the time step u^{n+1} = 2u^n - u^{n-1} + F[u^n] and the start value
 *     u^1 = u^0 + F[u^0]/2 for zero initial velocity (Sec. 3.2).
 *
 * Readings of points the paper leaves open (each is listed in the design
 * notes of the repository):
 *   - Local interpolant (Sec. 2 says only "O(1) operations"; the quadrature
 *     is deferred to the authors' earlier paper).  quad = 2 (default): the
 *     quadratic through the nodes j-1, j, j+1 of the destination node j,
 *     integrated exactly over the cell next to x_j; in the cells touching a
 *     Dirichlet end the three nodes nearest inside the domain are used.
 *     quad = 1: the linear interpolant of the cell.  The quadratic rule
 *     reproduces every error of Table 2.
 *   - Dirichlet: the corrected L^{-1} returns w = v at both end nodes, so
 *     D v = 0 there (Sec. 3.2: the boundary values of D^m u are the even
 *     derivatives of the boundary data, zero for homogeneous data).
 *   - Periodic: the left/right parts include every periodic image, which
 *     fixes A = I^L(b)/(1-mu), B = I^R(a)/(1-mu) on the line closed by
 *     x_n = x_0 (mu = e^{-alpha L}).
 *
 * Grid convention: a field of shape (nx, ny, nz) is stored with x fastest,
 * index = x + nx*(y + ny*z).  A Dirichlet axis of n points includes both end
 * nodes (spacing L/(n-1)); a periodic axis holds n distinct points (L/n).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PERIODIC 0
#define ORC_DIRICHLET 1

/* ------------------------------------------------------------------------ */
/* Exponential moments M_k(nu) = int_0^nu t^k e^{-t} dt, k = 0, 1, 2.        */
/* For small nu the closed forms cancel, so the power series is summed.      */
/* ------------------------------------------------------------------------ */
static double moment(int k, double nu)
{
    if (nu < 0.5) {
        /* int_0^nu t^k sum_i (-t)^i / i! dt = sum_i (-1)^i nu^{k+i+1} / (i! (k+i+1)) */
        double sum = 0.0, term_pow = pow(nu, k + 1), fact = 1.0;
        for (int i = 0; i < 40; ++i) {
            if (i > 0) { term_pow *= nu; fact *= i; }
            double t = ((i & 1) ? -1.0 : 1.0) * term_pow / (fact * (k + i + 1));
            sum += t;
        }
        return sum;
    }
    double e = exp(-nu);
    if (k == 0) return 1.0 - e;
    if (k == 1) return 1.0 - (1.0 + nu) * e;
    return 2.0 - (2.0 + 2.0 * nu + nu * nu) * e;
}

/*
 * Quadrature weights of one increment (Sec. 2):
 *   J^L_j = (alpha/2) int_0^h e^{-alpha y} p(x_j - y) dy,
 * with p the interpolant written in Newton form about x_j and s = -y/h:
 *   p = v_j + s (v_j - v_{j-1}) + s (s+1)/2 * S,
 * where S is the second difference of the three interpolation nodes.  With
 * t = alpha y, s = -t/nu this integrates to
 *   J^L_j = 1/2 [ W0 v_j + W1 v_{j-1} + R S ],
 *   W0 = M0 - M1/nu,  W1 = M1/nu,  R = (M2/nu^2 - M1/nu)/2.
 * The mirror image gives J^R_j with v_{j+1} in place of v_{j-1}.
 * quad = 1 drops the S term (linear interpolant).
 */
void orc_weights(double nu, int quad, double out[4])
{
    double M0 = moment(0, nu), M1 = moment(1, nu), M2 = moment(2, nu);
    out[0] = exp(-nu);                    /* d = e^{-alpha h} */
    out[1] = M0 - M1 / nu;                /* W0 */
    out[2] = M1 / nu;                     /* W1 */
    out[3] = (quad >= 2) ? 0.5 * (M2 / (nu * nu) - M1 / nu) : 0.0; /* R */
}

/* ------------------------------------------------------------------------ */
/* L^{-1} on one line (eq. L_Inverse with the boundary correction).          */
/* v and w are read/written with stride sv / sw.                             */
/* ------------------------------------------------------------------------ */
static double vat(const double *v, long sv, long n, int bc, long j)
{
    if (bc == ORC_PERIODIC) { j %= n; if (j < 0) j += n; }
    return v[j * sv];
}

/* second difference centred at node c */
static double sdiff(const double *v, long sv, long n, int bc, long c)
{
    return vat(v, sv, n, bc, c + 1) - 2.0 * vat(v, sv, n, bc, c) + vat(v, sv, n, bc, c - 1);
}

/* gL, gR (Dirichlet): the values that D v = v - w must take at the end
 * nodes (zero for homogeneous data, see orc_linv_line_bc). */
static void linv_line_impl(const double *v, long sv, double *w, long sw, long n,
                           double nu, int quad, int bc, double gL, double gR)
{
    double c4[4];
    orc_weights(nu, quad, c4);
    double d = c4[0], W0 = c4[1], W1 = c4[2], R = c4[3];
    /* Dirichlet: cells 1..n-1 between nodes 0..n-1.  Periodic: the line is
     * closed by node n == node 0, giving n cells. */
    long N = (bc == ORC_PERIODIC) ? n : n - 1;
    int use_quad = (R != 0.0) && n >= 3;   /* a quadratic needs three nodes */
    double *JL = calloc((size_t)(N + 1), sizeof(double));
    double *JR = calloc((size_t)(N + 1), sizeof(double));
    double *IL = calloc((size_t)(N + 1), sizeof(double));
    double *IR = calloc((size_t)(N + 1), sizeof(double));

    /* increments of the left-going part, cells [x_{j-1}, x_j] */
    for (long j = 1; j <= N; ++j) {
        double S = 0.0;
        if (use_quad) {
            long c = j;                                     /* nodes j-1, j, j+1 */
            if (bc == ORC_DIRICHLET && c + 1 > n - 1) c = j - 1;  /* nodes j-2, j-1, j */
            S = sdiff(v, sv, n, bc, c);
        }
        JL[j] = 0.5 * (W0 * vat(v, sv, n, bc, j) + W1 * vat(v, sv, n, bc, j - 1) + R * S);
    }
    /* increments of the right-going part, cells [x_j, x_{j+1}] */
    for (long j = 0; j < N; ++j) {
        double S = 0.0;
        if (use_quad) {
            long c = j;                                     /* nodes j-1, j, j+1 */
            if (bc == ORC_DIRICHLET && c - 1 < 0) c = j + 1;      /* nodes j, j+1, j+2 */
            S = sdiff(v, sv, n, bc, c);
        }
        JR[j] = 0.5 * (W0 * vat(v, sv, n, bc, j) + W1 * vat(v, sv, n, bc, j + 1) + R * S);
    }
    /* exponential recurrences: I^L(x) = e^{-alpha h} I^L(x - h) + J^L,
     * I^R(x) = e^{-alpha h} I^R(x + h) + J^R, no inflow at the line ends */
    IL[0] = 0.0;
    for (long j = 1; j <= N; ++j) IL[j] = d * IL[j - 1] + JL[j];
    IR[N] = 0.0;
    for (long j = N - 1; j >= 0; --j) IR[j] = d * IR[j + 1] + JR[j];

    /* homogeneous terms A e^{-alpha (x - a)} + B e^{-alpha (b - x)} */
    double mu = pow(d, (double)N);     /* e^{-alpha (b - a)} */
    double A, B;
    if (bc == ORC_PERIODIC) {
        /* contributions of all periodic images to the left / right */
        A = IL[N] / (1.0 - mu);
        B = IR[0] / (1.0 - mu);
    } else {
        /* w(a) = v(a) - gL, w(b) = v(b) - gR:
         *   A + mu B = v_0 - gL - I^R_0,   mu A + B = v_N - gR - I^L_N  */
        double r0 = vat(v, sv, n, bc, 0) - gL - IR[0];
        double r1 = vat(v, sv, n, bc, N) - gR - IL[N];
        A = (r0 - mu * r1) / (1.0 - mu * mu);
        B = (r1 - mu * r0) / (1.0 - mu * mu);
    }
    for (long j = 0; j < n; ++j)
        w[j * sw] = IL[j] + IR[j] + A * pow(d, (double)j) + B * pow(d, (double)(N - j));
    free(JL); free(JR); free(IL); free(IR);
}

void orc_linv_line(const double *v, long sv, double *w, long sw, long n,
                   double nu, int quad, int bc)
{
    linv_line_impl(v, sv, w, sw, n, nu, quad, bc, 0.0, 0.0);
}

/* ------------------------------------------------------------------------ */
/* Embedded boundaries (Sec. 4.3): L^{-1} on a line object.  The line is the */
/* part of a grid line inside the domain: m interior grid nodes x_1..x_m     */
/* with spacing h, and two boundary points, x_0 = a at distance da before    */
/* x_1 and x_{m+1} = b at distance db after x_m (0 < da, db), where the      */
/* homogeneous Dirichlet data are zero.  The quadrature is the rule of the   */
/* rectangular line written for arbitrary node positions: J^L on the cell    */
/* [x_{j-1}, x_j] integrates the quadratic through x_{j-1}, x_j, x_{j+1}     */
/* (x_{j-2}, x_{j-1}, x_j in the last cell), J^R on [x_j, x_{j+1}] the one   */
/* through x_{j-1}, x_j, x_{j+1} (x_j, x_{j+1}, x_{j+2} in the first cell), */
/* each exactly against the kernel; the recurrences decay by e^{-alpha dx}  */
/* over each cell; A, B make w vanish at a and b.  With da = db = h this is  */
/* orc_linv_line on the m + 2 nodes of a rectangular Dirichlet line.         */
/* ------------------------------------------------------------------------ */

/* out[i] = (alpha/2) int_0^len e^{-alpha s} l_i(s) ds for the Lagrange basis
 * l_i of three nodes at coordinates ts[] (s = distance from the destination
 * node into the cell), from int_0^len s^k e^{-alpha s} ds = M_k(alpha len) /
 * alpha^{k+1}: l_i(s) = (s^2 - (ta + tb) s + ta tb) / ((t_i - ta)(t_i - tb)).
 * The moments of short cells come from their power series (moment()), which
 * is what keeps boundary points arbitrarily close to a grid node usable. */
static void basis_weights(const double ts[3], double len, double alpha, double out[3])
{
    double nu = alpha * len;
    double m0 = moment(0, nu) / alpha;
    double m1 = moment(1, nu) / (alpha * alpha);
    double m2 = moment(2, nu) / (alpha * alpha * alpha);
    for (int i = 0; i < 3; ++i) {
        double ta = ts[(i + 1) % 3], tb = ts[(i + 2) % 3];
        double den = (ts[i] - ta) * (ts[i] - tb);
        out[i] = 0.5 * alpha * (m2 - (ta + tb) * m1 + ta * tb * m0) / den;
    }
}

void orc_linv_obj(const double *v, long sv, double *w, long sw, long m, double h, double da, double db,
                  double alpha)
{
    long N = m + 1;                                   /* cells between the nodes 0..N */
    double *x = malloc(sizeof(double) * (size_t)(N + 1));
    double *u = malloc(sizeof(double) * (size_t)(N + 1));
    double *JL = calloc((size_t)(N + 1), sizeof(double));
    double *JR = calloc((size_t)(N + 1), sizeof(double));
    double *IL = calloc((size_t)(N + 1), sizeof(double));
    double *IR = calloc((size_t)(N + 1), sizeof(double));
    x[0] = 0.0;
    u[0] = 0.0;
    for (long j = 1; j <= m; ++j) { x[j] = da + (double)(j - 1) * h; u[j] = v[(j - 1) * sv]; }
    x[N] = x[m] + db;
    u[N] = 0.0;
    for (long j = 1; j <= N; ++j) {                   /* cell [x_{j-1}, x_j], destination x_j */
        long c0 = (j + 1 <= N) ? j - 1 : j - 2;
        double ts[3], wt[3];
        for (int i = 0; i < 3; ++i) ts[i] = x[j] - x[c0 + i];
        basis_weights(ts, x[j] - x[j - 1], alpha, wt);
        JL[j] = wt[0] * u[c0] + wt[1] * u[c0 + 1] + wt[2] * u[c0 + 2];
    }
    for (long j = 0; j < N; ++j) {                    /* cell [x_j, x_{j+1}], destination x_j */
        long c0 = (j - 1 >= 0) ? j - 1 : j;
        double ts[3], wt[3];
        for (int i = 0; i < 3; ++i) ts[i] = x[c0 + i] - x[j];
        basis_weights(ts, x[j + 1] - x[j], alpha, wt);
        JR[j] = wt[0] * u[c0] + wt[1] * u[c0 + 1] + wt[2] * u[c0 + 2];
    }
    IL[0] = 0.0;
    for (long j = 1; j <= N; ++j) IL[j] = exp(-alpha * (x[j] - x[j - 1])) * IL[j - 1] + JL[j];
    IR[N] = 0.0;
    for (long j = N - 1; j >= 0; --j) IR[j] = exp(-alpha * (x[j + 1] - x[j])) * IR[j + 1] + JR[j];
    double mu = exp(-alpha * (x[N] - x[0]));
    double r0 = u[0] - IL[0] - IR[0];                 /* w(a) = 0 */
    double r1 = u[N] - IL[N] - IR[N];                 /* w(b) = 0 */
    double A = (r0 - mu * r1) / (1.0 - mu * mu);
    double B = (r1 - mu * r0) / (1.0 - mu * mu);
    for (long j = 1; j <= m; ++j)
        w[(j - 1) * sw] = IL[j] + IR[j] + A * exp(-alpha * (x[j] - x[0])) + B * exp(-alpha * (x[N] - x[j]));
    free(x); free(u); free(JL); free(JR); free(IL); free(IR);
}

/* A 2D domain embedded in an nx x ny grid (x fastest): row j holds the
 * interior nodes i = r0[j] .. r1[j] (none when r0[j] > r1[j]) with the
 * boundary points at distances ra[j] before r0[j] and rb[j] after r1[j];
 * column i likewise holds the rows c0[i] .. c1[i] with gaps ca[i], cb[i].
 * Nodes outside the domain hold zero. */
typedef struct {
    long nx, ny;
    double hx, hy;
    const long *r0, *r1, *c0, *c1;
    const double *ra, *rb, *ca, *cb;
} orc_geom;

/* L_gamma^{-1} on every line object of one axis */
static void linv_axis_obj(const orc_geom *g, const double *v, double *w, int axis, double alpha)
{
    long T = g->nx * g->ny;
    memset(w, 0, sizeof(double) * (size_t)T);
    if (axis == 0) {
        #pragma omp parallel for schedule(static)
        for (long j = 0; j < g->ny; ++j) {
            if (g->r0[j] > g->r1[j]) continue;
            long b = j * g->nx + g->r0[j];
            orc_linv_obj(v + b, 1, w + b, 1, g->r1[j] - g->r0[j] + 1, g->hx, g->ra[j], g->rb[j], alpha);
        }
    } else {
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < g->nx; ++i) {
            if (g->c0[i] > g->c1[i]) continue;
            long b = g->c0[i] * g->nx + i;
            orc_linv_obj(v + b, g->nx, w + b, g->nx, g->c1[i] - g->c0[i] + 1, g->hy, g->ca[i], g->cb[i], alpha);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* (L^{-1})^T on one line: the statements of orc_linv_line transposed and     */
/* executed in reverse order (each read x = v_j becomes vbar_j += xbar, each  */
/* recurrence runs backwards).  Used by the adjoint of the time stepping; the */
/* paper itself has no adjoint.                                               */
/* ------------------------------------------------------------------------ */
static void vadd(double *v, long sv, long n, int bc, long j, double x)
{
    if (bc == ORC_PERIODIC) { j %= n; if (j < 0) j += n; }
    v[j * sv] += x;
}

static void sdiff_T(double *v, long sv, long n, int bc, long c, double x)
{
    vadd(v, sv, n, bc, c + 1, x);
    vadd(v, sv, n, bc, c, -2.0 * x);
    vadd(v, sv, n, bc, c - 1, x);
}

void orc_linv_line_T(const double *w, long sw, double *v, long sv, long n,
                     double nu, int quad, int bc)
{
    double c4[4];
    orc_weights(nu, quad, c4);
    double d = c4[0], W0 = c4[1], W1 = c4[2], R = c4[3];
    long N = (bc == ORC_PERIODIC) ? n : n - 1;
    int use_quad = (R != 0.0) && n >= 3;
    double *gJL = calloc((size_t)(N + 1), sizeof(double));
    double *gJR = calloc((size_t)(N + 1), sizeof(double));
    double *gIL = calloc((size_t)(N + 1), sizeof(double));
    double *gIR = calloc((size_t)(N + 1), sizeof(double));
    for (long j = 0; j < n; ++j) v[j * sv] = 0.0;

    /* w_j = IL_j + IR_j + A d^j + B d^{N-j} */
    double gA = 0.0, gB = 0.0;
    for (long j = 0; j < n; ++j) {
        double x = w[j * sw];
        gIL[j] += x;
        gIR[j] += x;
        gA += x * pow(d, (double)j);
        gB += x * pow(d, (double)(N - j));
    }
    double mu = pow(d, (double)N);
    if (bc == ORC_PERIODIC) {
        gIL[N] += gA / (1.0 - mu);              /* A = IL_N / (1 - mu) */
        gIR[0] += gB / (1.0 - mu);              /* B = IR_0 / (1 - mu) */
    } else {
        double gr0 = (gA - mu * gB) / (1.0 - mu * mu);
        double gr1 = (gB - mu * gA) / (1.0 - mu * mu);
        vadd(v, sv, n, bc, 0, gr0);             /* r0 = v_0 - IR_0 */
        gIR[0] -= gr0;
        vadd(v, sv, n, bc, N, gr1);             /* r1 = v_N - IL_N */
        gIL[N] -= gr1;
    }
    /* IR_j = d IR_{j+1} + JR_j, computed for j = N-1 down to 0 */
    for (long j = 0; j < N; ++j) {
        gJR[j] += gIR[j];
        gIR[j + 1] += d * gIR[j];
    }
    /* IL_j = d IL_{j-1} + JL_j, computed for j = 1 up to N */
    for (long j = N; j >= 1; --j) {
        gJL[j] += gIL[j];
        gIL[j - 1] += d * gIL[j];
    }
    /* JR_j = (W0 v_j + W1 v_{j+1} + R S)/2 */
    for (long j = 0; j < N; ++j) {
        double g = 0.5 * gJR[j];
        vadd(v, sv, n, bc, j, W0 * g);
        vadd(v, sv, n, bc, j + 1, W1 * g);
        if (use_quad) {
            long c = j;
            if (bc == ORC_DIRICHLET && c - 1 < 0) c = j + 1;
            sdiff_T(v, sv, n, bc, c, R * g);
        }
    }
    /* JL_j = (W0 v_j + W1 v_{j-1} + R S)/2 */
    for (long j = 1; j <= N; ++j) {
        double g = 0.5 * gJL[j];
        vadd(v, sv, n, bc, j, W0 * g);
        vadd(v, sv, n, bc, j - 1, W1 * g);
        if (use_quad) {
            long c = j;
            if (bc == ORC_DIRICHLET && c + 1 > n - 1) c = j - 1;
            sdiff_T(v, sv, n, bc, c, R * g);
        }
    }
    free(gJL); free(gJR); free(gIL); free(gIR);
}

/* ------------------------------------------------------------------------ */
/* Axis operators on a whole field: L_gamma^{-1} and D_gamma (eq. LD_gam)     */
/* ------------------------------------------------------------------------ */
static long total_size(int ndim, const long *shape)
{
    long t = 1;
    for (int a = 0; a < ndim; ++a) t *= shape[a];
    return t;
}

void orc_linv_axis(const double *v, double *w, int ndim, const long *shape,
                   int axis, double nu, int quad, int bc)
{
    long n = shape[axis];
    long stride = 1;
    for (int a = 0; a < axis; ++a) stride *= shape[a];
    long total = total_size(ndim, shape);
    long nlines = total / n;
    #pragma omp parallel for schedule(static)
    for (long line = 0; line < nlines; ++line) {
        /* line = (inner index below the axis) + stride * (outer index) */
        long inner = line % stride, outer = line / stride;
        long base = inner + outer * stride * n;
        orc_linv_line(v + base, stride, w + base, stride, n, nu, quad, bc);
    }
}

void orc_D_axis(const double *v, double *out, int ndim, const long *shape,
                int axis, double nu, int quad, int bc)
{
    long total = total_size(ndim, shape);
    double *w = malloc(sizeof(double) * (size_t)total);
    orc_linv_axis(v, w, ndim, shape, axis, nu, quad, bc);
    for (long i = 0; i < total; ++i) out[i] = v[i] - w[i];
    free(w);
}

void orc_linv_axis_T(const double *v, double *w, int ndim, const long *shape,
                     int axis, double nu, int quad, int bc)
{
    long n = shape[axis];
    long stride = 1;
    for (int a = 0; a < axis; ++a) stride *= shape[a];
    long total = total_size(ndim, shape);
    long nlines = total / n;
#pragma omp parallel for schedule(static)
    for (long line = 0; line < nlines; ++line) {
        long inner = line % stride, outer = line / stride;
        long base = inner + outer * stride * n;
        orc_linv_line_T(v + base, stride, w + base, stride, n, nu, quad, bc);
    }
}

/* D^T = 1 - (L^{-1})^T along one axis */
void orc_D_axis_T(const double *v, double *out, int ndim, const long *shape,
                  int axis, double nu, int quad, int bc)
{
    long total = total_size(ndim, shape);
    double *w = malloc(sizeof(double) * (size_t)total);
    orc_linv_axis_T(v, w, ndim, shape, axis, nu, quad, bc);
    for (long i = 0; i < total; ++i) out[i] = v[i] - w[i];
    free(w);
}

/* ------------------------------------------------------------------------ */
/* Coefficients of eq. (update_P):                                           */
/*   A_p(beta) = 2 sum_{m=1}^{p} (-1)^m beta^{2m}/(2m)! binom(p-1, m-1)       */
/* ------------------------------------------------------------------------ */
static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

static double factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

/* c_{p,m} = (-1)^m 2 beta^{2m}/(2m)! binom(p-1, m-1), the weight of
 * C^m D^{p-m} in eq. (Full_2D); in 1D C = D and sum_m c_{p,m} = A_p. */
static double cpm(int p, int m, double beta)
{
    return ((m & 1) ? -1.0 : 1.0) * 2.0 * pow(beta, 2.0 * m) / factorial(2 * m) * binom(p - 1, m - 1);
}

void orc_Ap(int P, double beta, double *A)
{
    for (int p = 1; p <= P; ++p) {
        double s = 0.0;
        for (int m = 1; m <= p; ++m) s += cpm(p, m, beta);
        A[p - 1] = s;
    }
}

/* beta_max: the first positive root of -sum_{p=1}^P A_p(beta) = 4
 * (eq. Stab_cond), found by a scan for the first sign change then bisection */
double orc_beta_max(int P)
{
    double A[16];
    double prev_b = 1e-6, prev_f;
    orc_Ap(P, prev_b, A);
    prev_f = -4.0;
    for (int p = 0; p < P; ++p) prev_f -= A[p];
    for (int i = 1; i <= 40000; ++i) {
        double b = 1e-4 * i;
        orc_Ap(P, b, A);
        double f = -4.0;
        for (int p = 0; p < P; ++p) f -= A[p];
        if (prev_f < 0.0 && f >= 0.0) {
            double lo = prev_b, hi = b;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                orc_Ap(P, mid, A);
                double fm = -4.0;
                for (int p = 0; p < P; ++p) fm -= A[p];
                if (fm < 0.0) lo = mid; else hi = mid;
            }
            return 0.5 * (lo + hi);
        }
        prev_b = b; prev_f = f;
    }
    return -1.0;
}

/* ------------------------------------------------------------------------ */
/* ADI operators of Sec. 4.                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int ndim; const long *shape; const double *nu; int quad; int bc; long total;
    long napplied;            /* number of applications of C or D (Table 3) */
    int transpose;            /* 1: every per-axis operator replaced by its transpose */
    const orc_geom *geom;     /* 2D embedded domain (line objects), else NULL */
    double alpha;             /* alpha of the line objects */
} orc_ctx;

static void Linv(orc_ctx *c, const double *v, double *w, int axis)
{
    if (c->geom) linv_axis_obj(c->geom, v, w, axis, c->alpha);
    else if (c->transpose) orc_linv_axis_T(v, w, c->ndim, c->shape, axis, c->nu[axis], c->quad, c->bc);
    else orc_linv_axis(v, w, c->ndim, c->shape, axis, c->nu[axis], c->quad, c->bc);
}

static void Dgam(orc_ctx *c, const double *v, double *w, int axis)
{
    if (c->geom) {
        /* D_gamma = 1 - L_gamma^{-1} on the interior nodes (zero outside) */
        linv_axis_obj(c->geom, v, w, axis, c->alpha);
        for (long i = 0; i < c->total; ++i) w[i] = v[i] - w[i];
        return;
    }
    if (c->transpose) orc_D_axis_T(v, w, c->ndim, c->shape, axis, c->nu[axis], c->quad, c->bc);
    else orc_D_axis(v, w, c->ndim, c->shape, axis, c->nu[axis], c->quad, c->bc);
}

/* C[v]: 1D: D_x v;  2D: L_y^{-1} D_x v + L_x^{-1} D_y v (eq. C_def_ADI);
 * 3D: L_y^{-1}L_z^{-1} D_x v + L_z^{-1}L_x^{-1} D_y v + L_x^{-1}L_y^{-1} D_z v
 * (eq. C_def_ADI_3). */
static void applyC(orc_ctx *c, const double *v, double *out)
{
    long T = c->total;
    double *t1 = malloc(sizeof(double) * (size_t)T);
    double *t2 = malloc(sizeof(double) * (size_t)T);
    c->napplied++;
    if (c->ndim == 1) {
        Dgam(c, v, out, 0);
    } else if (c->ndim == 2) {
        Dgam(c, v, t1, 0); Linv(c, t1, out, 1);          /* L_y^{-1} D_x v */
        Dgam(c, v, t1, 1); Linv(c, t1, t2, 0);           /* L_x^{-1} D_y v */
        for (long i = 0; i < T; ++i) out[i] += t2[i];
    } else {
        /* term g is L_outer^{-1} L_inner^{-1} D_g, applied right to left:
         * (x: L_y L_z D_x), (y: L_z L_x D_y), (z: L_x L_y D_z) */
        memset(out, 0, sizeof(double) * (size_t)T);
        for (int g = 0; g < 3; ++g) {
            int outer = (g + 1) % 3, inner = (g + 2) % 3;
            Dgam(c, v, t1, g); Linv(c, t1, t2, inner); Linv(c, t2, t1, outer);
            for (long i = 0; i < T; ++i) out[i] += t1[i];
        }
    }
    free(t1); free(t2);
}

/* D[v]: 1D: D_x v;  2D: v - L_x^{-1}L_y^{-1} v (eq. D_def_ADI);
 * 3D: v - L_x^{-1}L_y^{-1}L_z^{-1} v (eq. D_def_ADI_3). */
static void applyD(orc_ctx *c, const double *v, double *out)
{
    long T = c->total;
    double *t1 = malloc(sizeof(double) * (size_t)T);
    double *t2 = malloc(sizeof(double) * (size_t)T);
    c->napplied++;
    if (c->ndim == 1) {
        Dgam(c, v, out, 0);
    } else {
        const double *src = v;
        double *bufs[2] = {t1, t2};
        int k = 0;
        for (int a = c->ndim - 1; a >= 0; --a) {   /* innermost operator first */
            Linv(c, src, bufs[k], a);
            src = bufs[k]; k ^= 1;
        }
        for (long i = 0; i < T; ++i) out[i] = v[i] - src[i];
    }
    free(t1); free(t2);
}

/*
 * F[u] = sum_{p=1}^{P} sum_{m=1}^{p} c_{p,m} C^m D^{p-m} u   (eq. Full_2D;
 * in 1D it is sum_p A_p D^p u, eq. update_P, since C = D there).
 * The terms are built with the re-use scheme of Table 3: after stage p the
 * auxiliaries hold v_k = C^{p-k+1} D^{k-1} u, k = 1..p, obtained from stage
 * p-1 by v_p = D[v_{p-1}] and v_k = C[v_k] (k < p); stage p costs p
 * applications.  *nops (if given) receives the number of applications.
 */
static void F_core(orc_ctx c, const double *u, double *F, int P, double beta, long *nops)
{
    long T = c.total;
    double **v = calloc((size_t)P + 1, sizeof(double *));
    for (int k = 1; k <= P; ++k) v[k] = malloc(sizeof(double) * (size_t)T);
    double *tmp = malloc(sizeof(double) * (size_t)T);
    memset(F, 0, sizeof(double) * (size_t)T);
    for (int p = 1; p <= P; ++p) {
        if (p == 1) {
            applyC(&c, u, v[1]);
        } else {
            applyD(&c, v[p - 1], v[p]);
            for (int k = 1; k < p; ++k) {
                applyC(&c, v[k], tmp);
                memcpy(v[k], tmp, sizeof(double) * (size_t)T);
            }
        }
        for (int k = 1; k <= p; ++k) {
            double w = cpm(p, p - k + 1, beta);
            for (long i = 0; i < T; ++i) F[i] += w * v[k][i];
        }
    }
    if (nops) *nops = c.napplied;
    for (int k = 1; k <= P; ++k) free(v[k]);
    free(v); free(tmp);
}

static void F_impl(const double *u, double *F, int ndim, const long *shape, const double *nu, int quad,
                   int bc, int P, double beta, long *nops, int transpose)
{
    orc_ctx c = {ndim, shape, nu, quad, bc, total_size(ndim, shape), 0, transpose, NULL, 0.0};
    F_core(c, u, F, P, beta, nops);
}

void orc_F(const double *u, double *F, int ndim, const long *shape,
           const double *nu, int quad, int bc, int P, double beta, long *nops)
{
    F_impl(u, F, ndim, shape, nu, quad, bc, P, beta, nops, 0);
}

/* F^T: every per-axis operator transposed.  The per-axis operators act on
 * different indices and commute, so (C^m D^{p-m})^T = (C^T)^m (D^T)^{p-m}
 * with C^T, D^T the expressions of C, D in the transposed per-axis
 * operators: the same sum with the same weights. */
void orc_FT(const double *u, double *F, int ndim, const long *shape,
            const double *nu, int quad, int bc, int P, double beta)
{
    F_impl(u, F, ndim, shape, nu, quad, bc, P, beta, NULL, 1);
}

/* u^{n+1} = 2 u^n - u^{n-1} + F[u^n]   (eq. update_P / Full_2D) */
void orc_step(const double *uprev, const double *ucur, double *unext, int ndim,
              const long *shape, const double *nu, int quad, int bc, int P, double beta)
{
    long T = total_size(ndim, shape);
    double *F = malloc(sizeof(double) * (size_t)T);
    orc_F(ucur, F, ndim, shape, nu, quad, bc, P, beta, NULL);
    for (long i = 0; i < T; ++i) unext[i] = 2.0 * ucur[i] - uprev[i] + F[i];
    free(F);
}

/* u^1 = u^0 + F[u^0]/2: the Taylor series of Sec. 3.2 with zero initial
 * velocity keeps only the even terms, each half the weight it has in F. */
void orc_start(const double *u0, double *u1, int ndim, const long *shape,
               const double *nu, int quad, int bc, int P, double beta)
{
    long T = total_size(ndim, shape);
    double *F = malloc(sizeof(double) * (size_t)T);
    orc_F(u0, F, ndim, shape, nu, quad, bc, P, beta, NULL);
    for (long i = 0; i < T; ++i) u1[i] = u0[i] + 0.5 * F[i];
    free(F);
}

/* Advance (uprev, ucur) = (u^{n-1}, u^n) by nsteps steps in place. */
void orc_run(double *uprev, double *ucur, long nsteps, int ndim, const long *shape,
             const double *nu, int quad, int bc, int P, double beta)
{
    long T = total_size(ndim, shape);
    double *un = malloc(sizeof(double) * (size_t)T);
    for (long s = 0; s < nsteps; ++s) {
        orc_step(uprev, ucur, un, ndim, shape, nu, quad, bc, P, beta);
        memcpy(uprev, ucur, sizeof(double) * (size_t)T);
        memcpy(ucur, un, sizeof(double) * (size_t)T);
    }
    free(un);
}

/* ------------------------------------------------------------------------ */
/* Receiver traces and the adjoint of the time stepping (no counterpart in    */
/* the paper).  The forward map u^0 -> (u^1, ..., u^N) is                     */
/*   u^1 = u^0 + F u^0 / 2,  u^{n+1} = 2 u^n - u^{n-1} + F u^n,               */
/* and the traces are t^n_r = u^n[rec_r].  For a loss J of the traces with    */
/* g^n = R^T dJ/dt^n (scatter of the trace gradients to the receiver nodes),   */
/* the adjoint states mu^n = dJ/du^n satisfy, from mu^{N+1} = 0, mu^N = g^N,  */
/*   mu^n = 2 mu^{n+1} - mu^{n+2} + F^T mu^{n+1} + g^n,   n = N-1 .. 1,        */
/* and dJ/du^0 = mu^1 + F^T mu^1 / 2 - mu^2.                                  */
/* ------------------------------------------------------------------------ */
void orc_traces(const double *u0, long nsteps, int nrec, const long *rec, double *traces,
                int ndim, const long *shape, const double *nu, int quad, int bc, int P, double beta)
{
    long T = total_size(ndim, shape);
    double *a = malloc(sizeof(double) * (size_t)T);
    double *b = malloc(sizeof(double) * (size_t)T);
    double *c = malloc(sizeof(double) * (size_t)T);
    memcpy(a, u0, sizeof(double) * (size_t)T);
    orc_start(u0, b, ndim, shape, nu, quad, bc, P, beta);
    for (long n = 1; n <= nsteps; ++n) {
        for (int r = 0; r < nrec; ++r) traces[(n - 1) * nrec + r] = b[rec[r]];
        if (n == nsteps) break;
        orc_step(a, b, c, ndim, shape, nu, quad, bc, P, beta);
        double *t = a; a = b; b = c; c = t;
    }
    free(a); free(b); free(c);
}

void orc_adjoint(const double *tgrad, long nsteps, int nrec, const long *rec, double *grad,
                 int ndim, const long *shape, const double *nu, int quad, int bc, int P, double beta)
{
    long T = total_size(ndim, shape);
    double *m2 = calloc((size_t)T, sizeof(double));   /* mu^{n+2} */
    double *m1 = calloc((size_t)T, sizeof(double));   /* mu^{n+1} */
    double *m0 = malloc(sizeof(double) * (size_t)T);  /* mu^n */
    double *F = malloc(sizeof(double) * (size_t)T);
    for (int r = 0; r < nrec; ++r) m1[rec[r]] += tgrad[(nsteps - 1) * nrec + r];   /* mu^N = g^N */
    for (long n = nsteps - 1; n >= 1; --n) {
        orc_FT(m1, F, ndim, shape, nu, quad, bc, P, beta);
        for (long i = 0; i < T; ++i) m0[i] = 2.0 * m1[i] - m2[i] + F[i];
        for (int r = 0; r < nrec; ++r) m0[rec[r]] += tgrad[(n - 1) * nrec + r];
        double *t = m2; m2 = m1; m1 = m0; m0 = t;
    }
    /* now m1 = mu^1, m2 = mu^2 (zero when nsteps == 1) */
    orc_FT(m1, F, ndim, shape, nu, quad, bc, P, beta);
    for (long i = 0; i < T; ++i) grad[i] = m1[i] + 0.5 * F[i] - m2[i];
    free(m0); free(m1); free(m2); free(F);
}

/* Threads OpenMP would use (1 when built without OpenMP). */
/* C[v] (eq. C_def_ADI): sum over the axes g of D_g v smoothed by L^{-1} of
 * the other axes */
void orc_C(const double *v, double *out, int ndim, const long *shape, const double *nu, int quad, int bc)
{
    orc_ctx c = {ndim, shape, nu, quad, bc, total_size(ndim, shape), 0, 0, NULL, 0.0};
    applyC(&c, v, out);
}

/* ------------------------------------------------------------------------ */
/* Source terms (Sec. 4.1): (1/c^2) u_tt = lap u + S, S(x, t) = g(x) f(t).    */
/* P = 1: u^{n+1} - 2u^n + u^{n-1} = F[u^n] + (c dt)^2 S^n.                    */
/* P = 2 (the fourth-order scheme of Sec. 4.1): the Taylor terms of S up to   */
/* dt^4, S_tt by the three-level difference and dt^4 c^4 lap S / 12 by        */
/* -beta^2 (c dt)^2 C[S] / 12 (lap ~ -alpha^2 C):                             */
/*   + (c dt)^2 (S^{n+1} + 10 S^n + S^{n-1}) / 12 - beta^2 (c dt)^2 C[S^n]/12. */
/* Start (zero initial velocity): u^1 = u^0 + F[u^0]/2 + (the same source     */
/* terms at n = 0)/2 with f(t_{-1}) = f(t_1) (exact for a source even about   */
/* t_0).  sc = (c dt)^2; f[k] = f(t_k), k = 0..nsteps.  Returns 0, or 1 for   */
/* P > 2 (the paper gives no higher-order source terms).                      */
/* ------------------------------------------------------------------------ */
int orc_run_source(const double *u0, double *u_out, long nsteps, int ndim, const long *shape, const double *nu,
                   int quad, int bc, int P, double beta, double sc, const double *g, const double *f)
{
    if (P < 1 || P > 2) return 1;
    long T = total_size(ndim, shape);
    double *Cg = malloc(sizeof(double) * (size_t)T), *F = malloc(sizeof(double) * (size_t)T);
    double *up = malloc(sizeof(double) * (size_t)T), *uc = malloc(sizeof(double) * (size_t)T);
    double *un = malloc(sizeof(double) * (size_t)T);
    orc_C(g, Cg, ndim, shape, nu, quad, bc);
    memcpy(uc, u0, sizeof(double) * (size_t)T);
    for (long k = 0; k < nsteps; ++k) {
        const double fm = k > 0 ? f[k - 1] : f[1], f0 = f[k], fp = f[k + 1];
        double a, b;
        if (P == 1) { a = sc * f0; b = 0.0; }
        else { a = sc * (fp + 10.0 * f0 + fm) / 12.0; b = -beta * beta * sc * f0 / 12.0; }
        orc_F(uc, F, ndim, shape, nu, quad, bc, P, beta, NULL);
        if (k == 0) {
            for (long i = 0; i < T; ++i) un[i] = uc[i] + 0.5 * (F[i] + a * g[i] + b * Cg[i]);
        } else {
            for (long i = 0; i < T; ++i) un[i] = 2.0 * uc[i] - up[i] + F[i] + a * g[i] + b * Cg[i];
        }
        memcpy(up, uc, sizeof(double) * (size_t)T);
        memcpy(uc, un, sizeof(double) * (size_t)T);
    }
    memcpy(u_out, uc, sizeof(double) * (size_t)T);
    free(Cg); free(F); free(up); free(uc); free(un);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Time-dependent Dirichlet data on a 1D line (Sec. 3.2): u(a, t) = u_L(t),  */
/* u(b, t) = u_R(t).  As an operator on smooth functions D = 1 - L^{-1} =     */
/* -(d_xx/alpha^2)(1 - d_xx/alpha^2)^{-1}, and in the limit x -> a the wave   */
/* equation turns d_xx^j into (d_tt/c^2)^j.  With s_j = (d_tt/(c alpha)^2)^j  */
/* u_L(t) (the data), the boundary value of D^p u expanded to the scheme's   */
/* order is g_p = (-1)^p sum_{j=p}^{P} C(j-1, p-1) s_j (and the same at b).   */
/* One application of D that must return e with e(a) = gL, e(b) = gR        */
/* corrects L^{-1} to w(a) = v(a) - gL, w(b) = v(b) - gR.                      */
/* ------------------------------------------------------------------------ */
void orc_linv_line_bc(const double *v, double *w, long n, double nu, int quad, double gL, double gR)
{
    linv_line_impl(v, 1, w, 1, n, nu, quad, ORC_DIRICHLET, gL, gR);
}

void orc_D_line_bc(const double *v, double *e, long n, double nu, int quad, double gL, double gR)
{
    double *w = malloc(sizeof(double) * (size_t)n);
    orc_linv_line_bc(v, w, n, nu, quad, gL, gR);
    for (long j = 0; j < n; ++j) e[j] = v[j] - w[j];
    free(w);
}

/* F = sum_{p=1}^P A_p D^p u with D^p u = D(D^{p-1} u) taking the boundary
 * values g[2p] (at a) and g[2p + 1] (at b); g[0], g[1] (the data itself)
 * are not used here. */
void orc_F_bc(const double *u, double *F, long n, double nu, int quad, int P, double beta, const double *g)
{
    double A[16];
    orc_Ap(P, beta, A);
    double *v = malloc(sizeof(double) * (size_t)n), *e = malloc(sizeof(double) * (size_t)n);
    memcpy(v, u, sizeof(double) * (size_t)n);
    memset(F, 0, sizeof(double) * (size_t)n);
    for (int p = 1; p <= P; ++p) {
        orc_D_line_bc(v, e, n, nu, quad, g[2 * p], g[2 * p + 1]);
        for (long j = 0; j < n; ++j) F[j] += A[p - 1] * e[j];
        memcpy(v, e, sizeof(double) * (size_t)n);
    }
    free(v); free(e);
}

/* boundary values g[2p + side] (p = 1..P) of D^p u from the data
 * s[side * (P + 1) + j] = (d_tt / (c alpha)^2)^j u_side, j = 0..P */
void orc_bc_values(const double *s, int P, double *g)
{
    for (int side = 0; side < 2; ++side) {
        g[side] = s[side * (P + 1)];
        for (int p = 1; p <= P; ++p) {
            double acc = 0.0;
            for (int j = p; j <= P; ++j) acc += binom(j - 1, p - 1) * s[side * (P + 1) + j];
            g[2 * p + side] = ((p & 1) ? -1.0 : 1.0) * acc;
        }
    }
}

/* u^0 -> u^{nsteps} with the data gam[(k * 2 + side) * (P + 1) + j] =
 * (d_tt / (c alpha)^2)^j u_side(t_k), k = 0 .. nsteps: u^1 = u^0 + F[u^0]/2
 * (zero initial velocity) and u^{k+1} = 2 u^k - u^{k-1} + F[u^k], F with
 * the boundary values from the data at t_k; the end nodes of every new
 * level take the data (j = 0) at its time. */
void orc_run_bc(const double *u0, double *u_out, long nsteps, long n, double nu, int quad, int P, double beta,
                const double *gam)
{
    const int Q = P + 1;
    double *g = malloc(sizeof(double) * 2 * (size_t)Q);
    double *up = malloc(sizeof(double) * (size_t)n), *uc = malloc(sizeof(double) * (size_t)n);
    double *un = malloc(sizeof(double) * (size_t)n), *F = malloc(sizeof(double) * (size_t)n);
    for (long k = 0; k < nsteps; ++k) {
        orc_bc_values(gam + k * 2 * Q, P, g);
        if (k == 0) {
            memcpy(uc, u0, sizeof(double) * (size_t)n);
            orc_F_bc(uc, F, n, nu, quad, P, beta, g);
            for (long j = 0; j < n; ++j) un[j] = uc[j] + 0.5 * F[j];
        } else {
            orc_F_bc(uc, F, n, nu, quad, P, beta, g);
            for (long j = 0; j < n; ++j) un[j] = 2.0 * uc[j] - up[j] + F[j];
        }
        un[0] = gam[((k + 1) * 2 + 0) * Q];
        un[n - 1] = gam[((k + 1) * 2 + 1) * Q];
        memcpy(up, uc, sizeof(double) * (size_t)n);
        memcpy(uc, un, sizeof(double) * (size_t)n);
    }
    memcpy(u_out, nsteps > 0 ? uc : u0, sizeof(double) * (size_t)n);
    free(g); free(up); free(uc); free(un); free(F);
}

/* ------------------------------------------------------------------------ */
/* The 2D scheme of eq. (Full_2D) on an embedded domain (Sec. 4.3): C and D   */
/* of eqs. (C_def_ADI), (D_def_ADI) built from the line-object operators,     */
/* the terms in the order of Table 3 (on a domain that is not a rectangle the */
/* x and y operators do not commute, so this order is part of the scheme).   */
/* Geometry arrays as in orc_geom; alpha = beta / (c dt).                     */
/* ------------------------------------------------------------------------ */
static orc_geom make_geom(long nx, long ny, double hx, double hy, const long *r0, const long *r1,
                          const double *ra, const double *rb, const long *c0, const long *c1,
                          const double *ca, const double *cb)
{
    orc_geom g = {nx, ny, hx, hy, r0, r1, c0, c1, ra, rb, ca, cb};
    return g;
}

void orc_linv_axis_embed(const double *v, double *w, int axis, long nx, long ny, double hx, double hy,
                         const long *r0, const long *r1, const double *ra, const double *rb, const long *c0,
                         const long *c1, const double *ca, const double *cb, double alpha)
{
    orc_geom g = make_geom(nx, ny, hx, hy, r0, r1, ra, rb, c0, c1, ca, cb);
    linv_axis_obj(&g, v, w, axis, alpha);
}

void orc_F_embed(const double *u, double *F, long nx, long ny, double hx, double hy, const long *r0,
                 const long *r1, const double *ra, const double *rb, const long *c0, const long *c1,
                 const double *ca, const double *cb, double alpha, int P, double beta)
{
    orc_geom g = make_geom(nx, ny, hx, hy, r0, r1, ra, rb, c0, c1, ca, cb);
    long shape[2] = {nx, ny};
    double nu[2] = {alpha * hx, alpha * hy};
    orc_ctx c = {2, shape, nu, 2, ORC_DIRICHLET, nx * ny, 0, 0, &g, alpha};
    F_core(c, u, F, P, beta, NULL);
}

/* u^1 = u^0 + F[u^0]/2, then nsteps - 1 steps u^{n+1} = 2u^n - u^{n-1} + F[u^n];
 * u_out = u^{nsteps} (u^0 when nsteps = 0) */
void orc_run_embed(const double *u0, double *u_out, long nsteps, long nx, long ny, double hx, double hy,
                   const long *r0, const long *r1, const double *ra, const double *rb, const long *c0,
                   const long *c1, const double *ca, const double *cb, double alpha, int P, double beta)
{
    long T = nx * ny;
    double *up = malloc(sizeof(double) * (size_t)T), *uc = malloc(sizeof(double) * (size_t)T);
    double *F = malloc(sizeof(double) * (size_t)T);
    memcpy(uc, u0, sizeof(double) * (size_t)T);
    for (long k = 0; k < nsteps; ++k) {
        orc_F_embed(uc, F, nx, ny, hx, hy, r0, r1, ra, rb, c0, c1, ca, cb, alpha, P, beta);
        for (long i = 0; i < T; ++i) {
            double un = (k == 0) ? uc[i] + 0.5 * F[i] : 2.0 * uc[i] - up[i] + F[i];
            up[i] = uc[i];
            uc[i] = un;
        }
    }
    memcpy(u_out, uc, sizeof(double) * (size_t)T);
    free(up); free(uc); free(F);
}

#ifdef _OPENMP
#include <omp.h>
int orc_num_threads(void) { return omp_get_max_threads(); }
/* threads of the parallel loops that follow (timing only; results do not
   depend on it: every loop is over independent lines) */
void orc_set_threads(int n) { if (n > 0) omp_set_num_threads(n); }
#else
int orc_num_threads(void) { return 1; }
void orc_set_threads(int n) { (void)n; }
#endif
