/*
 * meta_oracle.c -- plain FP64 CPU oracle of semi-Lagrangian geodesic shooting
 * for Metamorphosis / LDDMM image registration (François, Gori, Glaunès,
 * arXiv:2106.08817) and of the gradient of its inexact-matching cost.
 *
 * TEST INFRASTRUCTURE ONLY.  The CUDA library never includes, links or calls
 * this file; the two share no code.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it.
 *
 * Every routine is the plain definition: one loop per formula, no blocking,
 * no fusion.  The only parallelism is "#pragma omp parallel for" over voxels
 * in loops whose iterations are independent (each writes only its own output
 * voxel with a fixed summation order), so results do not depend on the
 * thread count.  Scatter loops (transposes) and reductions stay serial.
 *
 * Conventions (readings of the paper; each is marked where it is used):
 *   - arrays are row-major, axis 0 first; voxel centres at integer indices,
 *     unit spacing; dt = 1/T.
 *   - K: Gaussian with normalised taps w_k ~ exp(-k^2/(2 sigma^2)), |k| <= r,
 *     r = ceil(3 sigma), applied separably with zero padding (Sec. 2.1 takes
 *     V inside C^l_0, fields vanish on the boundary; K is a Gaussian blur).
 *   - D_i: central difference along axis i, neighbour replicated at the edge.
 *   - v = -rho K*(p grad I)  (Eq. 3 first row, with rho standing for rho/mu
 *     so that mu = 0, rho = 1 is LDDMM).
 *   - one step (Sec. 2.3, Eq. 5-9 in semi-Lagrangian form):
 *       y = x - dt v, clamped to the domain; I~ = I_t(y), p~ = p_t(y) by
 *       multilinear interpolation; p_{t+1} = p~ (1 - dt div v);
 *       I_{t+1} = I~ + dt mu p~.
 *   - variant of the momentum update (p_update = 1): p_{t+1} = p~ J with
 *       J = det(Id - dt Dv), Dv_ae = D_e v_a, the Jacobian of the backtrack
 *       Id - dt v, of which 1 - dt div v is the first-order part.
 *   - the two other integration schemes of Sec. 2.3 (shooting and adjoint),
 *       explicit Euler steps of Eq. 5 and of the conservative form of Eq. 7
 *       with the same central differences D:
 *       Eulerian: I_{t+1} = I_t - dt sum_a (D_a I_t) v_a + dt mu p_t,
 *                 p_{t+1} = p_t - dt sum_a D_a (p_t v_a);
 *       hybrid:   I_{t+1} = I~ + dt mu p~ (the semi-Lagrangian advection),
 *                 p_{t+1} = p_t - dt sum_a D_a (p_t v_a) (Eulerian momentum).
 *   - cost (Eq. 4): 1/2 sum (I_T - J)^2 + lambda [ sum_i <m0_i, K m0_i>
 *       + rho sum p0^2 ], m0 = p0 grad S.
 *   - gradient: the exact transpose of the discrete scheme above
 *     (discretise-then-differentiate), which is what automatic
 *     differentiation of the scheme computes (Sec. 3).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXTAPS 4097

typedef struct {
    int ndim;   /* 2 or 3 */
    long n[3];  /* extents, axis 0 first */
    long st[3]; /* element stride of each axis */
    long N;     /* voxel count */
} grid_t;

static int grid_init(grid_t* g, int ndim, const long* dims) {
    if (ndim < 1 || ndim > 3) return -1;
    g->ndim = ndim;
    g->N = 1;
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 2) return -1;
        g->n[a] = dims[a];
        g->N *= dims[a];
    }
    g->st[ndim - 1] = 1;
    for (int a = ndim - 2; a >= 0; --a) g->st[a] = g->st[a + 1] * g->n[a + 1];
    return 0;
}

static void coords(const grid_t* g, long idx, long* c) {
    for (int a = 0; a < g->ndim; ++a) c[a] = (idx / g->st[a]) % g->n[a];
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- K ---- */

/* Gaussian taps of the RKHS kernel: w[k + r] = exp(-k^2 / (2 sigma^2)) / Z,
 * |k| <= r = ceil(3 sigma), Z making them sum to one.  Returns r, or -1. */
int oracle_taps(double sigma, double* w, int cap) {
    if (!(sigma > 0.0)) return -1;
    int r = (int)ceil(3.0 * sigma);
    if (2 * r + 1 > cap) return -1;
    double Z = 0.0;
    for (int k = -r; k <= r; ++k) {
        w[k + r] = exp(-(double)k * (double)k / (2.0 * sigma * sigma));
        Z += w[k + r];
    }
    for (int k = 0; k < 2 * r + 1; ++k) w[k] /= Z;
    return r;
}

/* One 1-D pass along `ax`: out(x) = sum_k w_k in(x + k e_ax), zero outside. */
static void blur_axis(const grid_t* g, int ax, const double* w, int r,
                      const double* in, double* out) {
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < g->N; ++idx) {
        long c[3];
        coords(g, idx, c);
        double s = 0.0;
        for (int k = -r; k <= r; ++k) {
            long q = c[ax] + k;
            if (q < 0 || q >= g->n[ax]) continue; /* zero padding */
            s += w[k + r] * in[idx + (long)k * g->st[ax]];
        }
        out[idx] = s;
    }
}

/* K * f: the separable Gaussian, last axis first.  tmp has N entries. */
static void blur(const grid_t* g, const double* w, int r, const double* in,
                 double* out, double* tmp) {
    const double* src = in;
    for (int ax = g->ndim - 1; ax >= 0; --ax) {
        /* alternate buffers so that the last pass lands in `out` */
        int passes_left = ax + 1;
        double* dst = (passes_left % 2 == 1) ? out : tmp;
        blur_axis(g, ax, w, r, src, dst);
        src = dst;
    }
}

/* ---------------------------------------------------------------- D ---- */

/* D_ax f: (f[x+1] - f[x-1]) / 2 with the neighbour replicated at an edge. */
static void diff_axis(const grid_t* g, int ax, const double* in, double* out) {
#pragma omp parallel for schedule(static)
    for (long idx = 0; idx < g->N; ++idx) {
        long c[3];
        coords(g, idx, c);
        long lo = (c[ax] > 0) ? idx - g->st[ax] : idx;
        long hi = (c[ax] < g->n[ax] - 1) ? idx + g->st[ax] : idx;
        out[idx] = 0.5 * (in[hi] - in[lo]);
    }
}

/* D_ax^T f, by scattering every row of D_ax (serial). */
static void diff_axis_T(const grid_t* g, int ax, const double* in, double* out) {
    memset(out, 0, sizeof(double) * (size_t)g->N);
    for (long idx = 0; idx < g->N; ++idx) {
        long c[3];
        coords(g, idx, c);
        long lo = (c[ax] > 0) ? idx - g->st[ax] : idx;
        long hi = (c[ax] < g->n[ax] - 1) ? idx + g->st[ax] : idx;
        out[hi] += 0.5 * in[idx];
        out[lo] -= 0.5 * in[idx];
    }
}

/* ------------------------------------------------------ interpolation ---- */

/* Foot of the characteristic through voxel c, displaced by disp (y = c + disp),
 * clamped to [0, n-1] per axis (border replication outside the domain).
 * i0 = floor(y), lowered to n-2 at the far edge so that the cell [i0, i0+1]
 * always exists; f = y - i0 in [0, 1].  inside = 1 when the clamp is inactive
 * (0 < y < n-1): the derivative through the clamp is taken as 0 otherwise. */
typedef struct {
    long i0[3];
    double f[3];
    int inside[3];
} foot_t;

static void foot_of(const grid_t* g, const long* c, const double* disp, foot_t* ft) {
    for (int a = 0; a < g->ndim; ++a) {
        double y = (double)c[a] + disp[a];
        double hi = (double)(g->n[a] - 1);
        ft->inside[a] = (y > 0.0 && y < hi);
        double yc = y < 0.0 ? 0.0 : (y > hi ? hi : y);
        long i0 = (long)floor(yc);
        if (i0 > g->n[a] - 2) i0 = g->n[a] - 2;
        ft->i0[a] = i0;
        ft->f[a] = yc - (double)i0;
    }
}

/* Weight of corner `b` (bit a = upper node along axis a) and its linear index. */
static double corner(const grid_t* g, const foot_t* ft, int b, long* lin) {
    double wgt = 1.0;
    long q = 0;
    for (int a = 0; a < g->ndim; ++a) {
        int up = (b >> a) & 1;
        wgt *= up ? ft->f[a] : 1.0 - ft->f[a];
        q += (ft->i0[a] + up) * g->st[a];
    }
    *lin = q;
    return wgt;
}

/* Multilinear interpolant of F at the foot. */
static double interp(const grid_t* g, const foot_t* ft, const double* F) {
    double s = 0.0;
    for (int b = 0; b < (1 << g->ndim); ++b) {
        long q;
        double wgt = corner(g, ft, b, &q);
        s += wgt * F[q];
    }
    return s;
}

/* d/dy_ax of the interpolant at the foot (cell fixed by the floor rule),
 * zero where the clamp on axis ax is active. */
static double interp_deriv(const grid_t* g, const foot_t* ft, int ax, const double* F) {
    if (!ft->inside[ax]) return 0.0;
    double s = 0.0;
    for (int b = 0; b < (1 << g->ndim); ++b) {
        double wgt = 1.0;
        long q = 0;
        for (int a = 0; a < g->ndim; ++a) {
            int up = (b >> a) & 1;
            if (a == ax)
                wgt *= up ? 1.0 : -1.0;
            else
                wgt *= up ? ft->f[a] : 1.0 - ft->f[a];
            q += (ft->i0[a] + up) * g->st[a];
        }
        s += wgt * F[q];
    }
    return s;
}

/* ------------------------------------------------------ forward step ---- */

typedef struct {
    grid_t g;
    int T;
    int pdet; /* momentum update: 0 = p~ (1 - dt div v), 1 = p~ det(Id - dt Dv) */
    int scheme; /* 0 semi-Lagrangian, 1 Eulerian, 2 hybrid (set by oracle_shoot) */
    double dt, mu, rho;
    int r;
    double w[OR_MAXTAPS];
} scheme_t;

static int scheme_init(scheme_t* s, int ndim, const long* dims, int T, double sigma,
                       double mu, double rho, int pdet) {
    if (grid_init(&s->g, ndim, dims) != 0) return -1;
    if (T < 1 || !(mu >= 0.0) || !(rho > 0.0) || (pdet != 0 && pdet != 1)) return -1;
    s->T = T;
    s->pdet = pdet;
    s->scheme = 0;
    s->dt = 1.0 / (double)T;
    s->mu = mu;
    s->rho = rho;
    s->r = oracle_taps(sigma, s->w, OR_MAXTAPS);
    return s->r < 0 ? -1 : 0;
}

/* Quantities of step t that both the forward and the adjoint need. */
typedef struct {
    double* g[3];  /* D_i I_t */
    double* u[3];  /* K (p_t D_i I_t);  v_i = -rho u_i */
    double* div;   /* sum_i D_i v_i */
    double* dv[3][3]; /* D_e v_a, kept for the det update only */
    double* tmp;
    double* tmp2;
} stepbuf_t;

static int stepbuf_alloc(stepbuf_t* b, long N, int ndim, int pdet) {
    memset(b, 0, sizeof(*b));
    for (int a = 0; a < ndim; ++a) {
        b->g[a] = (double*)malloc(sizeof(double) * (size_t)N);
        b->u[a] = (double*)malloc(sizeof(double) * (size_t)N);
        if (!b->g[a] || !b->u[a]) return -1;
        for (int e = 0; pdet && e < ndim; ++e) {
            b->dv[a][e] = (double*)malloc(sizeof(double) * (size_t)N);
            if (!b->dv[a][e]) return -1;
        }
    }
    b->div = (double*)malloc(sizeof(double) * (size_t)N);
    b->tmp = (double*)malloc(sizeof(double) * (size_t)N);
    b->tmp2 = (double*)malloc(sizeof(double) * (size_t)N);
    return (b->div && b->tmp && b->tmp2) ? 0 : -1;
}

static void stepbuf_free(stepbuf_t* b) {
    for (int a = 0; a < 3; ++a) {
        free(b->g[a]);
        free(b->u[a]);
        for (int e = 0; e < 3; ++e) free(b->dv[a][e]);
    }
    free(b->div);
    free(b->tmp);
    free(b->tmp2);
}

/* g = D I, m = p g, u = K m, v = -rho u, div = sum_i D_i v_i. */
static void velocity(const scheme_t* s, const double* I, const double* p, stepbuf_t* b) {
    const grid_t* g = &s->g;
    for (int a = 0; a < g->ndim; ++a) {
        diff_axis(g, a, I, b->g[a]);
        for (long x = 0; x < g->N; ++x) b->tmp[x] = p[x] * b->g[a][x]; /* m_a */
        blur(g, s->w, s->r, b->tmp, b->u[a], b->tmp2);
    }
    for (long x = 0; x < g->N; ++x) b->div[x] = 0.0;
    for (int a = 0; a < g->ndim; ++a) {
        for (long x = 0; x < g->N; ++x) b->tmp[x] = -s->rho * b->u[a][x]; /* v_a */
        diff_axis(g, a, b->tmp, b->tmp2);
        for (long x = 0; x < g->N; ++x) b->div[x] += b->tmp2[x];
        for (int e = 0; s->pdet && e < g->ndim; ++e) diff_axis(g, e, b->tmp, b->dv[a][e]);
    }
}

/* M = Id - dt Dv at voxel x; returns det M and its cofactors
 * cof[a][e] = d det M / d M_ae (the derivative of the determinant). */
static double jacobian_det(const scheme_t* s, const stepbuf_t* b, long x, double cof[3][3]) {
    const int d = s->g.ndim;
    double M[3][3];
    for (int a = 0; a < d; ++a)
        for (int e = 0; e < d; ++e) M[a][e] = (a == e ? 1.0 : 0.0) - s->dt * b->dv[a][e][x];
    if (d == 2) {
        cof[0][0] = M[1][1];
        cof[0][1] = -M[1][0];
        cof[1][0] = -M[0][1];
        cof[1][1] = M[0][0];
        return M[0][0] * M[1][1] - M[0][1] * M[1][0];
    }
    for (int a = 0; a < 3; ++a)
        for (int e = 0; e < 3; ++e) {
            /* minor of (a, e): rows a1 < a2 and columns e1 < e2 other than a and e */
            const int a1 = a == 0 ? 1 : 0, a2 = a == 2 ? 1 : 2;
            const int e1 = e == 0 ? 1 : 0, e2 = e == 2 ? 1 : 2;
            const double minor = M[a1][e1] * M[a2][e2] - M[a1][e2] * M[a2][e1];
            cof[a][e] = ((a + e) % 2 ? -1.0 : 1.0) * minor;
        }
    return M[0][0] * cof[0][0] + M[0][1] * cof[0][1] + M[0][2] * cof[0][2];
}

/* the factor of p~ in p_{t+1}: 1 - dt div v, or det(Id - dt Dv) */
static double p_factor(const scheme_t* s, const stepbuf_t* b, long x) {
    double cof[3][3];
    return s->pdet ? jacobian_det(s, b, x, cof) : 1.0 - s->dt * b->div[x];
}

/* displacement of the foot: y - x = -dt v = dt rho u */
static void displacement(const scheme_t* s, const stepbuf_t* b, long x, double* disp) {
    for (int a = 0; a < s->g.ndim; ++a) disp[a] = -s->dt * (-s->rho * b->u[a][x]);
}

/* Eulerian momentum step: p_{t+1} = p_t - dt sum_a D_a (p_t v_a), conservative form of
 * Eq. 7; uses b->tmp and b->tmp2. */
static void euler_momentum(const scheme_t* s, const double* p, stepbuf_t* b, double* p1) {
    const grid_t* g = &s->g;
    for (long x = 0; x < g->N; ++x) p1[x] = p[x];
    for (int a = 0; a < g->ndim; ++a) {
        for (long x = 0; x < g->N; ++x) b->tmp[x] = p[x] * (-s->rho * b->u[a][x]); /* p v_a */
        diff_axis(g, a, b->tmp, b->tmp2);
        for (long x = 0; x < g->N; ++x) p1[x] -= s->dt * b->tmp2[x];
    }
}

static void step_forward(const scheme_t* s, const double* I, const double* p, stepbuf_t* b,
                         double* I1, double* p1) {
    const grid_t* g = &s->g;
    velocity(s, I, p, b);
    if (s->scheme == 1) { /* Eulerian: Eq. 5 and Eq. 7 by explicit Euler steps */
        for (long x = 0; x < g->N; ++x) {
            double adv = 0.0; /* <grad I, v> */
            for (int a = 0; a < g->ndim; ++a) adv += b->g[a][x] * (-s->rho * b->u[a][x]);
            I1[x] = I[x] - s->dt * adv + s->dt * s->mu * p[x];
        }
        euler_momentum(s, p, b, p1);
        return;
    }
    if (s->scheme == 2) { /* hybrid: semi-Lagrangian I, Eulerian p */
#pragma omp parallel for schedule(static)
        for (long x = 0; x < g->N; ++x) {
            long c[3];
            double disp[3];
            foot_t ft;
            coords(g, x, c);
            displacement(s, b, x, disp);
            foot_of(g, c, disp, &ft);
            I1[x] = interp(g, &ft, I) + s->dt * s->mu * interp(g, &ft, p);
        }
        euler_momentum(s, p, b, p1);
        return;
    }
#pragma omp parallel for schedule(static)
    for (long x = 0; x < g->N; ++x) {
        long c[3];
        double disp[3];
        foot_t ft;
        coords(g, x, c);
        displacement(s, b, x, disp);
        foot_of(g, c, disp, &ft);
        double It = interp(g, &ft, I);
        double pt = interp(g, &ft, p);
        p1[x] = pt * p_factor(s, b, x);
        I1[x] = It + s->dt * s->mu * pt;
    }
}

/* --------------------------------------------------------- public API ---- */

int oracle_blur(int ndim, const long* dims, double sigma, const double* in, double* out) {
    grid_t g;
    double w[OR_MAXTAPS];
    if (grid_init(&g, ndim, dims) != 0) return -1;
    int r = oracle_taps(sigma, w, OR_MAXTAPS);
    if (r < 0) return -1;
    double* tmp = (double*)malloc(sizeof(double) * (size_t)g.N);
    if (!tmp) return -2;
    blur(&g, w, r, in, out, tmp);
    free(tmp);
    return 0;
}

int oracle_diff(int ndim, const long* dims, int axis, int transpose, const double* in,
                double* out) {
    grid_t g;
    if (grid_init(&g, ndim, dims) != 0 || axis < 0 || axis >= ndim) return -1;
    if (transpose)
        diff_axis_T(&g, axis, in, out);
    else
        diff_axis(&g, axis, in, out);
    return 0;
}

/* out = S(y) F (transpose = 0) or S(y)^T F (transpose = 1, scatter), where
 * the foot of voxel x is x + disp[a*N + x] per axis a. */
int oracle_interp(int ndim, const long* dims, const double* disp, int transpose,
                  const double* F, double* out) {
    grid_t g;
    if (grid_init(&g, ndim, dims) != 0) return -1;
    if (transpose) memset(out, 0, sizeof(double) * (size_t)g.N);
    for (long x = 0; x < g.N; ++x) {
        long c[3], q;
        double d[3];
        foot_t ft;
        coords(&g, x, c);
        for (int a = 0; a < ndim; ++a) d[a] = disp[(long)a * g.N + x];
        foot_of(&g, c, d, &ft);
        if (!transpose) {
            out[x] = interp(&g, &ft, F);
        } else {
            for (int b = 0; b < (1 << ndim); ++b) {
                double wgt = corner(&g, &ft, b, &q);
                out[q] += wgt * F[x];
            }
        }
    }
    return 0;
}

/* Shooting: states (I_t, p_t), t = 0..T, written to Itraj/ptraj [(T+1)*N];
 * u_traj (nullable) receives u_t = K(p_t grad I_t), [T*ndim*N].  pdet selects
 * the momentum update (0: p~ (1 - dt div v), 1: p~ det(Id - dt Dv)). */
static int shoot_scheme(int ndim, const long* dims, int T, double sigma, double mu,
                        double rho, int pdet, int scheme, const double* I0, const double* p0,
                        double* Itraj, double* ptraj, double* utraj) {
    scheme_t* s = (scheme_t*)malloc(sizeof(scheme_t));
    if (!s) return -2;
    if (scheme_init(s, ndim, dims, T, sigma, mu, rho, pdet) != 0 || scheme < 0 || scheme > 2 ||
        (scheme != 0 && pdet)) {
        free(s);
        return -1;
    }
    s->scheme = scheme;
    long N = s->g.N;
    stepbuf_t b;
    if (stepbuf_alloc(&b, N, ndim, pdet) != 0) {
        stepbuf_free(&b);
        free(s);
        return -2;
    }
    memcpy(Itraj, I0, sizeof(double) * (size_t)N);
    memcpy(ptraj, p0, sizeof(double) * (size_t)N);
    for (int t = 0; t < T; ++t) {
        step_forward(s, Itraj + (long)t * N, ptraj + (long)t * N, &b,
                     Itraj + (long)(t + 1) * N, ptraj + (long)(t + 1) * N);
        if (utraj)
            for (int a = 0; a < ndim; ++a)
                memcpy(utraj + ((long)t * ndim + a) * N, b.u[a], sizeof(double) * (size_t)N);
    }
    stepbuf_free(&b);
    free(s);
    return 0;
}

int oracle_shoot(int ndim, const long* dims, int T, double sigma, double mu, double rho,
                 int pdet, const double* I0, const double* p0, double* Itraj, double* ptraj,
                 double* utraj) {
    return shoot_scheme(ndim, dims, T, sigma, mu, rho, pdet, 0, I0, p0, Itraj, ptraj, utraj);
}

/* Forward shooting with integration scheme `scheme`: 0 semi-Lagrangian (as
 * oracle_shoot), 1 Eulerian, 2 hybrid (Sec. 2.3; see the header).  pdet must
 * be 0 unless scheme is 0. */
int oracle_shoot_scheme(int ndim, const long* dims, int T, double sigma, double mu, double rho,
                        int pdet, int scheme, const double* I0, const double* p0, double* Itraj,
                        double* ptraj, double* utraj) {
    return shoot_scheme(ndim, dims, T, sigma, mu, rho, pdet, scheme, I0, p0, Itraj, ptraj, utraj);
}

/* Transpose of one Eulerian (scheme 1) or hybrid (scheme 2) step up to v:
 * from (Ih, ph), the adjoints of (I', p'), it writes Inew, pnew (the adjoints of
 * (I, p) through every path except v) and vh (the adjoint of v).
 *   Eulerian: I' = I - dt sum_a g_a v_a + dt mu p, g_a = D_a I
 *   hybrid:   I' = I~ + dt mu p~ (the semi-Lagrangian image step)
 *   both:     p' = p - dt sum_a D_a (p v_a) */
static void other_scheme_T(const scheme_t* s, const double* I, const double* p, stepbuf_t* b,
                           const double* Ih, const double* ph, double* pth, double* Inew,
                           double* pnew, double** vh) {
    const grid_t* g = &s->g;
    const long N = g->N;
    const int d = g->ndim;
    const double dt = s->dt, mu = s->mu, rho = s->rho;
    if (s->scheme == 1) {
        for (long x = 0; x < N; ++x) {
            Inew[x] = Ih[x];
            pnew[x] = ph[x] + dt * mu * Ih[x];
        }
        for (int a = 0; a < d; ++a) {
            for (long x = 0; x < N; ++x) vh[a][x] = -dt * Ih[x] * b->g[a][x];
            /* g_a = D_a I  ->  I_hat += D_a^T (-dt I'_hat v_a) */
            for (long x = 0; x < N; ++x) b->tmp[x] = -dt * Ih[x] * (-rho * b->u[a][x]);
            diff_axis_T(g, a, b->tmp, b->tmp2);
            for (long x = 0; x < N; ++x) Inew[x] += b->tmp2[x];
        }
    } else {
        /* I~ = S I, p~ = S p, y = x - dt v: the adjoint of p~ is dt mu I'_hat */
        for (long x = 0; x < N; ++x) pth[x] = dt * mu * Ih[x];
#pragma omp parallel for schedule(static)
        for (long x = 0; x < N; ++x) {
            long c[3];
            double disp[3];
            foot_t ft;
            coords(g, x, c);
            displacement(s, b, x, disp);
            foot_of(g, c, disp, &ft);
            for (int a = 0; a < d; ++a)
                vh[a][x] = -dt * (interp_deriv(g, &ft, a, I) * Ih[x] +
                                  interp_deriv(g, &ft, a, p) * pth[x]);
        }
        memset(Inew, 0, sizeof(double) * (size_t)N);
        memset(pnew, 0, sizeof(double) * (size_t)N);
        for (long x = 0; x < N; ++x) {
            long c[3], q;
            double disp[3];
            foot_t ft;
            coords(g, x, c);
            displacement(s, b, x, disp);
            foot_of(g, c, disp, &ft);
            for (int bb = 0; bb < (1 << d); ++bb) {
                double wgt = corner(g, &ft, bb, &q);
                Inew[q] += wgt * Ih[x];
                pnew[q] += wgt * pth[x];
            }
        }
        for (long x = 0; x < N; ++x) pnew[x] += ph[x];
    }
    /* p' = p - dt sum_a D_a f_a, f_a = p v_a:  f_hat_a = -dt D_a^T p'_hat */
    for (int a = 0; a < d; ++a) {
        diff_axis_T(g, a, ph, b->tmp);
        for (long x = 0; x < N; ++x) {
            const double fh = -dt * b->tmp[x];
            pnew[x] += fh * (-rho * b->u[a][x]);
            vh[a][x] += fh * p[x];
        }
    }
}

/* Reverse sweep through the T steps.  On entry Ih/ph hold the adjoints of
 * (I_T, p_T); on exit those of (I_0, p_0).  Every step recomputes its forward
 * quantities from the stored state (I_t, p_t).  The i-th line of the step
 * below is the transpose of one assignment of step_forward/velocity. */
static int adjoint_sweep(const scheme_t* s, const double* Itraj, const double* ptraj,
                         double* Ih, double* ph) {
    const grid_t* g = &s->g;
    const long N = g->N;
    const int d = g->ndim;
    const double dt = s->dt;
    stepbuf_t b;
    double *pth = NULL, *dh = NULL, *Inew = NULL, *pnew = NULL, *vh[3] = {0, 0, 0};
    double* dvh[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}; /* adjoint of D_e v_a (det update) */
    int rc = -2;
    if (stepbuf_alloc(&b, N, d, s->pdet) != 0) goto done;
    for (int a = 0; s->pdet && a < d; ++a)
        for (int e = 0; e < d; ++e)
            if (!(dvh[a][e] = (double*)malloc(sizeof(double) * (size_t)N))) goto done;
    pth = (double*)malloc(sizeof(double) * (size_t)N);  /* adjoint of p~ */
    dh = (double*)malloc(sizeof(double) * (size_t)N);   /* adjoint of div v */
    Inew = (double*)malloc(sizeof(double) * (size_t)N);
    pnew = (double*)malloc(sizeof(double) * (size_t)N);
    for (int a = 0; a < d; ++a) vh[a] = (double*)malloc(sizeof(double) * (size_t)N);
    if (!pth || !dh || !Inew || !pnew || !vh[0] || !vh[1] || (d == 3 && !vh[2])) goto done;

    for (int t = s->T - 1; t >= 0; --t) {
        const double* I = Itraj + (long)t * N;
        const double* p = ptraj + (long)t * N;
        velocity(s, I, p, &b);
        if (s->scheme != 0) {
            other_scheme_T(s, I, p, &b, Ih, ph, pth, Inew, pnew, vh);
            goto velocity_T;
        }

        /* pointwise part: I' = I~ + dt mu p~ ; p' = p~ (1 - dt div), or
         * p' = p~ J with J = det M, M = Id - dt Dv, so that
         * Dv_hat_ae = (p~ p'_hat) dJ/dDv_ae = -dt (p~ p'_hat) cof(M)_ae */
#pragma omp parallel for schedule(static)
        for (long x = 0; x < N; ++x) {
            long c[3];
            double disp[3];
            foot_t ft;
            coords(g, x, c);
            displacement(s, &b, x, disp);
            foot_of(g, c, disp, &ft);
            double pt = interp(g, &ft, p);
            if (s->pdet) {
                double cof[3][3];
                const double J = jacobian_det(s, &b, x, cof);
                pth[x] = ph[x] * J + dt * s->mu * Ih[x];
                for (int a = 0; a < d; ++a)
                    for (int e = 0; e < d; ++e) dvh[a][e][x] = -dt * pt * ph[x] * cof[a][e];
            } else {
                pth[x] = ph[x] * (1.0 - dt * b.div[x]) + dt * s->mu * Ih[x];
                dh[x] = -dt * pt * ph[x];
            }
            /* y = x - dt v, so dy_a/dv_a = -dt; I~ and p~ both depend on y */
            for (int a = 0; a < d; ++a) {
                double yh = interp_deriv(g, &ft, a, I) * Ih[x] +
                            interp_deriv(g, &ft, a, p) * pth[x];
                vh[a][x] = -dt * yh;
            }
        }
        /* I~ = S I, p~ = S p  ->  I_hat = S^T I'_hat, p_hat = S^T p~_hat (scatter) */
        memset(Inew, 0, sizeof(double) * (size_t)N);
        memset(pnew, 0, sizeof(double) * (size_t)N);
        for (long x = 0; x < N; ++x) {
            long c[3], q;
            double disp[3];
            foot_t ft;
            coords(g, x, c);
            displacement(s, &b, x, disp);
            foot_of(g, c, disp, &ft);
            for (int bb = 0; bb < (1 << d); ++bb) {
                double wgt = corner(g, &ft, bb, &q);
                Inew[q] += wgt * Ih[x];
                pnew[q] += wgt * pth[x];
            }
        }
        /* div = sum_a D_a v_a  ->  v_hat_a += D_a^T div_hat;
         * det update: Dv_ae = D_e v_a  ->  v_hat_a += sum_e D_e^T Dv_hat_ae */
        for (int a = 0; a < d; ++a) {
            if (s->pdet) {
                for (int e = 0; e < d; ++e) {
                    diff_axis_T(g, e, dvh[a][e], b.tmp);
                    for (long x = 0; x < N; ++x) vh[a][x] += b.tmp[x];
                }
            } else {
                diff_axis_T(g, a, dh, b.tmp);
                for (long x = 0; x < N; ++x) vh[a][x] += b.tmp[x];
            }
        }
    velocity_T:
        for (int a = 0; a < d; ++a) {
            /* v_a = -rho u_a, u_a = K m_a  ->  m_hat_a = K^T(-rho v_hat_a), K^T = K */
            for (long x = 0; x < N; ++x) b.tmp[x] = -s->rho * vh[a][x];
            blur(g, s->w, s->r, b.tmp, b.u[a], b.tmp2); /* b.u[a] now holds m_hat_a */
            /* m_a = p g_a  ->  p_hat += m_hat_a g_a ; I_hat += D_a^T (m_hat_a p) */
            for (long x = 0; x < N; ++x) pnew[x] += b.u[a][x] * b.g[a][x];
            for (long x = 0; x < N; ++x) b.tmp[x] = b.u[a][x] * p[x];
            diff_axis_T(g, a, b.tmp, b.tmp2);
            for (long x = 0; x < N; ++x) Inew[x] += b.tmp2[x];
        }
        memcpy(Ih, Inew, sizeof(double) * (size_t)N);
        memcpy(ph, pnew, sizeof(double) * (size_t)N);
    }
    rc = 0;
done:
    stepbuf_free(&b);
    free(pth);
    free(dh);
    free(Inew);
    free(pnew);
    for (int a = 0; a < 3; ++a) {
        free(vh[a]);
        for (int e = 0; e < 3; ++e) free(dvh[a][e]);
    }
    return rc;
}

/* Adjoint of the shooting map (I0, p0) -> (I_T, p_T): given gI1, gp1 (the
 * gradient of some scalar w.r.t. I_T, p_T; gp1 nullable = 0) returns its
 * gradient w.r.t. I0 (gI0, nullable) and p0 (gp0). */
int oracle_adjoint(int ndim, const long* dims, int T, double sigma, double mu, double rho,
                   int pdet, int scheme, const double* I0, const double* p0, const double* gI1,
                   const double* gp1, double* gI0, double* gp0) {
    scheme_t* s = (scheme_t*)malloc(sizeof(scheme_t));
    if (!s) return -2;
    int rc = scheme_init(s, ndim, dims, T, sigma, mu, rho, pdet);
    if (rc == 0 && (scheme < 0 || scheme > 2 || (scheme != 0 && pdet))) rc = -1;
    if (rc == 0) s->scheme = scheme;
    if (rc != 0) {
        free(s);
        return -1;
    }
    long N = s->g.N;
    double* It = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(T + 1));
    double* pt = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(T + 1));
    double* Ih = (double*)malloc(sizeof(double) * (size_t)N);
    rc = -2;
    if (It && pt && Ih) {
        rc = shoot_scheme(ndim, dims, T, sigma, mu, rho, pdet, scheme, I0, p0, It, pt, NULL);
        if (rc == 0) {
            memcpy(Ih, gI1, sizeof(double) * (size_t)N);
            if (gp1)
                memcpy(gp0, gp1, sizeof(double) * (size_t)N);
            else
                memset(gp0, 0, sizeof(double) * (size_t)N);
            rc = adjoint_sweep(s, It, pt, Ih, gp0);
            if (rc == 0 && gI0) memcpy(gI0, Ih, sizeof(double) * (size_t)N);
        }
    }
    free(It);
    free(pt);
    free(Ih);
    free(s);
    return rc;
}

/* Cost of Eq. 4 and its gradient w.r.t. p0.
 * cost3 = { 1/2 sum (I_T - J)^2, lambda sum_i <m0_i, K m0_i>, lambda rho sum p0^2 }.
 * grad (nullable) = dL/dp0.  pdet as in oracle_shoot. */
int oracle_cost_and_grad(int ndim, const long* dims, int T, double sigma, double mu,
                         double rho, double lambda, int pdet, int scheme, const double* I0,
                         const double* J, const double* p0, double* cost3, double* grad) {
    scheme_t* s = (scheme_t*)malloc(sizeof(scheme_t));
    if (!s) return -2;
    int rc = scheme_init(s, ndim, dims, T, sigma, mu, rho, pdet);
    if (rc == 0 && (scheme < 0 || scheme > 2 || (scheme != 0 && pdet))) rc = -1;
    if (rc == 0) s->scheme = scheme;
    if (rc != 0 || !(lambda >= 0.0)) {
        free(s);
        return -1;
    }
    const grid_t* g = &s->g;
    long N = g->N;
    double* It = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(T + 1));
    double* pt = (double*)malloc(sizeof(double) * (size_t)N * (size_t)(T + 1));
    double* Ih = (double*)malloc(sizeof(double) * (size_t)N);
    double* ph = (double*)malloc(sizeof(double) * (size_t)N);
    stepbuf_t b;
    int have_b = stepbuf_alloc(&b, N, ndim, pdet) == 0;
    rc = -2;
    if (It && pt && Ih && ph && have_b) {
        rc = shoot_scheme(ndim, dims, T, sigma, mu, rho, pdet, scheme, I0, p0, It, pt, NULL);
        if (rc == 0) {
            const double* IT = It + (long)T * N;
            double data = 0.0, kin = 0.0, res = 0.0;
            for (long x = 0; x < N; ++x) data += 0.5 * (IT[x] - J[x]) * (IT[x] - J[x]);
            /* ||v0||_V^2 = <m0, K m0>, m0 = p0 grad S (Eq. 4, no rho^2 factor) */
            velocity(s, I0, p0, &b);
            for (int a = 0; a < ndim; ++a)
                for (long x = 0; x < N; ++x) kin += (p0[x] * b.g[a][x]) * b.u[a][x];
            for (long x = 0; x < N; ++x) res += p0[x] * p0[x];
            cost3[0] = data;
            cost3[1] = lambda * kin;
            cost3[2] = lambda * rho * res;
            if (grad) {
                for (long x = 0; x < N; ++x) {
                    Ih[x] = IT[x] - J[x];
                    ph[x] = 0.0;
                }
                rc = adjoint_sweep(s, It, pt, Ih, ph);
                if (rc == 0) {
                    /* d/dp0 of <m0, K m0> = 2 sum_a g0_a (K m0)_a, K symmetric */
                    velocity(s, I0, p0, &b);
                    for (long x = 0; x < N; ++x) {
                        double kg = 0.0;
                        for (int a = 0; a < ndim; ++a) kg += b.g[a][x] * b.u[a][x];
                        grad[x] = ph[x] + lambda * (2.0 * kg + 2.0 * rho * p0[x]);
                    }
                }
            }
        }
    }
    stepbuf_free(&b);
    (void)have_b;
    free(It);
    free(pt);
    free(Ih);
    free(ph);
    free(s);
    return rc;
}
