/*
 * FP64 CPU oracle for MFA-DVR ("MFA-DVR: direct volume rendering of MFA
 * models", Sun, Lenz, Yu, Peterka).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the package smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  The CUDA library never
 * loads it, and the two share no source, header, table or helper.
 *
 * What it computes, as plain definitions in double precision:
 *
 *  - The MFA model (Sec. 2.3, Sec. 3): a tensor product of B-splines of degree
 *    p_d on each axis d, with weights 1, over an n0 x n1 x n2 control-point
 *    lattice and clamped knot vectors on the parameter box [0,1]^3.  Knots:
 *    t_0..t_p = 0, t_{p+j} = j/m for j = 1..m-1, t_n..t_{n+p} = 1, m = n - p,
 *    unless the model gives its own clamped knot vector for an axis (the
 *    non-uniform knots an adaptive MFA fit places, Sec. 2.3); the span
 *    search and the basis below take any clamped, non-decreasing vector.
 *  - Rational models (NURBS, Sec. 2.3), when the model gives positive
 *    weights w_ijk: f = A / W with A = sum w P N N N and W = sum w N N N (the
 *    homogeneous form), and grad f = (grad A - f grad W) / W (quotient rule).
 *    Without weights the model is the plain tensor-product B-spline.
 *  - Value and first partial derivatives at a parameter point, computed
 *    together (queryValueMFA / queryGradientMFA of Algorithm 1; Sec. 3.1 asks
 *    for all three derivatives at once).  Two modes:
 *      span mode : find the knot span by binary search, evaluate the p+1
 *                  non-zero basis functions and derivatives from the
 *                  Cox-de Boor recurrence, sum the (p+1)^3 terms;
 *      brute mode: evaluate every basis function of the lattice by the raw
 *                  recursive Cox-de Boor definition and sum all n0*n1*n2
 *                  terms (tiny lattices only).
 *  - The ray caster of Algorithm 1 (Sec. 3.1): a ray per pixel, samples at a
 *    constant distance between the first and last sample inside the volume,
 *    the sample position normalised to [0,1]^3, value -> RGBA through a
 *    transfer function, optional gradient shading, front-to-back compositing
 *    and early ray termination once the cumulative opacity exceeds O_max.
 *
 * Readings where the paper is silent (camera model, sample placement, TF
 * interpolation, opacity correction, the shading formula) are stated beside
 * the code that implements them.  Rows of the image are split over threads as
 * in Algorithm 1 (each thread owns a set of rows).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_DEGREE 16

/* ------------------------------------------------------------------------ */
/* Knots, spans, basis functions                                             */
/* ------------------------------------------------------------------------ */

/* Clamped uniform knot vector of length n+p+1 (the model of Sec. 2.3 with
 * uniformly spaced interior knots). Returns 0, or -1 on bad sizes. */
int orc_make_knots(int n, int p, double *t)
{
    if (p < 1 || n < p + 1) return -1;
    int m = n - p;
    for (int i = 0; i <= p; ++i) t[i] = 0.0;
    for (int j = 1; j < m; ++j) t[p + j] = (double)j / (double)m;
    for (int i = n; i <= n + p; ++i) t[i] = 1.0;
    return 0;
}

/* Knot span s in [p, n-1] with t_s <= u < t_{s+1}; u at or beyond the right
 * end belongs to the last span, u at or before the left end to the first.
 * Binary search over the knot vector. */
int orc_find_span(int n, int p, const double *t, double u)
{
    if (u >= t[n]) return n - 1;
    if (u <= t[p]) return p;
    int lo = p, hi = n; /* invariant: t[lo] <= u < t[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (u < t[mid]) hi = mid;
        else lo = mid;
    }
    return lo;
}

/* The p+1 basis functions that are non-zero on span s, N_{s-p+r,p}(u) for
 * r = 0..p, and their first derivatives, from the Cox-de Boor recurrence
 *   N_{i,0}(u) = 1 on [t_i, t_{i+1}),
 *   N_{i,q}(u) = (u - t_i)/(t_{i+q} - t_i) N_{i,q-1}(u)
 *              + (t_{i+q+1} - u)/(t_{i+q+1} - t_{i+1}) N_{i+1,q-1}(u),
 *   N'_{i,p}(u) = p/(t_{i+p} - t_i) N_{i,p-1}(u)
 *              - p/(t_{i+p+1} - t_{i+1}) N_{i+1,p-1}(u).
 * B[q][r] holds N_{s-q+r,q}(u). */
void orc_basis_ders(int s, double u, int p, const double *t, double *N, double *dN)
{
    double B[ORC_MAX_DEGREE + 1][ORC_MAX_DEGREE + 1];
    B[0][0] = 1.0;
    for (int q = 1; q <= p; ++q) {
        for (int r = 0; r <= q; ++r) {
            int i = s - q + r;
            double val = 0.0;
            if (r > 0) /* N_{i,q-1} = B[q-1][r-1] */
                val += (u - t[i]) / (t[i + q] - t[i]) * B[q - 1][r - 1];
            if (r < q) /* N_{i+1,q-1} = B[q-1][r] */
                val += (t[i + q + 1] - u) / (t[i + q + 1] - t[i + 1]) * B[q - 1][r];
            B[q][r] = val;
        }
    }
    for (int r = 0; r <= p; ++r) {
        int i = s - p + r;
        double d = 0.0;
        if (r > 0) d += (double)p / (t[i + p] - t[i]) * B[p - 1][r - 1];
        if (r < p) d -= (double)p / (t[i + p + 1] - t[i + 1]) * B[p - 1][r];
        N[r] = B[p][r];
        dN[r] = d;
    }
}

/* Raw recursive definition of N_{i,q}(u) over the whole knot vector, with
 * 0/0 := 0.  The interval of the last non-empty span is closed on the right,
 * so that u = 1 evaluates to the limit from the left. */
double orc_basis_brute(int i, int q, double u, const double *t, int n)
{
    if (q == 0) {
        if (t[i] <= u && u < t[i + 1]) return 1.0;
        if (u >= t[n] && i == n - 1) return 1.0;
        return 0.0;
    }
    double v = 0.0;
    double d1 = t[i + q] - t[i];
    double d2 = t[i + q + 1] - t[i + 1];
    if (d1 > 0.0) v += (u - t[i]) / d1 * orc_basis_brute(i, q - 1, u, t, n);
    if (d2 > 0.0) v += (t[i + q + 1] - u) / d2 * orc_basis_brute(i + 1, q - 1, u, t, n);
    return v;
}

/* First derivative of N_{i,p}(u) from the derivative formula, brute mode. */
double orc_basis_brute_der(int i, int p, double u, const double *t, int n)
{
    double v = 0.0;
    double d1 = t[i + p] - t[i];
    double d2 = t[i + p + 1] - t[i + 1];
    if (d1 > 0.0) v += (double)p / d1 * orc_basis_brute(i, p - 1, u, t, n);
    if (d2 > 0.0) v -= (double)p / d2 * orc_basis_brute(i + 1, p - 1, u, t, n);
    return v;
}

/* k-th derivative of N_{i,p} at u by applying the derivative formula of the
 * definition recursively: D^k N_{i,p} = p (D^{k-1} N_{i,p-1} / (t_{i+p} - t_i)
 * - D^{k-1} N_{i+1,p-1} / (t_{i+p+1} - t_{i+1})), a term with a zero knot
 * difference dropped; D^0 is the raw recursion above.  k > p gives 0. */
double orc_basis_brute_dk(int i, int p, int k, double u, const double *t, int n)
{
    if (k == 0) return orc_basis_brute(i, p, u, t, n);
    if (k > p) return 0.0;
    double v = 0.0;
    const double d1 = t[i + p] - t[i];
    const double d2 = t[i + p + 1] - t[i + 1];
    if (d1 > 0.0) v += (double)p / d1 * orc_basis_brute_dk(i, p - 1, k - 1, u, t, n);
    if (d2 > 0.0) v -= (double)p / d2 * orc_basis_brute_dk(i + 1, p - 1, k - 1, u, t, n);
    return v;
}

/* ------------------------------------------------------------------------ */
/* Model and point queries                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t p[3];        /* degree per axis (u, v, w) */
    int32_t n[3];        /* control points per axis */
    const double *ctrl;  /* n0*n1*n2, index i + n0*(j + n1*k) (u fastest) */
    double box_min[3];   /* world box that maps onto the parameter box */
    double box_max[3];
    const double *knots[3]; /* NULL: clamped uniform knots; else the n+p+1
                               clamped, non-decreasing knots of the axis */
    const double *weights;  /* NULL: non-rational; else n0*n1*n2 positive
                               weights, indexed like ctrl */
} orc_model;

typedef struct {
    const orc_model *m;
    double *t[3];        /* knot vectors */
} orc_ctx;

static int ctx_init(orc_ctx *c, const orc_model *m)
{
    c->m = m;
    for (int d = 0; d < 3; ++d) c->t[d] = NULL;
    if (m->weights) { /* weights must be positive and finite */
        const size_t count = (size_t)m->n[0] * (size_t)m->n[1] * (size_t)m->n[2];
        for (size_t i = 0; i < count; ++i)
            if (!(m->weights[i] > 0.0) || !isfinite(m->weights[i])) return -1;
    }
    for (int d = 0; d < 3; ++d) {
        if (m->p[d] < 1 || m->p[d] > ORC_MAX_DEGREE || m->n[d] < m->p[d] + 1) return -1;
        const int n = m->n[d], p = m->p[d];
        c->t[d] = (double *)malloc(sizeof(double) * (size_t)(n + p + 1));
        if (!c->t[d]) return -1;
        if (!m->knots[d]) {
            orc_make_knots(n, p, c->t[d]);
            continue;
        }
        /* a given vector must be clamped to [0, 1] and non-decreasing */
        const double *t = m->knots[d];
        for (int i = 0; i <= p; ++i)
            if (t[i] != 0.0 || t[n + i] != 1.0) return -1;
        for (int i = 1; i < n + p + 1; ++i)
            if (!(t[i] >= t[i - 1])) return -1;
        memcpy(c->t[d], t, sizeof(double) * (size_t)(n + p + 1));
    }
    return 0;
}

static void ctx_free(orc_ctx *c)
{
    for (int d = 0; d < 3; ++d) free(c->t[d]);
}

static double clamp01(double x)
{
    return fmin(fmax(x, 0.0), 1.0); /* fmax(NaN, 0) = 0 */
}

static double ctrl_at(const orc_model *m, int i, int j, int k)
{
    return m->ctrl[(size_t)i + (size_t)m->n[0] * ((size_t)j + (size_t)m->n[1] * (size_t)k)];
}

static double weight_at(const orc_model *m, int i, int j, int k)
{
    return m->weights[(size_t)i + (size_t)m->n[0] * ((size_t)j + (size_t)m->n[1] * (size_t)k)];
}

/* Rational model: the value and gradient of A / W from the homogeneous sums
 * h = (A, A_u, A_v, A_w) and g = (W, W_u, W_v, W_w). */
static void rational_quotient(const double h[4], const double g[4], double out[4])
{
    const double f = h[0] / g[0];
    out[0] = f;
    for (int d = 1; d < 4; ++d) out[d] = (h[d] - f * g[d]) / g[0];
}

/* f, df/du, df/dv, df/dw at parameter point q (already in [0,1]^3), span
 * mode.  The spans are written to s3 when it is not NULL. */
static void eval_span(const orc_ctx *c, const double q[3], double out[4], int32_t *s3)
{
    const orc_model *m = c->m;
    double N[3][ORC_MAX_DEGREE + 1], dN[3][ORC_MAX_DEGREE + 1];
    int s[3];
    for (int d = 0; d < 3; ++d) {
        s[d] = orc_find_span(m->n[d], m->p[d], c->t[d], q[d]);
        orc_basis_ders(s[d], q[d], m->p[d], c->t[d], N[d], dN[d]);
        if (s3) s3[d] = s[d];
    }
    if (m->weights) {
        double h[4] = {0, 0, 0, 0}, g[4] = {0, 0, 0, 0};
        for (int c2 = 0; c2 <= m->p[2]; ++c2)
            for (int b = 0; b <= m->p[1]; ++b)
                for (int a = 0; a <= m->p[0]; ++a) {
                    const int i = s[0] - m->p[0] + a, j = s[1] - m->p[1] + b, k = s[2] - m->p[2] + c2;
                    const double w = weight_at(m, i, j, k), wP = w * ctrl_at(m, i, j, k);
                    const double B[4] = {N[0][a] * N[1][b] * N[2][c2], dN[0][a] * N[1][b] * N[2][c2],
                                         N[0][a] * dN[1][b] * N[2][c2], N[0][a] * N[1][b] * dN[2][c2]};
                    for (int d = 0; d < 4; ++d) {
                        h[d] += B[d] * wP;
                        g[d] += B[d] * w;
                    }
                }
        rational_quotient(h, g, out);
        return;
    }
    double f = 0, fu = 0, fv = 0, fw = 0;
    for (int c2 = 0; c2 <= m->p[2]; ++c2)
        for (int b = 0; b <= m->p[1]; ++b)
            for (int a = 0; a <= m->p[0]; ++a) {
                double P = ctrl_at(m, s[0] - m->p[0] + a, s[1] - m->p[1] + b, s[2] - m->p[2] + c2);
                f += N[0][a] * N[1][b] * N[2][c2] * P;
                fu += dN[0][a] * N[1][b] * N[2][c2] * P;
                fv += N[0][a] * dN[1][b] * N[2][c2] * P;
                fw += N[0][a] * N[1][b] * dN[2][c2] * P;
            }
    out[0] = f; out[1] = fu; out[2] = fv; out[3] = fw;
}

/* Same quantities by brute mode: all n0*n1*n2 terms, raw recursion. */
static void eval_brute(const orc_ctx *c, const double q[3], double out[4])
{
    const orc_model *m = c->m;
    double *N[3], *dN[3];
    for (int d = 0; d < 3; ++d) {
        N[d] = (double *)malloc(sizeof(double) * (size_t)m->n[d]);
        dN[d] = (double *)malloc(sizeof(double) * (size_t)m->n[d]);
        for (int i = 0; i < m->n[d]; ++i) {
            N[d][i] = orc_basis_brute(i, m->p[d], q[d], c->t[d], m->n[d]);
            dN[d][i] = orc_basis_brute_der(i, m->p[d], q[d], c->t[d], m->n[d]);
        }
    }
    double h[4] = {0, 0, 0, 0}, g[4] = {0, 0, 0, 0};
    for (int k = 0; k < m->n[2]; ++k)
        for (int j = 0; j < m->n[1]; ++j)
            for (int i = 0; i < m->n[0]; ++i) {
                const double w = m->weights ? weight_at(m, i, j, k) : 1.0, wP = w * ctrl_at(m, i, j, k);
                const double B[4] = {N[0][i] * N[1][j] * N[2][k], dN[0][i] * N[1][j] * N[2][k],
                                     N[0][i] * dN[1][j] * N[2][k], N[0][i] * N[1][j] * dN[2][k]};
                for (int d = 0; d < 4; ++d) {
                    h[d] += B[d] * wP;
                    g[d] += B[d] * w;
                }
            }
    if (m->weights) rational_quotient(h, g, out);
    else for (int d = 0; d < 4; ++d) out[d] = h[d];
    for (int d = 0; d < 3; ++d) { free(N[d]); free(dN[d]); }
}

typedef struct {
    const orc_ctx *c;
    int64_t npts, begin, end;
    const float *uvw;
    double *out4;
    int32_t *spans3;
    int brute;
} eval_job;

static void *eval_worker(void *arg)
{
    eval_job *j = (eval_job *)arg;
    for (int64_t i = j->begin; i < j->end; ++i) {
        double q[3];
        for (int d = 0; d < 3; ++d) q[d] = clamp01((double)j->uvw[3 * i + d]);
        if (j->brute) eval_brute(j->c, q, j->out4 + 4 * i);
        else eval_span(j->c, q, j->out4 + 4 * i, j->spans3 ? j->spans3 + 3 * i : NULL);
    }
    return NULL;
}

/* Value and parameter-space gradient at npts points uvw (FP32 triples,
 * clamped to [0,1]).  out4: f, df/du, df/dv, df/dw.  spans3 (optional, span
 * mode only): the knot-span index per axis.  Returns 0 or -1. */
int orc_eval_points(const orc_model *m, int64_t npts, const float *uvw, double *out4,
                    int32_t *spans3, int nthreads, int brute)
{
    orc_ctx c;
    if (ctx_init(&c, m)) { ctx_free(&c); return -1; }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    eval_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].c = &c; jobs[t].npts = npts; jobs[t].uvw = uvw; jobs[t].out4 = out4;
        jobs[t].spans3 = spans3; jobs[t].brute = brute;
        jobs[t].begin = npts * t / nthreads;
        jobs[t].end = npts * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, eval_worker, &jobs[t]);
    eval_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    ctx_free(&c);
    return 0;
}

/* Value, gradient and second partial derivatives at npts points uvw (FP32
 * triples clamped to [0,1]), the higher-order query of Sec. 3.1 (Sec. 2:
 * derivatives up to the degree are analytic).  out10 per point: f, f_u,
 * f_v, f_w, f_uu, f_vv, f_ww, f_uv, f_uw, f_vw.  The span comes from the
 * binary search; the derivatives of order 0..2 of the span's p+1 non-zero
 * functions from orc_basis_brute_dk.  A rational model differentiates
 * f = A / W twice: f_i = (A_i - f W_i) / W and
 * f_ij = (A_ij - f_i W_j - f_j W_i - f W_ij) / W.  Single-threaded (small
 * cases).  Returns 0 or -1. */
int orc_eval_hessian(const orc_model *m, int64_t npts, const float *uvw, double *out10)
{
    orc_ctx c;
    if (ctx_init(&c, m)) { ctx_free(&c); return -1; }
    /* (a, b) derivative orders per output: [out][axis] */
    static const int ord[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                   {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    for (int64_t q = 0; q < npts; ++q) {
        double x[3];
        int s[3];
        double D[3][3][ORC_MAX_DEGREE + 1]; /* [axis][order][r] */
        for (int d = 0; d < 3; ++d) {
            x[d] = clamp01((double)uvw[3 * q + d]);
            s[d] = orc_find_span(m->n[d], m->p[d], c.t[d], x[d]);
            for (int k = 0; k < 3; ++k)
                for (int r = 0; r <= m->p[d]; ++r)
                    D[d][k][r] = orc_basis_brute_dk(s[d] - m->p[d] + r, m->p[d], k, x[d], c.t[d], m->n[d]);
        }
        double h[10] = {0}, g[10] = {0};
        for (int cc = 0; cc <= m->p[2]; ++cc)
            for (int b = 0; b <= m->p[1]; ++b)
                for (int a = 0; a <= m->p[0]; ++a) {
                    const int i = s[0] - m->p[0] + a, j = s[1] - m->p[1] + b, k = s[2] - m->p[2] + cc;
                    const double w = m->weights ? weight_at(m, i, j, k) : 1.0, wP = w * ctrl_at(m, i, j, k);
                    for (int o = 0; o < 10; ++o) {
                        const double B = D[0][ord[o][0]][a] * D[1][ord[o][1]][b] * D[2][ord[o][2]][cc];
                        h[o] += B * wP;
                        g[o] += B * w;
                    }
                }
        double *out = out10 + 10 * q;
        if (!m->weights) {
            for (int o = 0; o < 10; ++o) out[o] = h[o];
            continue;
        }
        const double W = g[0], f = h[0] / W;
        double f1[3];
        for (int d = 0; d < 3; ++d) f1[d] = (h[1 + d] - f * g[1 + d]) / W;
        out[0] = f;
        for (int d = 0; d < 3; ++d) out[1 + d] = f1[d];
        /* second derivatives: outputs 4..9 with axis pairs (0,0) (1,1) (2,2) (0,1) (0,2) (1,2) */
        static const int pr[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
        for (int o = 0; o < 6; ++o) {
            const int di = pr[o][0], dj = pr[o][1];
            out[4 + o] = (h[4 + o] - f1[di] * g[1 + dj] - f1[dj] * g[1 + di] - f * g[4 + o]) / W;
        }
    }
    ctx_free(&c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Ray caster (Algorithm 1)                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t kind;          /* 0 orthographic, 1 perspective */
    double eye[3], center[3], up[3];
    double fovy_deg;       /* perspective: vertical field of view */
    double ortho_height;   /* orthographic: world height of the image */
} orc_camera;

typedef struct {
    int32_t width, height;
    double step;           /* constant sample distance (world units) */
    double max_opacity;    /* O_max: stop once cumulative opacity > O_max */
    double ref_step;       /* opacity-correction reference; <= 0 means = step */
    const float *tf_rgba;  /* tf_size RGBA entries */
    int32_t tf_size;
    double tf_lo, tf_hi;   /* value range of the TF; NaN = [min P, max P] */
    int32_t shading;
    double ka, kd, ks, shininess;
} orc_render_params;

/* Decision ties: an FP32 implementation may take the other branch where the
 * exact quantity sits this close to a threshold.
 *  - (t_exit - t_enter)/step: ORC_TIE_SAMPLES plus a per-ray bound of the
 *    FP32 rounding of the ray and the slab test (box_hit), which grows where
 *    a direction component comes out of cancelling terms.
 *  - cumulative opacity: each FP32 sample opacity 1 - (1 - a)^r carries an
 *    absolute rounding error near 6e-8, and rays run to a few thousand
 *    samples before the strict test A > O_max. */
#define ORC_TIE_SAMPLES 2e-3  /* distance of (t_exit - t_enter)/step from an integer */
#define ORC_TIE_OPACITY 2e-4  /* distance of the cumulative opacity from O_max */

typedef struct {
    orc_ctx c;
    const orc_camera *cam;
    const orc_render_params *rp;
    double fwd[3], right[3], upv[3];
    double lo, hi, gthresh;
    int row_step, nthreads, brute;
    double *rgba, *rgba_alt;
    int32_t *nsamples, *nambig, *ns_lo, *ns_hi;
} render_job;

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double a[3])
{
    double l = sqrt(dot3(a, a));
    a[0] /= l; a[1] /= l; a[2] /= l;
}

/* Relative rounding unit of FP32 with headroom for a few chained
 * operations; it sizes the tie window of the sample count. */
#define ORC_F32_EPS (8.0 / 16777216.0)

/* Ray through the centre of pixel (x, y), row 0 at the top (the "Ray
 * Definition" step of Sec. 3.1; the camera model itself is a reading).
 * eo/ed (optional): per component, a bound on how far an FP32 evaluation of
 * the same formulas can move the origin and the unit direction (the sums
 * cancel, so the bound scales with the magnitudes of their terms). */
static void make_ray(const render_job *J, int x, int y, double o[3], double d[3], double eo[3], double ed[3])
{
    const orc_camera *cam = J->cam;
    double W = J->rp->width, H = J->rp->height;
    double aspect = W / H;
    if (cam->kind == 0) {
        double sx = ((x + 0.5) / W - 0.5) * cam->ortho_height * aspect;
        double sy = (0.5 - (y + 0.5) / H) * cam->ortho_height;
        for (int a = 0; a < 3; ++a) {
            o[a] = cam->eye[a] + sx * J->right[a] + sy * J->upv[a];
            d[a] = J->fwd[a];
            if (eo) eo[a] = ORC_F32_EPS * (fabs(cam->eye[a]) + fabs(sx * J->right[a]) + fabs(sy * J->upv[a]));
            if (ed) ed[a] = ORC_F32_EPS;
        }
    } else {
        double th = tan(cam->fovy_deg * (M_PI / 180.0) * 0.5);
        double sx = (2.0 * (x + 0.5) / W - 1.0) * th * aspect;
        double sy = (1.0 - 2.0 * (y + 0.5) / H) * th;
        double mag[3];
        for (int a = 0; a < 3; ++a) {
            o[a] = cam->eye[a];
            d[a] = J->fwd[a] + sx * J->right[a] + sy * J->upv[a];
            mag[a] = fabs(J->fwd[a]) + fabs(sx * J->right[a]) + fabs(sy * J->upv[a]);
        }
        double l = sqrt(dot3(d, d));
        for (int a = 0; a < 3; ++a) {
            d[a] /= l;
            if (eo) eo[a] = ORC_F32_EPS * fabs(cam->eye[a]);
            if (ed) ed[a] = ORC_F32_EPS * (mag[a] / l + fabs(d[a]));
        }
    }
}

/* Slab test against the world box; [t_enter, t_exit] with t_enter >= 0.
 * Returns 0 on a miss.  With eo/ed given, e0/e1 bound how far FP32 can move
 * t_enter and t_exit: t = (b - o)/d moves by (|eo| + eps|b - o|)/|d| +
 * |t| |ed|/|d| on the slab that decides it. */
static int box_hit(const orc_model *m, const double o[3], const double d[3], double *t0, double *t1,
                   const double eo[3], const double ed[3], double *e0, double *e1)
{
    double a0 = 0.0, a1 = INFINITY, b0 = 0.0, b1 = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < m->box_min[a] || o[a] > m->box_max[a]) return 0;
            continue;
        }
        double ta = (m->box_min[a] - o[a]) / d[a];
        double tb = (m->box_max[a] - o[a]) / d[a];
        double ea = 0.0, eb = 0.0;
        if (eo && ed) {
            ea = (eo[a] + ORC_F32_EPS * fabs(m->box_min[a] - o[a])) / fabs(d[a]) + fabs(ta) * ed[a] / fabs(d[a]);
            eb = (eo[a] + ORC_F32_EPS * fabs(m->box_max[a] - o[a])) / fabs(d[a]) + fabs(tb) * ed[a] / fabs(d[a]);
        }
        if (ta > tb) {
            double s = ta; ta = tb; tb = s;
            s = ea; ea = eb; eb = s;
        }
        if (ta > a0) { a0 = ta; b0 = ea; }
        if (tb < a1) { a1 = tb; b1 = eb; }
    }
    if (!(a1 > a0)) return 0;
    *t0 = a0; *t1 = a1;
    if (e0) *e0 = b0;
    if (e1) *e1 = b1;
    return 1;
}

/* Value -> RGBA: linear interpolation in the table over [lo, hi] (the paper
 * names TF_Color and TF_Opacity; one RGBA table carries both). */
static void tf_lookup(const render_job *J, double v, double rgba[4])
{
    const orc_render_params *rp = J->rp;
    int nt = rp->tf_size;
    double x = (J->hi > J->lo) ? clamp01((v - J->lo) / (J->hi - J->lo)) : 0.0;
    if (nt == 1) {
        for (int c = 0; c < 4; ++c) rgba[c] = rp->tf_rgba[c];
        return;
    }
    x *= (double)(nt - 1);
    int i = (int)floor(x);
    if (i > nt - 2) i = nt - 2;
    double fr = x - i;
    for (int c = 0; c < 4; ++c) {
        double a = rp->tf_rgba[4 * i + c], b = rp->tf_rgba[4 * (i + 1) + c];
        rgba[c] = a + fr * (b - a);
    }
}

/* March one ray.  flip_n != 0 takes the sample-count decision the other way
 * when it is tied.  Returns 1 if the sample count was tied, else 0.
 * out/ns: the pixel and sample count of the exact FP64 march.
 * [ns_lo, ns_hi]: the sample counts an implementation whose cumulative
 * opacity stays within ORC_TIE_OPACITY of the exact one can stop at: from
 * the first sample with A > O_max - tol to the first with A > O_max + tol
 * (or the last sample). */
static int march(const render_job *J, int x, int y, int flip_n, double out[4], int32_t *ns, int32_t *ns_lo,
                 int32_t *ns_hi)
{
    const orc_model *m = J->c.m;
    const orc_render_params *rp = J->rp;
    double o[3], d[3], t0, t1;
    int tied = 0;
    out[0] = out[1] = out[2] = out[3] = 0.0;
    *ns = *ns_lo = *ns_hi = 0;
    double eo[3], ed[3], e0 = 0.0, e1 = 0.0;
    make_ray(J, x, y, o, d, eo, ed);
    if (!box_hit(m, o, d, &t0, &t1, eo, ed, &e0, &e1)) return 0;

    /* Samples t_k = t_enter + (k + 1/2) step, k = 0..N-1, N = floor(len/step):
     * every sample lies inside the volume (Sample_First..Sample_Last).  The
     * count is tied when FP32 rounding of the ray and the slab test can move
     * (t_exit - t_enter)/step across an integer. */
    double r = (t1 - t0) / rp->step;
    long N = (long)floor(r);
    double rn = floor(r + 0.5);
    double window = ORC_TIE_SAMPLES + (e0 + e1) / rp->step;
    if (rn >= 1.0 && fabs(r - rn) < window) {
        if (flip_n) N = (N == (long)rn) ? (long)rn - 1 : (long)rn;
        tied = 1;
    }
    double ratio = (rp->ref_step > 0.0) ? rp->step / rp->ref_step : 1.0;
    double ext[3];
    for (int a = 0; a < 3; ++a) ext[a] = m->box_max[a] - m->box_min[a];
    double C[3] = {0, 0, 0}, A = 0.0;
    long k, stop = -1, lo = -1, hi = -1;
    for (k = 0; k < N; ++k) {
        double t = t0 + ((double)k + 0.5) * rp->step;
        double q[3], f[4], rgba[4];
        for (int a = 0; a < 3; ++a) q[a] = clamp01((o[a] + t * d[a] - m->box_min[a]) / ext[a]);
        if (J->brute) eval_brute(&J->c, q, f);
        else eval_span(&J->c, q, f, NULL);
        tf_lookup(J, f[0], rgba);
        double alpha = clamp01(rgba[3]);
        if (ratio != 1.0) alpha = 1.0 - pow(1.0 - alpha, ratio);
        if (rp->shading) {
            /* Gradient shading (Alg. 1, getLightingCoefficient / addShading):
             * Blinn-Phong with one headlight, L = V = -d, so H = L; two-sided.
             * The world gradient is the parameter gradient over the extent. */
            double g[3] = {f[1] / ext[0], f[2] / ext[1], f[3] / ext[2]};
            double gn = sqrt(dot3(g, g));
            if (gn <= J->gthresh) {
                for (int c = 0; c < 3; ++c) rgba[c] *= rp->ka;
            } else {
                double ndl = fabs(-(g[0] * d[0] + g[1] * d[1] + g[2] * d[2]) / gn);
                double spec = pow(ndl, rp->shininess);
                for (int c = 0; c < 3; ++c)
                    rgba[c] = clamp01(rgba[c] * (rp->ka + rp->kd * ndl) + rp->ks * spec);
            }
        }
        /* Front-to-back compositing (doColorCompositing). */
        double w = (1.0 - A) * alpha;
        for (int c = 0; c < 3; ++c) C[c] += w * rgba[c];
        A += w;
        /* Early ray termination: strictly above O_max.  The march goes on
         * past the exact stop only to find where a tied stop could fall. */
        if (lo < 0 && A > rp->max_opacity - ORC_TIE_OPACITY) lo = k + 1;
        if (stop < 0 && A > rp->max_opacity) {
            stop = k + 1;
            out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = A;
        }
        if (A > rp->max_opacity + ORC_TIE_OPACITY) { hi = k + 1; break; }
    }
    if (stop < 0) {
        stop = N;
        out[0] = C[0]; out[1] = C[1]; out[2] = C[2]; out[3] = A;
    }
    if (lo < 0) lo = stop;
    if (hi < 0) hi = N;
    *ns = (int32_t)stop;
    *ns_lo = (int32_t)lo;
    *ns_hi = (int32_t)hi;
    return tied;
}

typedef struct { render_job *J; int tid; } render_arg;

static void *render_worker(void *arg)
{
    render_arg *ra = (render_arg *)arg;
    render_job *J = ra->J;
    int W = J->rp->width, H = J->rp->height;
    int rows_done = 0;
    for (int y = 0; y < H; y += J->row_step) {
        if ((rows_done++ % J->nthreads) != ra->tid) continue;
        for (int x = 0; x < W; ++x) {
            size_t px = (size_t)y * W + x;
            int32_t ns, lo, hi;
            int tied = march(J, x, y, 0, J->rgba + 4 * px, &ns, &lo, &hi);
            J->nsamples[px] = ns;
            if (J->nambig) J->nambig[px] = tied;
            if (tied) {
                /* the other sample count: its pixel, and the union of ranges */
                int32_t ns2, lo2, hi2;
                march(J, x, y, 1, J->rgba_alt + 4 * px, &ns2, &lo2, &hi2);
                if (lo2 < lo) lo = lo2;
                if (hi2 > hi) hi = hi2;
            } else {
                memcpy(J->rgba_alt + 4 * px, J->rgba + 4 * px, 4 * sizeof(double));
            }
            if (J->ns_lo) J->ns_lo[px] = lo;
            if (J->ns_hi) J->ns_hi[px] = hi;
        }
    }
    return NULL;
}

/* Render W x H pixels (row-major, row 0 at the top), premultiplied RGBA.
 * Only rows y = 0, row_step, 2*row_step, ... are rendered.
 *  nsamples: samples composited per pixel by the exact FP64 march;
 *  nambig (optional): 1 where the sample count (t_exit - t_enter)/step is
 *      tied, else 0;
 *  rgba_alt: the pixel with a tied sample count taken the other way (equal
 *      to rgba elsewhere);
 *  ns_lo, ns_hi (optional): the range of sample counts an FP32 march can
 *      stop at (tied sample count and tied early termination included).
 * Returns 0 or -1. */
int orc_render(const orc_model *m, const orc_camera *cam, const orc_render_params *rp,
               int row_step, int nthreads, int brute, double *rgba, int32_t *nsamples,
               int32_t *nambig, double *rgba_alt, int32_t *ns_lo, int32_t *ns_hi)
{
    if (!m || !cam || !rp || !rgba || !nsamples || !rgba_alt) return -1;
    if (rp->width <= 0 || rp->height <= 0 || !(rp->step > 0.0) || rp->tf_size < 1 || !rp->tf_rgba) return -1;
    render_job J;
    memset(&J, 0, sizeof J);
    if (ctx_init(&J.c, m)) { ctx_free(&J.c); return -1; }
    J.cam = cam; J.rp = rp;
    J.row_step = row_step < 1 ? 1 : row_step;
    J.nthreads = nthreads < 1 ? 1 : (nthreads > 256 ? 256 : nthreads);
    J.brute = brute;
    J.rgba = rgba; J.nsamples = nsamples; J.nambig = nambig;
    J.rgba_alt = rgba_alt; J.ns_lo = ns_lo; J.ns_hi = ns_hi;

    /* Camera frame: forward, right = up x forward, true up = forward x right. */
    for (int a = 0; a < 3; ++a) J.fwd[a] = cam->center[a] - cam->eye[a];
    normalize3(J.fwd);
    cross3(cam->up, J.fwd, J.right);
    normalize3(J.right);
    cross3(J.fwd, J.right, J.upv);

    size_t np = (size_t)m->n[0] * m->n[1] * m->n[2];
    double pmin = INFINITY, pmax = -INFINITY, pabs = 0.0;
    for (size_t i = 0; i < np; ++i) {
        double v = m->ctrl[i];
        if (v < pmin) pmin = v;
        if (v > pmax) pmax = v;
        if (fabs(v) > pabs) pabs = fabs(v);
    }
    J.lo = isnan(rp->tf_lo) ? pmin : rp->tf_lo;
    J.hi = isnan(rp->tf_hi) ? pmax : rp->tf_hi;
    J.gthresh = 1e-20 * pabs;

    pthread_t th[256];
    render_arg args[256];
    for (int t = 0; t < J.nthreads; ++t) { args[t].J = &J; args[t].tid = t; }
    for (int t = 1; t < J.nthreads; ++t) pthread_create(&th[t], NULL, render_worker, &args[t]);
    render_worker(&args[0]);
    for (int t = 1; t < J.nthreads; ++t) pthread_join(th[t], NULL);
    ctx_free(&J.c);
    return 0;
}
