/*
 * pdhg_oracle.c -- plain FP64 CPU oracle for batched restarted reflected-Halpern
 * PDHG ("Batched First-Order Methods for Parallel LP Solving in MIP").
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file's library.  It shares no code,
 * header or constant with the CUDA library and never calls it; the CUDA
 * library never calls this.
 *
 * Everything is FP64, loops over CSR, one vector per LP, no blocking and no
 * fusion, in the order of the paper's equations:
 *   Sec. 3, Eq. main_lp / lp_saddle ...... problem, dual, support function phi,
 *                                           barrier cone B
 *   Sec. 4, Eq. mainiter + operator T .... reflected Halpern PDHG step
 *   Sec. 4, Eq. residual ................. fixed-point residual in the M-norm
 *   Sec. 4 "Restarts" .................... three restart conditions
 *   Sec. 4 "Step-size and primal weight" . eta = 0.998/||A||_2, w smoothing
 *   Sec. 4, Eq. stopping ................. relative KKT test, reduced cost
 *   Sec. 4, Eq. primal-infeas/dual-infeas  infeasibility certificates
 *   Sec. 5, Eq. batched_iter ............. batch with per-LP tau, sigma, w and
 *                                           the batch-averaged restart test
 *   Sec. 5.1 / 5.2 ....................... strong-branching / OBBT overrides
 *
 * Readings taken where the paper is silent or garbled (each also stated at
 * the line that implements it):
 *   R1 scaling: 10 Ruiz infinity-norm passes, then Pock-Chambolle alpha=1.
 *   R2 ||A||_2 by power iteration on A~^T A~ from a SplitMix64 start vector.
 *   R3 w0 = ||c~|| / ||b~||, b~_i the finite row bound of larger magnitude.
 *   R4 M-norm cross term taken with a minus sign (standard PDHG metric);
 *      option mnorm_sign = +1 gives the printed plus sign.
 *   R5 restart parameters beta_s=0.2, beta_n=0.8, beta_a=0.36, theta=0.5;
 *      restart anchor = the PDHG output T(z) at the check.
 *   R6 primal weight d = ||dy0|| / ||dx0|| (the printed ratio is inverted
 *      with respect to tau = eta/w, sigma = eta*w).
 *   R7 termination evaluated at T(z^k) in the unscaled space.
 *   R8 primal infeasibility compares against |phi(dy)+phi(dr)| (the printed
 *      right-hand side is negative whenever the first condition holds).
 *   R9 recession cone of an interval infinite on both sides is the real line.
 *   R10 eps for infeasibility = the termination tolerance.
 *   R11 restart averages r over the LPs still active at the check.
 *   R19 the reduced cost of the stopping test is either Pi_B(-c - A^T y) as
 *      printed (reduced_cost = 0, the default) or the variant robust to large
 *      finite bounds that the paper's implementation uses (reduced_cost = 1):
 *      a component counts against a finite bound only where the primal point
 *      is no farther from that bound than from zero (robust_rc below).  The
 *      infeasibility tests keep Pi_B in both modes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* public types (mirrored by oracle/__init__.py through ctypes)              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t m, n;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col_idx;
    const double* vals;
    const double* c;
    const double* row_lo;
    const double* row_hi;
    const double* var_lo;
    const double* var_hi;
} orc_problem;

typedef struct {
    int32_t check_every;
    int32_t ruiz_iters;
    int32_t pock_chambolle;
    int32_t lockstep;            /* 1: one batch, averaged restarts; 0: each LP alone */
    double beta_s, beta_n, beta_a, theta;
    double mnorm_sign;           /* -1 (reading R4) or +1 (as printed) */
    int32_t restart_to_pdhg_output;
    int32_t power_max_iter;
    double power_tol;
    uint64_t power_seed;
    double eps_infeas;           /* < 0: use tol (reading R10) */
    int32_t threads;
    int32_t detect_infeasibility;
    int32_t mutation;            /* 0; a test sets 1..12 to plant one known mistake */
    int32_t reduced_cost;        /* 0: Pi_B as printed; 1: robust to large bounds (R19) */
} orc_options;

typedef struct {
    int32_t status;
    int32_t restarts;
    int64_t iters;
    double obj, dual_obj, rel_primal, rel_dual, rel_gap;
} orc_result;

enum { ORC_OPTIMAL = 0, ORC_PRIMAL_INFEASIBLE = 1, ORC_DUAL_INFEASIBLE = 2,
       ORC_ITERATION_LIMIT = 3, ORC_NUMERICAL = 4 };
enum { ORC_KIND_BASE = 0, ORC_KIND_BOUND = 1, ORC_KIND_OBJECTIVE = 2 };

void orc_default_options(orc_options* o) {
    o->check_every = 64;
    o->ruiz_iters = 10;
    o->pock_chambolle = 1;
    o->lockstep = 1;
    o->beta_s = 0.2;
    o->beta_n = 0.8;
    o->beta_a = 0.36;
    o->theta = 0.5;
    o->mnorm_sign = -1.0;
    o->restart_to_pdhg_output = 1;
    o->power_max_iter = 5000;
    o->power_tol = 1e-10;
    o->power_seed = 0x5eedULL;
    o->eps_infeas = -1.0;
    o->threads = 1;
    o->detect_infeasibility = 1;
    o->mutation = 0;
    o->reduced_cost = 0;
}

/* Planted mistakes, used only by the test that checks the pins catch them:
 *  1 x-step sign flipped        2 dual step without its projection term
 *  3 Halpern anchor term dropped 4 reduced cost left out of the dual residual
 *  5 c scaled by 1/D_c           6 support function with a and b swapped
 *  7 M-norm diagonal weights swapped
 *  8 robust reduced cost paired with the wrong bound
 *  9 primal-weight ratio inverted (||dx|| / ||dy||, as printed)              */
static int32_t g_mutation = 0;
void orc_set_mutation(int32_t k) { g_mutation = k; }

/* ------------------------------------------------------------------------ */
/* Sec. 3 primitives                                                        */
/* ------------------------------------------------------------------------ */

/* Pi_[a,b](v) = max(min(v, b), a), elementwise (Sec. 4, after Eq. mainiter). */
static double proj_box(double v, double a, double b) {
    double t = v < b ? v : b;
    return t > a ? t : a;
}

/* Euclidean projection onto the barrier cone B_[a,b] (Sec. 3):
 * v >= 0 where a = -inf, v <= 0 where b = +inf, free where both finite. */
static double proj_barrier(double v, double a, double b) {
    int lo_inf = isinf(a), hi_inf = isinf(b);
    if (lo_inf && hi_inf) return 0.0;
    if (lo_inf) return v > 0.0 ? v : 0.0;
    if (hi_inf) return v < 0.0 ? v : 0.0;
    return v;
}

/* Projection onto the recession cone R_[a,b] (Sec. 4, after Eq. dual-infeas):
 * 0 where both bounds are finite, >= 0 where only b is infinite, <= 0 where
 * only a is infinite, free where both are infinite (reading R9). */
static double proj_recession(double v, double a, double b) {
    int lo_inf = isinf(a), hi_inf = isinf(b);
    if (lo_inf && hi_inf) return v;
    if (hi_inf) return v > 0.0 ? v : 0.0;
    if (lo_inf) return v < 0.0 ? v : 0.0;
    return 0.0;
}

/* Reduced cost robust to large finite bounds (Sec. 4 "Stopping criteria":
 * the paper's implementation replaces Pi_B by the variant of PDLP's
 * Appendix A; reading R19).  A component v of -c - A^T y pairs with the
 * upper bound b when positive and with the lower bound a when negative (the
 * pairing of phi_[a,b]).  It is kept as a reduced cost only where that bound
 * is finite and the primal value x lies no farther from it than from zero,
 * |x - bound| <= |x|; otherwise the component is 0 and v stays in the dual
 * residual c + A^T y + r.  With x on the paired bound this equals Pi_B(v).  */
static double robust_rc(double v, double x, double a, double b) {
    if (g_mutation == 8) { double t = a; a = b; b = t; }
    if (v > 0.0) return (!isinf(b) && fabs(x - b) <= fabs(x)) ? v : 0.0;
    if (v < 0.0) return (!isinf(a) && fabs(x - a) <= fabs(x)) ? v : 0.0;
    return 0.0;
}

/* One term of phi_[a,b](v) = b^T v_+ + a^T v_- (Sec. 3), with 0 * inf = 0. */
static double support_term(double v, double a, double b) {
    if (g_mutation == 6) { double t = a; a = b; b = t; }
    if (v > 0.0) return b * v;
    if (v < 0.0) return a * v;
    return 0.0;
}

/* exported elementwise helpers (pinned by hand-computed vectors in tests) */
void orc_project_box(int32_t k, const double* v, const double* a, const double* b, double* out) {
    for (int32_t i = 0; i < k; ++i) out[i] = proj_box(v[i], a[i], b[i]);
}
void orc_project_barrier(int32_t k, const double* v, const double* a, const double* b, double* out) {
    for (int32_t i = 0; i < k; ++i) out[i] = proj_barrier(v[i], a[i], b[i]);
}
void orc_project_recession(int32_t k, const double* v, const double* a, const double* b, double* out) {
    for (int32_t i = 0; i < k; ++i) out[i] = proj_recession(v[i], a[i], b[i]);
}
void orc_robust_reduced_cost(int32_t k, const double* v, const double* x, const double* a, const double* b,
                             double* out) {
    for (int32_t i = 0; i < k; ++i) out[i] = robust_rc(v[i], x[i], a[i], b[i]);
}
double orc_support(int32_t k, const double* v, const double* a, const double* b) {
    double s = 0.0;
    for (int32_t i = 0; i < k; ++i) s += support_term(v[i], a[i], b[i]);
    return s;
}

/* ------------------------------------------------------------------------ */
/* CSR products                                                             */
/* ------------------------------------------------------------------------ */
static void csr_mv(int32_t m, const int64_t* rp, const int32_t* ci, const double* v,
                   const double* x, double* out) {
    for (int32_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += v[e] * x[ci[e]];
        out[i] = s;
    }
}

/* out = A^T y using the CSR of A (scatter form; no transpose is stored). */
static void csr_tmv(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci, const double* v,
                    const double* y, double* out) {
    for (int32_t j = 0; j < n; ++j) out[j] = 0.0;
    for (int32_t i = 0; i < m; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) out[ci[e]] += v[e] * y[i];
}

static double* dvec(int64_t k) { return (double*)calloc((size_t)(k > 0 ? k : 1), sizeof(double)); }

static double dot(int64_t k, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < k; ++i) s += a[i] * b[i];
    return s;
}
static double nrm2(int64_t k, const double* a) { return sqrt(dot(k, a, a)); }

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number     */
/* generators", OOPSLA 2014): state += golden gamma, then the mix13 finaliser */
/* ------------------------------------------------------------------------ */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t index) {
    uint64_t z = seed + (index + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* uniform in [-1, 1) from the top 53 bits */
static double splitmix_sym(uint64_t seed, uint64_t index) {
    return 2.0 * ((double)(orc_splitmix64_at(seed, index) >> 11) * 0x1.0p-53) - 1.0;
}

/* ------------------------------------------------------------------------ */
/* R2: ||A||_2 by power iteration on A^T A (the paper fixes eta = 0.998/||A||_2
 * but not how ||A||_2 is obtained).  sigma_est = ||A v|| for unit v; stop when
 * the estimate changes by <= tol relative, or after max_iter products.      */
/* ------------------------------------------------------------------------ */
double orc_norm2_estimate(int32_t m, int32_t n, const int64_t* rp, const int32_t* ci,
                          const double* vals, int32_t max_iter, double tol, uint64_t seed,
                          int32_t* iters_out) {
    double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* u = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t j = 0; j < n; ++j) v[j] = splitmix_sym(seed, (uint64_t)j);
    double nv = nrm2(n, v);
    if (nv > 0) for (int32_t j = 0; j < n; ++j) v[j] /= nv;
    double est = 0.0, prev = -1.0;
    int32_t it = 0;
    for (it = 1; it <= max_iter; ++it) {
        csr_mv(m, rp, ci, vals, v, u);
        est = nrm2(m, u);
        csr_tmv(m, n, rp, ci, vals, u, w);
        double nw = nrm2(n, w);
        if (!(nw > 0.0)) break;
        for (int32_t j = 0; j < n; ++j) v[j] = w[j] / nw;
        if (prev >= 0.0 && fabs(est - prev) <= tol * est) break;
        prev = est;
    }
    if (iters_out) *iters_out = it;
    free(v); free(u); free(w);
    return est;
}

/* ------------------------------------------------------------------------ */
/* R1: Ruiz equilibration then Pock-Chambolle (alpha = 1).  A~ = D_r A D_c.  */
/* Zero rows / columns keep scale 1.                                         */
/* ------------------------------------------------------------------------ */
void orc_scaling(const orc_problem* p, int32_t ruiz_iters, int32_t pock_chambolle,
                 double* D_r, double* D_c) {
    int32_t m = p->m, n = p->n;
    double* rs = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* cs = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int32_t i = 0; i < m; ++i) D_r[i] = 1.0;
    for (int32_t j = 0; j < n; ++j) D_c[j] = 1.0;
    for (int32_t it = 0; it < ruiz_iters; ++it) {
        for (int32_t i = 0; i < m; ++i) rs[i] = 0.0;
        for (int32_t j = 0; j < n; ++j) cs[j] = 0.0;
        for (int32_t i = 0; i < m; ++i)
            for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) {
                int32_t j = p->col_idx[e];
                double a = fabs(D_r[i] * p->vals[e] * D_c[j]);
                if (a > rs[i]) rs[i] = a;
                if (a > cs[j]) cs[j] = a;
            }
        for (int32_t i = 0; i < m; ++i) if (rs[i] > 0.0) D_r[i] /= sqrt(rs[i]);
        for (int32_t j = 0; j < n; ++j) if (cs[j] > 0.0) D_c[j] /= sqrt(cs[j]);
    }
    if (pock_chambolle) {
        for (int32_t i = 0; i < m; ++i) rs[i] = 0.0;
        for (int32_t j = 0; j < n; ++j) cs[j] = 0.0;
        for (int32_t i = 0; i < m; ++i)
            for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e) {
                int32_t j = p->col_idx[e];
                double a = fabs(D_r[i] * p->vals[e] * D_c[j]);
                rs[i] += a;
                cs[j] += a;
            }
        for (int32_t i = 0; i < m; ++i) if (rs[i] > 0.0) D_r[i] /= g_mutation == 12 ? rs[i] : sqrt(rs[i]);
        for (int32_t j = 0; j < n; ++j) if (cs[j] > 0.0) D_c[j] /= g_mutation == 12 ? cs[j] : sqrt(cs[j]);
    }
    free(rs); free(cs);
}

/* ------------------------------------------------------------------------ */
/* per-LP data from the shared LP and one override record (Sec. 5.1, 5.2)   */
/* ------------------------------------------------------------------------ */
static void lp_vectors(const orc_problem* p, int32_t kind, int32_t var, double lo, double hi,
                       double sign, double* c, double* xl, double* xu) {
    int32_t n = p->n;
    for (int32_t j = 0; j < n; ++j) { c[j] = p->c[j]; xl[j] = p->var_lo[j]; xu[j] = p->var_hi[j]; }
    if (kind == ORC_KIND_BOUND && var >= 0 && var < n) {
        if (lo > xl[var]) xl[var] = lo;          /* child box = base box intersected */
        if (hi < xu[var]) xu[var] = hi;          /* with the override interval       */
    } else if (kind == ORC_KIND_OBJECTIVE && var >= 0 && var < n) {
        for (int32_t j = 0; j < n; ++j) c[j] = 0.0;  /* C = [I, -I] columns */
        c[var] = sign;
    }
}

/* ------------------------------------------------------------------------ */
/* Eq. stopping: relative KKT of (x, y) in the original space.               */
/* out = {obj, dual_obj, rel_primal, rel_dual, rel_gap}; rc_mode 1 takes the */
/* robust reduced cost (R19) in place of Pi_B.                               */
/* ------------------------------------------------------------------------ */
static void kkt_eval(const orc_problem* p, const double* c, const double* xl, const double* xu,
                     const double* x, const double* y, double* ax, double* aty, int rc_mode, double* out) {
    int32_t m = p->m, n = p->n;
    csr_mv(m, p->row_ptr, p->col_idx, p->vals, x, ax);
    csr_tmv(m, n, p->row_ptr, p->col_idx, p->vals, y, aty);
    double pres2 = 0.0, ax2 = 0.0, phy = 0.0;
    for (int32_t i = 0; i < m; ++i) {
        double d = ax[i] - proj_box(ax[i], p->row_lo[i], p->row_hi[i]);
        pres2 += d * d;
        ax2 += ax[i] * ax[i];
        phy += support_term(y[i], p->row_lo[i], p->row_hi[i]);
    }
    double dres2 = 0.0, c2 = 0.0, ctx = 0.0, phr = 0.0;
    for (int32_t j = 0; j < n; ++j) {
        double q = c[j] + aty[j];
        double r = rc_mode ? robust_rc(-q, x[j], xl[j], xu[j])   /* R19 */
                           : proj_barrier(-q, xl[j], xu[j]);      /* r = Pi_B(-c - A^T y) */
        double d = g_mutation == 4 ? q : q + r;      /* c + A^T y + r */
        dres2 += d * d;
        c2 += c[j] * c[j];
        ctx += c[j] * x[j];
        phr += support_term(r, xl[j], xu[j]);
    }
    double rel_p = sqrt(pres2) / (1.0 + sqrt(ax2));
    double rel_d = sqrt(dres2) / (1.0 + sqrt(c2));
    double dsum = phr + phy;
    double rel_g = isfinite(dsum) ? fabs(ctx + dsum) / (1.0 + fabs(ctx) + fabs(dsum)) : INFINITY;
    out[0] = ctx;
    out[1] = -dsum;
    out[2] = rel_p;
    out[3] = rel_d;
    out[4] = rel_g;
}

void orc_kkt_rc(const orc_problem* p, int32_t kind, int32_t var, double lo, double hi, double sign,
                const double* x, const double* y, int32_t rc_mode, double* out) {
    int32_t m = p->m, n = p->n;
    double* c = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* xl = c + n;
    double* xu = xl + n;
    double* ax = (double*)malloc(sizeof(double) * (size_t)(m + 1));
    double* aty = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    lp_vectors(p, kind, var, lo, hi, sign, c, xl, xu);
    kkt_eval(p, c, xl, xu, x, y, ax, aty, rc_mode, out);
    free(c); free(ax); free(aty);
}

void orc_kkt(const orc_problem* p, int32_t kind, int32_t var, double lo, double hi, double sign,
             const double* x, const double* y, double* out) {
    orc_kkt_rc(p, kind, var, lo, hi, sign, x, y, 0, out);
}

/* ------------------------------------------------------------------------ */
/* the solver                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    /* original-space LP j */
    double *c, *xl, *xu;
    /* scaled-space LP j: c~ = D_c c, box / D_c */
    double *cs, *xls, *xus;
    /* iterates (scaled): z^k, anchor z^{n,0}, T(z^k), next Halpern iterate */
    double *x, *y, *x0, *y0, *xh, *yh, *xn, *yn;
    /* scratch */
    double *g, *xb, *h, *dx, *adx, *xo, *yo, *ax, *aty, *tn, *tm;
    double w, tau, sigma, r;
    int32_t active, status, restarts;
    int64_t iters;
    double kkt[5];
    int32_t lp;               /* index into the caller's batch */
} lp_state;

typedef struct {
    const orc_problem* p;
    orc_problem ps;           /* scaled A~ */
    double* svals;
    const double *Dr, *Dc;
    double *lts, *uts;        /* scaled row bounds */
    double eta;
    int32_t rc_mode;          /* orc_options.reduced_cost */
} shared_data;


static void lp_alloc(lp_state* s, int32_t m, int32_t n) {
    memset(s, 0, sizeof(*s));
    s->c = dvec(n); s->xl = dvec(n); s->xu = dvec(n);
    s->cs = dvec(n); s->xls = dvec(n); s->xus = dvec(n);
    s->x = dvec(n); s->x0 = dvec(n); s->xh = dvec(n); s->xn = dvec(n);
    s->y = dvec(m); s->y0 = dvec(m); s->yh = dvec(m); s->yn = dvec(m);
    s->g = dvec(n); s->xb = dvec(n); s->dx = dvec(n); s->xo = dvec(n); s->aty = dvec(n); s->tn = dvec(n);
    s->h = dvec(m); s->adx = dvec(m); s->yo = dvec(m); s->ax = dvec(m); s->tm = dvec(m);
}
static void lp_free(lp_state* s) {
    double* v[] = {s->c, s->xl, s->xu, s->cs, s->xls, s->xus, s->x, s->x0, s->xh, s->xn, s->y, s->y0,
                   s->yh, s->yn, s->g, s->xb, s->dx, s->xo, s->aty, s->tn, s->h, s->adx, s->yo, s->ax, s->tm};
    for (size_t i = 0; i < sizeof(v) / sizeof(v[0]); ++i) free(v[i]);
}

/* The PDHG operator T of Sec. 4 on scaled data:
 *   x^ = Pi_[xl,xu](x - tau (c + A^T y))
 *   y^ = y + sigma A(2x^ - x) - sigma Pi_[l,u](y/sigma + A(2x^ - x))
 * g (n), xb (n), h (m) are scratch.                                          */
static void apply_T(const orc_problem* a, const double* c, const double* xl, const double* xu,
                    const double* l, const double* u, double tau, double sigma, const double* x,
                    const double* y, double* g, double* xb, double* h, double* xh, double* yh) {
    int32_t m = a->m, n = a->n;
    csr_tmv(m, n, a->row_ptr, a->col_idx, a->vals, y, g);
    double ts = g_mutation == 1 ? -tau : tau;
    for (int32_t j = 0; j < n; ++j) {
        xh[j] = proj_box(x[j] - ts * (c[j] + g[j]), xl[j], xu[j]);
        xb[j] = 2.0 * xh[j] - x[j];
    }
    csr_mv(m, a->row_ptr, a->col_idx, a->vals, xb, h);
    for (int32_t i = 0; i < m; ++i) {
        double v = y[i] / sigma + h[i];
        /* y + sigma*h - sigma*Pi(v) written as sigma*(v - Pi(v)): the same
         * quantity, and exactly 0 where Pi(v) = v, so y^ stays in the barrier
         * cone of [l, u] without rounding noise. */
        yh[i] = g_mutation == 2 ? sigma * v : sigma * (v - proj_box(v, l[i], u[i]));
    }
}

/* exported for the nonexpansiveness pin: T applied to (x, y) */
void orc_apply_T(const orc_problem* a, const double* c, const double* xl, const double* xu,
                 const double* l, const double* u, double tau, double sigma, const double* x,
                 const double* y, double* xh, double* yh) {
    int32_t m = a->m, n = a->n;
    double* g = dvec(n);
    double* xb = dvec(n);
    double* h = dvec(m);
    apply_T(a, c, xl, xu, l, u, tau, sigma, x, y, g, xb, h, xh, yh);
    free(g); free(xb); free(h);
}

/* Eq. residual: ||(dx, dy)||_M^2 with M = [[w/eta I, s A^T], [s A, 1/(eta w) I]],
 * s = mnorm_sign; adx (m) receives A dx.                                     */
static double mnorm2(const orc_problem* a, double w, double eta, double sgn, const double* dx,
                     const double* dy, double* adx) {
    int32_t m = a->m, n = a->n;
    csr_mv(m, a->row_ptr, a->col_idx, a->vals, dx, adx);
    double dx2 = dot(n, dx, dx), dy2 = dot(m, dy, dy), cross = dot(m, dy, adx);
    double wx = w / eta, wy = 1.0 / (eta * w);
    if (g_mutation == 7) { double t = wx; wx = wy; wy = t; }
    return wx * dx2 + wy * dy2 + 2.0 * sgn * cross;
}

double orc_mnorm2(const orc_problem* a, double w, double eta, double sgn, const double* dx,
                  const double* dy) {
    double* adx = dvec(a->m);
    double r = mnorm2(a, w, eta, sgn, dx, dy, adx);
    free(adx);
    return r;
}

/* One application of T and the reflected Halpern update (Eq. mainiter) for LP
 * s at inner index k:  z_next = (k+1)/(k+2) (2 T(z) - z) + z0/(k+2).         */
static void pdhg_step(const shared_data* sd, lp_state* s, int64_t k) {
    int32_t m = sd->ps.m, n = sd->ps.n;
    apply_T(&sd->ps, s->cs, s->xls, s->xus, sd->lts, sd->uts, s->tau, s->sigma, s->x, s->y, s->g,
            s->xb, s->h, s->xh, s->yh);
    double ca = (double)(k + 1) / (double)(k + 2), cb = g_mutation == 3 ? 0.0 : 1.0 / (double)(k + 2);
    for (int32_t j = 0; j < n; ++j) s->xn[j] = ca * (2.0 * s->xh[j] - s->x[j]) + cb * s->x0[j];
    for (int32_t i = 0; i < m; ++i) s->yn[i] = ca * (2.0 * s->yh[i] - s->y[i]) + cb * s->y0[i];
}

/* Check-time evaluation of LP s at z^k (Eq. residual, stopping, primal-infeas,
 * dual-infeas).  Returns the LP's new status, or -1 to keep iterating.      */
static int32_t evaluate(const shared_data* sd, lp_state* s, double tol, double eps_inf,
                        double mnorm_sign, int detect_inf) {
    const orc_problem* p = sd->p;
    const orc_problem* a = &sd->ps;
    int32_t m = p->m, n = p->n;
    const double eta = sd->eta;
    /* Eq. residual: r = ||T(z) - z||_M */
    for (int32_t j = 0; j < n; ++j) s->dx[j] = s->xh[j] - s->x[j];
    for (int32_t i = 0; i < m; ++i) s->tm[i] = s->yh[i] - s->y[i];
    double r2 = mnorm2(a, s->w, eta, mnorm_sign, s->dx, s->tm, s->adx);
    s->r = sqrt(r2 > 0.0 ? r2 : 0.0);

    /* R7: KKT at T(z) in the original space, x = D_c x~, y = D_r y~ */
    for (int32_t j = 0; j < n; ++j) s->xo[j] = proj_box(sd->Dc[j] * s->xh[j], s->xl[j], s->xu[j]);
    for (int32_t i = 0; i < m; ++i) s->yo[i] = sd->Dr[i] * s->yh[i];
    kkt_eval(p, s->c, s->xl, s->xu, s->xo, s->yo, s->ax, s->aty, sd->rc_mode, s->kkt);
    for (int k = 0; k < 5; ++k)
        if (isnan(s->kkt[k]) || !isfinite(s->r)) return ORC_NUMERICAL;
    if (s->kkt[2] <= tol && s->kkt[3] <= tol && s->kkt[4] <= tol) return ORC_OPTIMAL;
    if (!detect_inf) return -1;

    /* Eq. primal-infeas with dy = Pi_B(y~ - y), dr = Pi_B(r~ - r) */
    {
        double* dyo = s->tm;   /* dy, original space */
        double* atdy = s->tn;  /* A^T dy */
        for (int32_t i = 0; i < m; ++i)
            dyo[i] = proj_barrier(sd->Dr[i] * (s->yh[i] - s->y[i]), p->row_lo[i], p->row_hi[i]);
        double phi_dy = 0.0;
        for (int32_t i = 0; i < m; ++i) phi_dy += support_term(dyo[i], p->row_lo[i], p->row_hi[i]);
        /* r^k needs A^T y^k; reuse s->g as scratch for it */
        double* yk = s->adx;   /* adx no longer needed */
        for (int32_t i = 0; i < m; ++i) yk[i] = sd->Dr[i] * s->y[i];
        double* atyk = s->g;
        csr_tmv(m, n, p->row_ptr, p->col_idx, p->vals, yk, atyk);
        csr_tmv(m, n, p->row_ptr, p->col_idx, p->vals, dyo, atdy);
        double phi_dr = 0.0, res2 = 0.0;
        for (int32_t j = 0; j < n; ++j) {
            double rt = proj_barrier(-s->c[j] - s->aty[j], s->xl[j], s->xu[j]);
            double rk = proj_barrier(-s->c[j] - atyk[j], s->xl[j], s->xu[j]);
            double dr = proj_barrier(rt - rk, s->xl[j], s->xu[j]);
            phi_dr += support_term(dr, s->xl[j], s->xu[j]);
            double t = atdy[j] + dr;
            res2 += t * t;
        }
        double ph = phi_dy + phi_dr;
        if (ph < 0.0 && sqrt(res2) <= eps_inf * fabs(ph)) return ORC_PRIMAL_INFEASIBLE;  /* R8 */
    }
    /* Eq. dual-infeas with dx = x~ - x (original space) */
    {
        double* dxo = s->tn;
        double* adxo = s->tm;
        double cdx = 0.0, rx2 = 0.0, ra2 = 0.0;
        for (int32_t j = 0; j < n; ++j) {
            dxo[j] = sd->Dc[j] * (s->xh[j] - s->x[j]);
            cdx += s->c[j] * dxo[j];
            double t = dxo[j] - proj_recession(dxo[j], s->xl[j], s->xu[j]);
            rx2 += t * t;
        }
        csr_mv(m, p->row_ptr, p->col_idx, p->vals, dxo, adxo);
        for (int32_t i = 0; i < m; ++i) {
            double t = adxo[i] - proj_recession(adxo[i], p->row_lo[i], p->row_hi[i]);
            ra2 += t * t;
        }
        if (cdx < 0.0 && sqrt(rx2) <= eps_inf * fabs(cdx) && sqrt(ra2) <= eps_inf * fabs(cdx))
            return ORC_DUAL_INFEASIBLE;
    }
    return -1;
}

static void finish(const shared_data* sd, lp_state* s, int32_t status, int64_t iters,
                   double* x_out, double* y_out, orc_result* res) {
    const orc_problem* p = sd->p;
    s->active = 0;
    s->status = status;
    s->iters = iters;
    orc_result* r = &res[s->lp];
    r->status = status;
    r->restarts = s->restarts;
    r->iters = iters;
    r->obj = s->kkt[0];
    r->dual_obj = s->kkt[1];
    r->rel_primal = s->kkt[2];
    r->rel_dual = s->kkt[3];
    r->rel_gap = s->kkt[4];
    if (x_out) memcpy(x_out + (int64_t)s->lp * p->n, s->xo, sizeof(double) * (size_t)p->n);
    if (y_out) memcpy(y_out + (int64_t)s->lp * p->m, s->yo, sizeof(double) * (size_t)p->m);
}

/* Run the restarted loop on the LPs of `st` (count `cnt`) as one batch. */
static void run_group(const shared_data* sd, lp_state* st, int32_t cnt, double tol, int64_t max_iter,
                      const orc_options* o, double* x_out, double* y_out, orc_result* res) {
    const double eps_inf = o->eps_infeas >= 0.0 ? o->eps_infeas : tol;
    int32_t m = sd->p->m, n = sd->p->n;
    int64_t k = 0;
    double r0 = -1.0, r_prev = -1.0;
    int32_t nact = 0;
    for (int32_t j = 0; j < cnt; ++j) nact += st[j].active;
    int nthreads = o->threads > 0 ? o->threads : 1;
    (void)nthreads;
    for (int64_t K = 0; K < max_iter && nact > 0; ++K) {
        int is_check = ((K + 1) % o->check_every == 0) || (K + 1 == max_iter);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(nthreads)
#endif
        for (int32_t j = 0; j < cnt; ++j)
            if (st[j].active) pdhg_step(sd, &st[j], k);
        if (!is_check) {
            for (int32_t j = 0; j < cnt; ++j)
                if (st[j].active) {
                    memcpy(st[j].x, st[j].xn, sizeof(double) * (size_t)n);
                    memcpy(st[j].y, st[j].yn, sizeof(double) * (size_t)m);
                }
            ++k;
            continue;
        }
        int32_t stat[1];
        (void)stat;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(nthreads)
#endif
        for (int32_t j = 0; j < cnt; ++j)
            if (st[j].active)
                st[j].status = evaluate(sd, &st[j], tol, eps_inf, o->mnorm_sign, o->detect_infeasibility);
        for (int32_t j = 0; j < cnt; ++j)
            if (st[j].active && st[j].status >= 0) finish(sd, &st[j], st[j].status, K + 1, x_out, y_out, res);
        nact = 0;
        double rsum = 0.0;
        for (int32_t j = 0; j < cnt; ++j)
            if (st[j].active) { ++nact; rsum += st[j].r; }
        if (nact == 0) break;
        if (K + 1 == max_iter) break;
        /* Sec. 5 "Restarts": averaged residual over the LPs still active (R11) */
        double rt = rsum / (double)(g_mutation == 11 ? cnt : nact);
        if (r0 < 0.0) { r0 = rt; r_prev = rt; }
        int no_progress = g_mutation == 10 ? rt < r_prev : rt > r_prev;
        int restart = (rt <= o->beta_s * r0) ||                       /* sufficient decay */
                      (rt <= o->beta_n * r0 && no_progress) ||         /* necessary decay, no progress */
                      ((double)k > o->beta_a * (double)K);             /* artificial: k > beta_a K */
        if (restart) {
            for (int32_t j = 0; j < cnt; ++j) {
                lp_state* s = &st[j];
                if (!s->active) continue;
                const double* ax_ = o->restart_to_pdhg_output ? s->xh : s->xn;
                const double* ay_ = o->restart_to_pdhg_output ? s->yh : s->yn;
                /* R6: d = ||y^{n+1,0} - y^{n,0}|| / ||x^{n+1,0} - x^{n,0}|| */
                double ddx = 0.0, ddy = 0.0;
                for (int32_t q = 0; q < n; ++q) { double t = ax_[q] - s->x0[q]; ddx += t * t; }
                for (int32_t q = 0; q < m; ++q) { double t = ay_[q] - s->y0[q]; ddy += t * t; }
                double d = g_mutation == 9 ? sqrt(ddx) / sqrt(ddy) : sqrt(ddy) / sqrt(ddx);
                if (ddx > 0.0 && ddy > 0.0 && isfinite(d) && d > 0.0) {
                    s->w = exp(o->theta * log(d) + (1.0 - o->theta) * log(s->w));
                    s->tau = sd->eta / s->w;
                    s->sigma = sd->eta * s->w;
                }
                memcpy(s->x0, ax_, sizeof(double) * (size_t)n);
                memcpy(s->y0, ay_, sizeof(double) * (size_t)m);
                memcpy(s->x, ax_, sizeof(double) * (size_t)n);
                memcpy(s->y, ay_, sizeof(double) * (size_t)m);
                s->restarts += 1;
            }
            k = 0;
            r0 = rt;
            r_prev = rt;
        } else {
            for (int32_t j = 0; j < cnt; ++j)
                if (st[j].active) {
                    memcpy(st[j].x, st[j].xn, sizeof(double) * (size_t)n);
                    memcpy(st[j].y, st[j].yn, sizeof(double) * (size_t)m);
                }
            ++k;
            r_prev = rt;
        }
    }
    for (int32_t j = 0; j < cnt; ++j)
        if (st[j].active) finish(sd, &st[j], ORC_ITERATION_LIMIT, max_iter, x_out, y_out, res);
}

/* ------------------------------------------------------------------------ */
/* Per-matrix set-up, done once and shared by any number of solves: the      */
/* scaling factors (R1), the scaled values A~ and row bounds, eta (Sec. 4    */
/* "Step-size", R2) and ||b~|| (R3).  The problem's arrays are referenced,   */
/* not copied: they must outlive the prepared object.                       */
/* ------------------------------------------------------------------------ */
struct orc_prepared {
    orc_problem p;            /* the caller's arrays */
    shared_data sd;
    double* Dr;
    double* Dc;
    double bn;                /* ||b~|| (R3) */
};
typedef struct orc_prepared orc_prepared;

orc_prepared* orc_prepare(const orc_problem* p, const orc_options* o) {
    if (!p || !o) return NULL;
    g_mutation = o->mutation;
    int32_t m = p->m, n = p->n;
    orc_prepared* h = (orc_prepared*)calloc(1, sizeof(orc_prepared));
    h->p = *p;
    shared_data* sd = &h->sd;
    sd->p = &h->p;
    h->Dr = dvec(m);
    h->Dc = dvec(n);
    orc_scaling(p, o->ruiz_iters, o->pock_chambolle, h->Dr, h->Dc);
    sd->Dr = h->Dr;
    sd->Dc = h->Dc;
    sd->svals = dvec(p->nnz);
    for (int32_t i = 0; i < m; ++i)
        for (int64_t e = p->row_ptr[i]; e < p->row_ptr[i + 1]; ++e)
            sd->svals[e] = h->Dr[i] * p->vals[e] * h->Dc[p->col_idx[e]];
    sd->ps = *p;
    sd->ps.vals = sd->svals;
    sd->lts = dvec(m);
    sd->uts = dvec(m);
    for (int32_t i = 0; i < m; ++i) { sd->lts[i] = h->Dr[i] * p->row_lo[i]; sd->uts[i] = h->Dr[i] * p->row_hi[i]; }
    /* Sec. 4 "Step-size": eta = 0.998 / ||A~||_2 (R2) */
    double nrm = orc_norm2_estimate(m, n, p->row_ptr, p->col_idx, sd->svals, o->power_max_iter,
                                    o->power_tol, o->power_seed, NULL);
    sd->eta = 0.998 / (nrm > 0.0 ? nrm : 1.0);
    /* R3: ||b~||, b~_i = the finite row bound of larger magnitude */
    double b2 = 0.0;
    for (int32_t i = 0; i < m; ++i) {
        double l = sd->lts[i], u = sd->uts[i], b = 0.0;
        if (isfinite(l) && isfinite(u)) b = fabs(l) > fabs(u) ? l : u;
        else if (isfinite(l)) b = l;
        else if (isfinite(u)) b = u;
        b2 += b * b;
    }
    h->bn = sqrt(b2);
    g_mutation = 0;
    return h;
}

double orc_prepared_eta(const orc_prepared* h) { return h ? h->sd.eta : 0.0; }

void orc_prepared_free(orc_prepared* h) {
    if (!h) return;
    free(h->Dr); free(h->Dc); free(h->sd.svals); free(h->sd.lts); free(h->sd.uts);
    free(h);
}

/* Solve `num_lps` LPs on a prepared matrix.  Override record q: kind[q],
 * var[q], lo[q], hi[q], sign[q].  warm_x (n x num_lps, column q = LP q) and
 * warm_y may be NULL.  x_out / y_out (n x num_lps, m x num_lps) may be NULL.
 * The set-up options of `o` (scaling, power iteration) are those the matrix
 * was prepared with; the rest apply to this solve.  Returns 0, or a negative
 * code for invalid arguments.                                              */
int32_t orc_solve_prepared(const orc_prepared* h, int32_t num_lps, const int32_t* kind, const int32_t* var,
                           const double* lo, const double* hi, const double* sign, double tol, int64_t max_iter,
                           const orc_options* o, const double* warm_x, const double* warm_y, double* x_out,
                           double* y_out, orc_result* res) {
    if (!h || !o || num_lps < 0 || max_iter < 1 || !(tol > 0.0) || o->check_every < 1) return -1;
    g_mutation = o->mutation;
    const orc_problem* p = &h->p;
    int32_t m = p->m, n = p->n;
    shared_data sd = h->sd;
    sd.rc_mode = o->reduced_cost ? 1 : 0;
    const double* Dr = h->Dr;
    const double* Dc = h->Dc;
    const double bn = h->bn;

    lp_state* st = (lp_state*)calloc((size_t)(num_lps > 0 ? num_lps : 1), sizeof(lp_state));
    for (int32_t q = 0; q < num_lps; ++q) {
        lp_state* s = &st[q];
        lp_alloc(s, m, n);
        s->lp = q;
        lp_vectors(p, kind[q], var[q], lo[q], hi[q], sign[q], s->c, s->xl, s->xu);
        int empty_box = 0;
        for (int32_t j = 0; j < n; ++j) {
            s->cs[j] = g_mutation == 5 ? s->c[j] / Dc[j] : Dc[j] * s->c[j];
            s->xls[j] = s->xl[j] / Dc[j];
            s->xus[j] = s->xu[j] / Dc[j];
            if (s->xl[j] > s->xu[j]) empty_box = 1;
        }
        double cn = nrm2(n, s->cs);
        double w0 = cn / bn;
        s->w = (cn > 0.0 && bn > 0.0 && isfinite(w0)) ? w0 : 1.0;
        s->tau = sd.eta / s->w;
        s->sigma = sd.eta * s->w;
        /* z0: Pi_box(0) or the projected warm start */
        for (int32_t j = 0; j < n; ++j) {
            double v = warm_x ? warm_x[(int64_t)q * n + j] / Dc[j] : 0.0;
            s->x[j] = s->x0[j] = proj_box(v, s->xls[j], s->xus[j]);
        }
        for (int32_t i = 0; i < m; ++i) s->y[i] = s->y0[i] = warm_y ? warm_y[(int64_t)q * m + i] / Dr[i] : 0.0;
        s->active = 1;
        s->status = -1;
        if (empty_box) {   /* an override that empties the box: infeasible, 0 iterations */
            for (int k = 0; k < 5; ++k) s->kkt[k] = NAN;
            finish(&sd, s, ORC_PRIMAL_INFEASIBLE, 0, x_out, y_out, res);
        }
    }
    if (o->lockstep) {
        run_group(&sd, st, num_lps, tol, max_iter, o, x_out, y_out, res);
    } else {
        orc_options o1 = *o;
        int nthreads = o->threads > 0 ? o->threads : 1;
        o1.threads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic) num_threads(nthreads)
#endif
        for (int32_t q = 0; q < num_lps; ++q)
            if (st[q].active) run_group(&sd, &st[q], 1, tol, max_iter, &o1, x_out, y_out, res);
    }
    for (int32_t q = 0; q < num_lps; ++q) lp_free(&st[q]);
    free(st);
    g_mutation = 0;
    return 0;
}

/* Solve `num_lps` LPs sharing A: set-up, solve, release (see
 * orc_solve_prepared for the arguments).                                   */
int32_t orc_solve(const orc_problem* p, int32_t num_lps, const int32_t* kind, const int32_t* var,
                  const double* lo, const double* hi, const double* sign, double tol, int64_t max_iter,
                  const orc_options* o, const double* warm_x, const double* warm_y, double* x_out,
                  double* y_out, orc_result* res, double* eta_out) {
    if (!p || !o || num_lps < 0 || max_iter < 1 || !(tol > 0.0) || o->check_every < 1) return -1;
    orc_prepared* h = orc_prepare(p, o);
    if (eta_out) *eta_out = orc_prepared_eta(h);
    int32_t rc = orc_solve_prepared(h, num_lps, kind, var, lo, hi, sign, tol, max_iter, o, warm_x, warm_y,
                                    x_out, y_out, res);
    orc_prepared_free(h);
    return rc;
}
