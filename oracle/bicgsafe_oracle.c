/*
 * TEST INFRASTRUCTURE — the CPU oracle.  Only tests/, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  The product path
 * (the CUDA library under paper_2108_10591_gb300/) never calls it, and the
 * two share no source, header, helper or table.
 *
 * Plain, slow, single-threaded FP64 implementation of the solvers of
 * Huynh & Suito, "Communication-hiding pipelined BiCGSafe methods for solving
 * large linear systems" (arXiv 2108.10591):
 *   - ssBiCGSafe2           (Section 2, Algorithm 3)
 *   - p-BiCGSafe            (Section 3, Algorithm 4, Eqs. (s)-(g))
 *   - p-BiCGSafe-rr         (Section 4, Algorithm 5)
 * Each iteration follows the listing's statements in the listing's order.
 * Readings where the paper is silent or ambiguous (all also listed in the
 * design notes of the repository):
 *   R1  s_0 = A r_0 for the pipelined variants (Alg. 4/5 use s_0 but never set it).
 *   R2  y_0, t_{-1}, p_{-1}, u_{-1}, z_{-1}, w_{-1}, l_{-1}, g_0 are all zero
 *       (Alg. 2 zero-initialises its auxiliaries; g_0 = A y_0 = 0).
 *   R3  i = 0 uses the listing's special branch (beta=0, alpha=f/g, zeta=d/a, eta=0).
 *   R4  for i>0, a zero or non-finite a*b-c^2 falls back to the i=0 formulas
 *       for zeta and eta (counted); zero g+beta*h, zeta_{i-1} f_{i-1} or a is a
 *       breakdown; any non-finite scalar is reported as non-finite.
 *   R5  nine inner products per iteration (five at i=0), the (r,r) product
 *       moved into the same phase as the stop test (Section 2).
 *   R6  the stop test is on the recursive residual sqrt(r_i) <= eps*||r_0||,
 *       evaluated after the inner products and before the updates; the
 *       returned x is x_i.
 *   R8  shadow residual r0* = r_0.
 *   R9  in Alg. 5 the replacement sets l_i = A t_i.
 *   R10 residual replacement at i mod m == 0, 0 < i < M.
 *   R17 (build addition) block-Jacobi right preconditioning (orc_solve_bjacobi):
 *       the runs above on A M^-1 with M = the diagonal blocks of A, from
 *       y_0 = M x_0, returning x = M^-1 y (see the block-Jacobi section).
 *   R14 (build addition) at recursive convergence the FP64 true residual
 *       ||b - A x|| is computed; if it exceeds eps*||r_0|| of the first run, the
 *       method restarts from x (new r_0 = b - A x, r0* = r_0, auxiliaries
 *       zero) with the same absolute threshold, up to max_restarts times.
 *       Iterations are summed over the runs.
 *
 * Arithmetic: every multiply-add that the listing writes as "a + b*c" is one
 * C99 fma() (correctly rounded); nothing else is contracted (the file is
 * compiled with -ffp-contract=off).  SpMV sums a row's entries sequentially in
 * storage order.  Inner products are correctly rounded (exact sum of exact
 * products, rounded once): the paper writes them as the mathematical (x, y)
 * and fixes no summation order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/*
 * Every loop over rows below is free of cross-row dependences.  The parity
 * build compiles this file without OpenMP and runs them in order; the
 * all-cores timing build (-fopenmp, the CPU baseline only) splits them over
 * threads.  Both give identical bits: each row is computed by the same
 * statements, and an inner product is the exact sum of exact products
 * (per-thread exact partial sums merged exactly) rounded once.
 */
#define ORC_ROWS _Pragma("omp parallel for schedule(static)")

enum { ORC_SSBICGSAFE2 = 0, ORC_P_BICGSAFE = 1, ORC_P_BICGSAFE_RR = 2 };
enum { ORC_OK = 0, ORC_NOT_CONVERGED = 1, ORC_ERR_ARG = -1, ORC_ERR_BREAKDOWN = -3, ORC_ERR_NONFINITE = -5 };

/* Slots of the state dump (see orc_solve). */
enum { SV_X = 0, SV_R, SV_RS, SV_S, SV_Y, SV_T, SV_P, SV_U, SV_Z, SV_W, SV_O, SV_Q, SV_L, SV_G, SV_AS, SV_AW, SV_COUNT };
/* Slots of the scalar dump. */
enum { SC_ALPHA = 0, SC_BETA, SC_ZETA, SC_ETA, SC_A, SC_B, SC_C, SC_D, SC_E, SC_F, SC_G, SC_H, SC_R, SC_RR, SC_I, SC_COUNT };

typedef struct {
    int kind;          /* ORC_SSBICGSAFE2 | ORC_P_BICGSAFE | ORC_P_BICGSAFE_RR */
    double tol;        /* epsilon of the stop test */
    int maxit;         /* total iteration limit over all runs */
    int rr_m, rr_M;    /* residual-replacement epoch m and limit M (Alg. 5) */
    int max_restarts;  /* R14: restarts from x when the true residual is above tol; 0 = paper behaviour */
    int dump_iter;     /* >=0: stop in the first run at iteration dump_iter and dump the state */
    int dump_phase;    /* 0: dump after the scalars of dump_iter, 1: after its vector updates */
} orc_opts;

typedef struct {
    int iterations;        /* total iterations (sum over runs) */
    int restarts;          /* runs after the first */
    int status;            /* ORC_* */
    int fallbacks;         /* R4 fallbacks of zeta/eta to the i=0 formulas */
    int rr_steps;          /* residual replacements performed */
    double rel_res_recursive; /* sqrt(r_i)/||r_0|| at exit (last run) */
    double rel_res_true;   /* ||b - A x||_2 / ||r_0||_2 at exit */
    double r0_norm;        /* ||r_0||_2 of the first run */
} orc_result;

/* ---- building blocks --------------------------------------------------- */

/* y = A x, CSR, each row summed in storage order with fma. */
void orc_spmv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
              const double* x, double* y)
{
    ORC_ROWS
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) acc = fma(val[k], x[col[k]], acc);
        y[i] = acc;
    }
}

/*
 * Inner product (x, y) = sum_i x_i y_i, correctly rounded: every product is
 * formed exactly (53 x 53-bit integer product) and added exactly into a
 * fixed-point integer wide enough for the whole FP64 product range; the exact
 * sum is rounded once, to nearest even.  The result therefore does not depend
 * on the order of the terms.  Any NaN or infinity among the inputs falls back
 * to the plain left-to-right sum so that it propagates as IEEE arithmetic does.
 */
#define XB_LIMBS 70          /* 4480 bits */
#define XB_BIAS 2240         /* bit index of 2^0 */
typedef struct { uint64_t l[XB_LIMBS]; } bigfix;

static void big_addsub(bigfix* a, int limb, uint64_t v, int neg)
{
    /* a += v * 2^(64*limb) or a -= v * 2^(64*limb), two's complement */
    for (int k = limb; k < XB_LIMBS && (v != 0 || neg == 2); ++k) {
        if (!neg) {
            uint64_t o = a->l[k];
            a->l[k] = o + v;
            v = (a->l[k] < o) ? 1 : 0;
        } else {
            uint64_t o = a->l[k];
            a->l[k] = o - v;
            v = (o < v) ? 1 : 0;
        }
    }
}

static void split(double v, uint64_t* m, int* e)
{
    uint64_t b; memcpy(&b, &v, 8);
    int E = (int)((b >> 52) & 0x7FF);
    *m = b & 0xFFFFFFFFFFFFFull;
    if (E) { *m |= 1ull << 52; *e = E - 1075; } else { *e = -1074; }
}

static double big_round(const bigfix* a0)
{
    bigfix a = *a0;
    int neg = (int)(a.l[XB_LIMBS - 1] >> 63);
    if (neg) { /* negate */
        int carry = 1;
        for (int k = 0; k < XB_LIMBS; ++k) {
            uint64_t v = ~a.l[k];
            a.l[k] = v + (uint64_t)carry;
            carry = carry && a.l[k] == 0;
        }
    }
    int top = -1;
    for (int k = XB_LIMBS - 1; k >= 0; --k)
        if (a.l[k]) { top = 64 * k + 63 - __builtin_clzll(a.l[k]); break; }
    if (top < 0) return 0.0;
    int exp_msb = top - XB_BIAS;                   /* value in [2^exp_msb, 2^(exp_msb+1)) */
    int lsb = (exp_msb >= -1022) ? top - 52 : -1074 + XB_BIAS;  /* lowest kept bit (absolute) */
    /* kept bits [lsb, top] (at most 53), round bit lsb-1, sticky below */
    uint64_t mant = 0;
    for (int p = top; p >= lsb; --p) mant = (mant << 1) | ((a.l[p / 64] >> (p % 64)) & 1u);
    int rbit = (lsb - 1 >= 0) ? (int)((a.l[(lsb - 1) / 64] >> ((lsb - 1) % 64)) & 1u) : 0;
    int sticky = 0;
    for (int p = lsb - 2; p >= 0 && !sticky; --p) {
        if (p % 64 == 63 && a.l[p / 64] == 0) { p -= 63; continue; }
        sticky = (int)((a.l[p / 64] >> (p % 64)) & 1u);
    }
    if (rbit && (sticky || (mant & 1u))) mant += 1;
    double r = ldexp((double)mant, lsb - XB_BIAS);  /* exact: mant < 2^54 and fits the format */
    return neg ? -r : r;
}

/* Adds x_i y_i for i in [i0, i1) exactly into a; returns 0 (and stops) at a
 * non-finite operand. */
static int dot_accumulate(bigfix* a, int64_t i0, int64_t i1, const double* x, const double* y)
{
    for (int64_t i = i0; i < i1; ++i) {
        if (!isfinite(x[i]) || !isfinite(y[i])) return 0;
        uint64_t mx, my;
        int ex, ey;
        split(x[i], &mx, &ex);
        split(y[i], &my, &ey);
        if (mx == 0 || my == 0) continue;
        unsigned __int128 p = (unsigned __int128)mx * my;
        int neg = (signbit(x[i]) != 0) != (signbit(y[i]) != 0);
        int pos = ex + ey + XB_BIAS;               /* bit index of the product's bit 0 */
        int limb = pos / 64, sh = pos % 64;
        uint64_t lo = (uint64_t)p, hi = (uint64_t)(p >> 64);
        uint64_t v0 = lo << sh;
        uint64_t v1 = sh ? ((lo >> (64 - sh)) | (hi << sh)) : hi;
        uint64_t v2 = sh ? (hi >> (64 - sh)) : 0;
        big_addsub(a, limb, v0, neg);
        big_addsub(a, limb + 1, v1, neg);
        big_addsub(a, limb + 2, v2, neg);
    }
    return 1;
}

/* a += b exactly (two's complement integers of XB_LIMBS limbs). */
static void big_add(bigfix* a, const bigfix* b)
{
    uint64_t carry = 0;
    for (int k = 0; k < XB_LIMBS; ++k) {
        uint64_t o = a->l[k];
        uint64_t s1 = o + b->l[k];
        uint64_t c1 = s1 < o;
        uint64_t s2 = s1 + carry;
        uint64_t c2 = s2 < s1;
        a->l[k] = s2;
        carry = c1 | c2;
    }
}

double orc_dot(int64_t n, const double* x, const double* y)
{
    bigfix a;
    memset(&a, 0, sizeof(a));
    int finite_ops = 1;
#ifdef _OPENMP
    #pragma omp parallel
    {
        bigfix part;
        memset(&part, 0, sizeof(part));
        const int64_t nt = omp_get_num_threads(), t = omp_get_thread_num();
        const int64_t i0 = n * t / nt, i1 = n * (t + 1) / nt;
        const int ok = dot_accumulate(&part, i0, i1, x, y);
        #pragma omp critical
        {
            big_add(&a, &part);
            if (!ok) finite_ops = 0;
        }
    }
#else
    finite_ops = dot_accumulate(&a, 0, n, x, y);
#endif
    if (!finite_ops) {
        /* a NaN or infinity among the operands: the plain left-to-right sum,
           so that it propagates as IEEE arithmetic does */
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += x[j] * y[j];
        return s;
    }
    return big_round(&a);
}

/*
 * The pieces of orc_dot for a sum split over several owners of the rows (a
 * row-partitioned run): the exact partial sum of x_i y_i over [0, n) as
 * XB_LIMBS 64-bit limbs (two's complement fixed point, bit XB_BIAS = 2^0;
 * returns 0 when an operand is not finite), the exact merge of two partials,
 * and the final rounding to nearest even.
 */
int orc_dot_limbs(void) { return XB_LIMBS; }
int orc_dot_partial(int64_t n, const double* x, const double* y, uint64_t* limbs)
{
    bigfix a;
    memset(&a, 0, sizeof(a));
    const int ok = dot_accumulate(&a, 0, n, x, y);
    memcpy(limbs, a.l, sizeof(a.l));
    return ok;
}
void orc_dot_merge(uint64_t* a, const uint64_t* b)
{
    bigfix x, y;
    memcpy(x.l, a, sizeof(x.l));
    memcpy(y.l, b, sizeof(y.l));
    big_add(&x, &y);
    memcpy(a, x.l, sizeof(x.l));
}
double orc_dot_round(const uint64_t* limbs)
{
    bigfix a;
    memcpy(a.l, limbs, sizeof(a.l));
    return big_round(&a);
}

/* ||b - A x||_2, computed with the routines above. */
double orc_true_residual(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                         const double* b, const double* x)
{
    double* ax = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    ORC_ROWS
    for (int64_t i = 0; i < n; ++i) ax[i] = 0.0;
    orc_spmv(n, rowptr, col, val, x, ax);
    ORC_ROWS
    for (int64_t i = 0; i < n; ++i) ax[i] = b[i] - ax[i];
    double r = sqrt(orc_dot(n, ax, ax));
    free(ax);
    return r;
}

static int finite(double v) { return isfinite(v); }

/* ---- one run of Algorithm 3 / 4 / 5 ----------------------------------- */

/*
 * The two operations of the method that involve every row: y = A x and the
 * inner product (x, y).  A plain run uses the CSR routines above on the whole
 * system; a row-partitioned run (orc_solve_hooked) supplies its own, over its
 * block of rows, with the halo exchange and the sum over all blocks inside.
 */
typedef void (*orc_mv_fn)(void* ctx, const double* x, double* y);
typedef double (*orc_dot_fn)(void* ctx, const double* x, const double* y);

typedef struct {
    int64_t n;
    const int64_t* rowptr; const int32_t* col; const double* val;
    const double* b;
    double* v[SV_COUNT];
    orc_mv_fn mv;
    orc_dot_fn dot;
    void* ctx;
} orc_ws;

#define MV(x, y) w->mv(w->ctx, (x), (y))
#define DOT(x, y) w->dot(w->ctx, (x), (y))

static void mv_whole(void* ctx, const double* x, double* y)
{
    const orc_ws* w = (const orc_ws*)ctx;
    orc_spmv(w->n, w->rowptr, w->col, w->val, x, y);
}
static double dot_whole(void* ctx, const double* x, const double* y)
{
    return orc_dot(((const orc_ws*)ctx)->n, x, y);
}

/* ||b - A x||_2 with the run's operations (the same steps as orc_true_residual). */
static double ws_true_residual(orc_ws* w, const double* x)
{
    const int64_t n = w->n;
    double* ax = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    ORC_ROWS
    for (int64_t i = 0; i < n; ++i) ax[i] = 0.0;
    MV(x, ax);
    ORC_ROWS
    for (int64_t i = 0; i < n; ++i) ax[i] = w->b[i] - ax[i];
    double r = sqrt(DOT(ax, ax));
    free(ax);
    return r;
}

/*
 * One run from the current x.  thresh = absolute threshold of the stop test
 * (eps*||r_0|| of the first run).  Returns the ORC status, the iterations of
 * this run in *its, and appends sqrt(r_i)/r0ref to hist.
 */
static int run_once(orc_ws* w, const orc_opts* o, double thresh, double r0ref, int it_budget,
                    int first_run, double* hist, int hist_cap, int* hist_len,
                    double* scal_hist, int* its, orc_result* res, double* dump_scalars, int* dumped)
{
    const int64_t n = w->n;
    double *x = w->v[SV_X], *r = w->v[SV_R], *rs = w->v[SV_RS], *s = w->v[SV_S], *y = w->v[SV_Y];
    double *t = w->v[SV_T], *p = w->v[SV_P], *u = w->v[SV_U], *z = w->v[SV_Z], *wv = w->v[SV_W];
    double *ov = w->v[SV_O], *q = w->v[SV_Q], *l = w->v[SV_L], *g = w->v[SV_G];
    double *As = w->v[SV_AS], *Aw = w->v[SV_AW];
    const int pipelined = (o->kind != ORC_SSBICGSAFE2);
    const int rr = (o->kind == ORC_P_BICGSAFE_RR);

    /* Alg. 3/4/5 set-up: r_0 = b - A x_0, r0* = r_0 (R8). */
    MV(x, As);                                                /* A x_0 (As used as scratch) */
    ORC_ROWS
    for (int64_t j = 0; j < n; ++j) r[j] = w->b[j] - As[j];
    ORC_ROWS
    for (int64_t j = 0; j < n; ++j) rs[j] = r[j];
    /* R2: zero auxiliaries. */
    for (int k = SV_Y; k < SV_COUNT; ++k)
        if (k != SV_S) memset(w->v[k], 0, sizeof(double) * (size_t)n);
    memset(s, 0, sizeof(double) * (size_t)n);
    /* R1: s_0 = A r_0 for the pipelined variants. */
    if (pipelined) MV(r, s);

    double alpha_prev = 0.0, zeta_prev = 0.0, f_prev = 0.0;
    for (int i = 0;; ++i) {
        double alpha, beta, zeta, eta;
        double da, db = 0, dc = 0, dd, de = 0, df, dg, dh = 0, drr;
        /* Alg. 3: s_i = A r_i.   Alg. 4/5: As_i = A s_i. */
        if (pipelined) MV(s, As);
        else           MV(r, s);
        /* Inner products (R5). */
        da = DOT(s, s);
        dd = DOT(s, r);
        df = DOT(rs, r);
        dg = DOT(rs, s);
        drr = DOT(r, r);
        if (i == 0) {
            /* R3: the i = 0 branch. */
            beta = 0.0;
            alpha = df / dg;
            zeta = dd / da;
            eta = 0.0;
            if (dg == 0.0 || da == 0.0) {
                if (!(sqrt(drr) <= thresh)) return ORC_ERR_BREAKDOWN;
            }
        } else {
            db = DOT(y, y);
            dc = DOT(s, y);
            de = DOT(y, r);
            dh = DOT(rs, t);
            beta = (alpha_prev * df) / (zeta_prev * f_prev);
            alpha = df / (dg + beta * dh);
            double den = da * db - dc * dc;
            if (den == 0.0 || !finite(den)) {
                /* R4: fall back to the minimal-residual step of the i = 0 branch. */
                zeta = dd / da;
                eta = 0.0;
                res->fallbacks++;
            } else {
                zeta = (db * dd - dc * de) / den;
                eta = (da * de - dc * dd) / den;
            }
            if (zeta_prev * f_prev == 0.0 || dg + beta * dh == 0.0 || da == 0.0) {
                if (!(sqrt(drr) <= thresh)) return ORC_ERR_BREAKDOWN;
            }
        }
        if (hist && *hist_len < hist_cap) hist[(*hist_len)++] = sqrt(drr) / r0ref;
        if (scal_hist && first_run && i < hist_cap) {
            scal_hist[4 * i + 0] = alpha; scal_hist[4 * i + 1] = beta;
            scal_hist[4 * i + 2] = zeta;  scal_hist[4 * i + 3] = eta;
        }
        res->rel_res_recursive = sqrt(drr) / r0ref;
        const int rr_step = rr && i > 0 && (i % o->rr_m) == 0 && i < o->rr_M;
        if (dump_scalars && first_run && i == o->dump_iter) {
            double* S = dump_scalars;
            S[SC_ALPHA] = alpha; S[SC_BETA] = beta; S[SC_ZETA] = zeta; S[SC_ETA] = eta;
            S[SC_A] = da; S[SC_B] = db; S[SC_C] = dc; S[SC_D] = dd; S[SC_E] = de;
            S[SC_F] = df; S[SC_G] = dg; S[SC_H] = dh; S[SC_R] = drr; S[SC_RR] = rr_step; S[SC_I] = i;
            if (o->dump_phase == 0) { *its = i; *dumped = 1; return ORC_OK; }
        }
        /* R6: stop test on the recursive residual. */
        if (sqrt(drr) <= thresh) { *its = i; return ORC_OK; }
        if (!finite(alpha) || !finite(beta) || !finite(zeta) || !finite(eta) || !finite(drr)) {
            *its = i; return ORC_ERR_NONFINITE;
        }
        if (i >= it_budget) { *its = i; return ORC_NOT_CONVERGED; }

        /* p_i = r_i + beta_i (p_{i-1} - u_{i-1}) */
        ORC_ROWS
        for (int64_t j = 0; j < n; ++j) p[j] = fma(beta, p[j] - u[j], r[j]);
        /* o_i = s_i + beta_i t_{i-1} */
        ORC_ROWS
        for (int64_t j = 0; j < n; ++j) ov[j] = fma(beta, t[j], s[j]);
        /* u_i = zeta_i o_i + eta_i (y_i + beta_i u_{i-1}) */
        ORC_ROWS
        for (int64_t j = 0; j < n; ++j) u[j] = fma(zeta, ov[j], eta * fma(beta, u[j], y[j]));
        if (!pipelined) {
            /* Alg. 3: w_i = A u_i */
            MV(u, wv);
        } else if (rr_step) {
            /* Alg. 5: q_i = A o_i, w_i = A u_i */
            MV(ov, q);
            MV(u, wv);
        } else {
            /* q_i = As_i + beta_i l_{i-1}   (Eq. q) */
            ORC_ROWS
            for (int64_t j = 0; j < n; ++j) q[j] = fma(beta, l[j], As[j]);
            /* w_i = zeta_i q_i + eta_i (g_i + beta_i w_{i-1})   (Eq. w) */
            ORC_ROWS
            for (int64_t j = 0; j < n; ++j) wv[j] = fma(zeta, q[j], eta * fma(beta, wv[j], g[j]));
        }
        /* t_i = o_i - w_i */
        ORC_ROWS
        for (int64_t j = 0; j < n; ++j) t[j] = ov[j] - wv[j];
        /* z_i = zeta_i r_i + eta_i z_{i-1} - alpha_i u_i */
        ORC_ROWS
        for (int64_t j = 0; j < n; ++j) z[j] = fma(-alpha, u[j], fma(zeta, r[j], eta * z[j]));
        /* y_{i+1} = zeta_i s_i + eta_i y_i - alpha_i w_i */
        ORC_ROWS
        for (int64_t j = 0; j < n; ++j) y[j] = fma(-alpha, wv[j], fma(zeta, s[j], eta * y[j]));
        /* x_{i+1} = x_i + alpha_i p_i + z_i */
        ORC_ROWS
        for (int64_t j = 0; j < n; ++j) x[j] = fma(alpha, p[j], x[j]) + z[j];
        if (rr_step) {
            /* Alg. 5 replacement: r = b - A x, l_i = A t_i (R9), g = A y, s = A r */
            MV(x, Aw);
            ORC_ROWS
            for (int64_t j = 0; j < n; ++j) r[j] = w->b[j] - Aw[j];
            MV(t, l);
            MV(y, g);
            MV(r, s);
            res->rr_steps++;
        } else {
            /* r_{i+1} = r_i - alpha_i o_i - y_{i+1} */
            ORC_ROWS
            for (int64_t j = 0; j < n; ++j) r[j] = fma(-alpha, ov[j], r[j]) - y[j];
            if (pipelined) {
                /* Aw_i; l_i = q_i - Aw_i (Eq. l); g_{i+1} = zeta As_i + eta g_i - alpha Aw_i (Eq. g);
                   s_{i+1} = s_i - alpha q_i - g_{i+1} (Eq. sip1) */
                MV(wv, Aw);
                ORC_ROWS
                for (int64_t j = 0; j < n; ++j) l[j] = q[j] - Aw[j];
                ORC_ROWS
                for (int64_t j = 0; j < n; ++j) g[j] = fma(-alpha, Aw[j], fma(zeta, As[j], eta * g[j]));
                ORC_ROWS
                for (int64_t j = 0; j < n; ++j) s[j] = fma(-alpha, q[j], s[j]) - g[j];
            }
        }
        if (dump_scalars && first_run && i == o->dump_iter && o->dump_phase == 1) {
            *its = i + 1; *dumped = 1; return ORC_OK;
        }
        alpha_prev = alpha; zeta_prev = zeta; f_prev = df;
    }
}

/*
 * Solve A x = b.  x holds x_0 on entry and the result on exit.
 * hist (optional, hist_cap entries) receives sqrt(r_i)/||r_0|| for every
 * evaluated stop test (all runs); scal_hist (optional, 4*hist_cap) receives
 * alpha, beta, zeta, eta of the first run's iterations.  When dump_iter >= 0,
 * the first run stops there and state (SV_COUNT*n doubles, slot-major) and
 * scalars (SC_COUNT doubles) receive the dump.
 */
static int solve_runs(orc_ws* w, double* x, const orc_opts* o, double* hist, int hist_cap, int* hist_len,
                      double* scal_hist, double* state, double* scalars, orc_result* res)
{
    const int64_t n = w->n;
    memset(res, 0, sizeof(*res));
    if (hist_len) *hist_len = 0;
    int hl = 0;
    if (n < 0 || !o || o->kind < 0 || o->kind > 2 || o->maxit < 0 || (o->kind == 2 && o->rr_m <= 0)) {
        res->status = ORC_ERR_ARG;
        return ORC_ERR_ARG;
    }
    for (int k = 0; k < SV_COUNT; ++k) {
        if (k == SV_X) { w->v[k] = x; continue; }
        w->v[k] = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    }
    double r0 = ws_true_residual(w, x);
    res->r0_norm = r0;
    const double thresh = o->tol * r0;
    const double r0ref = (r0 > 0.0) ? r0 : 1.0;
    int status = ORC_OK, total = 0, dumped = 0;
    for (int run = 0;; ++run) {
        int its = 0;
        status = run_once(w, o, thresh, r0ref, o->maxit - total, run == 0, hist, hist_cap, &hl,
                          scal_hist, &its, res, (o->dump_iter >= 0) ? scalars : NULL, &dumped);
        total += its;
        if (dumped) {
            if (state) for (int k = 0; k < SV_COUNT; ++k) memcpy(state + (size_t)k * n, w->v[k], sizeof(double) * (size_t)n);
            break;
        }
        if (status != ORC_OK) break;
        double tr = ws_true_residual(w, x);
        res->rel_res_true = tr / r0ref;
        if (tr <= thresh || run >= o->max_restarts) {
            if (tr > thresh) status = ORC_NOT_CONVERGED;
            break;
        }
        if (total >= o->maxit) { status = ORC_NOT_CONVERGED; break; }
        res->restarts++;
    }
    if (!dumped) res->rel_res_true = ws_true_residual(w, x) / r0ref;
    res->iterations = total;
    res->status = status;
    if (hist_len) *hist_len = hl;
    for (int k = 0; k < SV_COUNT; ++k) if (k != SV_X) free(w->v[k]);
    return status;
}

int orc_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
              const double* b, double* x, const orc_opts* o,
              double* hist, int hist_cap, int* hist_len, double* scal_hist,
              double* state, double* scalars, orc_result* res)
{
    orc_ws w;
    memset(&w, 0, sizeof(w));
    w.n = n; w.rowptr = rowptr; w.col = col; w.val = val; w.b = b;
    w.mv = mv_whole; w.dot = dot_whole; w.ctx = &w;
    return solve_runs(&w, x, o, hist, hist_cap, hist_len, scal_hist, state, scalars, res);
}

/*
 * The same runs over one block of rows of a row-partitioned system (the
 * setting of Section 3: every process owns some rows of A and the same rows
 * of every vector).  n_local, b and x are the block's; mv(ctx, x, y) must set
 * y = (A x) on the block's rows and dot(ctx, x, y) must return the inner
 * product over all rows, both given the block's parts of x and y.  With
 * exact inner products and every row summed in CSR order the iterates are
 * those of orc_solve, bit for bit.
 */
int orc_solve_hooked(int64_t n_local, const double* b, double* x, const orc_opts* o, orc_mv_fn mv, orc_dot_fn dot,
                     void* ctx, double* hist, int hist_cap, int* hist_len, double* scal_hist, orc_result* res)
{
    orc_ws w;
    memset(&w, 0, sizeof(w));
    w.n = n_local; w.b = b;
    w.mv = mv; w.dot = dot; w.ctx = ctx;
    return solve_runs(&w, x, o, hist, hist_cap, hist_len, scal_hist, NULL, NULL, res);
}

/* ---- formats ----------------------------------------------------------- */

/*
 * SELL-C-sigma (Kreutzer et al.) from CSR.  Rows are sorted by length,
 * descending, inside windows of sigma consecutive rows (stable: ties keep the
 * original order); perm[p] = original row at permuted position p.  Slices of
 * C permuted rows are stored column-major and padded to the slice's longest
 * row with value 0 and column index p (the padded row's own position).
 * Column indices are renumbered into the permuted space (col' = perm^-1[col]);
 * a row's entries keep their CSR order.
 * slice_ptr has nslices+1 entries (element offsets); returns the padded size.
 * Pass NULL for scol/sval to only compute perm, slice_ptr and the size.
 */
int64_t orc_sell_build(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                       int C, int sigma, int32_t* perm, int64_t* slice_ptr, int32_t* scol, double* sval)
{
    int32_t* inv = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t w0 = 0; w0 < n; w0 += sigma) {
        int64_t w1 = w0 + sigma < n ? w0 + sigma : n;
        /* stable insertion sort by length descending */
        for (int64_t i = w0; i < w1; ++i) {
            int32_t row = (int32_t)i;
            int64_t len = rowptr[i + 1] - rowptr[i];
            int64_t k = i;
            while (k > w0 && (rowptr[perm[k - 1] + 1] - rowptr[perm[k - 1]]) < len) { perm[k] = perm[k - 1]; --k; }
            perm[k] = row;
        }
    }
    for (int64_t p = 0; p < n; ++p) inv[perm[p]] = (int32_t)p;
    int64_t nslices = (n + C - 1) / C;
    slice_ptr[0] = 0;
    for (int64_t sl = 0; sl < nslices; ++sl) {
        int64_t width = 0;
        for (int64_t lane = 0; lane < C; ++lane) {
            int64_t p = sl * C + lane;
            if (p < n) {
                int64_t len = rowptr[perm[p] + 1] - rowptr[perm[p]];
                if (len > width) width = len;
            }
        }
        slice_ptr[sl + 1] = slice_ptr[sl] + width * C;
    }
    if (scol && sval) {
        for (int64_t sl = 0; sl < nslices; ++sl) {
            int64_t width = (slice_ptr[sl + 1] - slice_ptr[sl]) / C;
            for (int64_t lane = 0; lane < C; ++lane) {
                int64_t p = sl * C + lane;
                for (int64_t k = 0; k < width; ++k) {
                    int64_t dst = slice_ptr[sl] + k * C + lane;
                    if (p < n && k < rowptr[perm[p] + 1] - rowptr[perm[p]]) {
                        int64_t src = rowptr[perm[p]] + k;
                        scol[dst] = inv[col[src]];
                        sval[dst] = val[src];
                    } else {
                        scol[dst] = (int32_t)(p < n ? p : n - 1);
                        sval[dst] = 0.0;
                    }
                }
            }
        }
    }
    free(inv);
    return slice_ptr[nslices];
}

/* Round-to-nearest-even FP64 -> BF16 (bit pattern), via FP32 as an exact
 * two-step only when the FP32 rounding is exact; done directly on the FP64
 * bits here so that no double rounding occurs. NaN maps to a quiet NaN. */
void orc_to_bf16(int64_t n, const double* in, uint16_t* out)
{
    for (int64_t i = 0; i < n; ++i) {
        double v = in[i];
        uint64_t bits; memcpy(&bits, &v, 8);
        uint16_t sign = (uint16_t)((bits >> 48) & 0x8000u);
        if (isnan(v)) { out[i] = (uint16_t)(sign | 0x7FC0u); continue; }
        double a = fabs(v);
        if (a == 0.0) { out[i] = sign; continue; }
        /* Find the bf16 neighbours by exponent: bf16 has 8 significant bits. */
        int e; frexp(a, &e);                /* a = m * 2^e, m in [0.5,1) */
        int emin = -125;                    /* smallest normal bf16 exponent (as frexp's e) */
        int q = (e < emin ? emin : e) - 8;  /* quantum exponent: ulp = 2^q */
        double ulp = ldexp(1.0, q);
        double k = floor(a / ulp);          /* exact: a/ulp is exact scaling by a power of two */
        double rem = a - k * ulp;
        double half = ulp * 0.5;
        if (rem > half || (rem == half && fmod(k, 2.0) != 0.0)) k += 1.0;
        double rounded = k * ulp;
        float f = (float)rounded;           /* exact: rounded has <= 8 significant bits */
        uint32_t fb; memcpy(&fb, &f, 4);
        if (rounded >= ldexp(1.0, 128)) fb = 0x7F800000u; /* overflow to infinity */
        out[i] = (uint16_t)(sign | (uint16_t)((fb >> 16) & 0x7FFFu));
    }
}

/* ---- block-Jacobi preconditioning (build addition: the paper, Section 5,
 *      uses no preconditioner) ------------------------------------------- */

/*
 * Right preconditioning with M = the block diagonal of A in blocks of bs
 * consecutive rows (the last block holds the remaining rows).  The runs
 * solve (A M^-1) y = b from y_0 = M x_0 and return x = M^-1 y; the residual
 * b - (A M^-1) y of the solved system is b - A x, so the tolerance keeps
 * its meaning.
 *
 * Storage: for row i of the block that starts at row b0 and holds m rows, the
 * row's m entries of the block D = A[b0..b0+m, b0..b0+m] and of its inverse
 * E = D^-1 are at i*bs + j, j = 0..m-1 (zero for j >= m).
 *
 * E is computed by Gauss-Jordan elimination on [D | I]: for each pivot column
 * p in order, the pivot is the first row r >= p with the largest |a[r][p]|;
 * that row is swapped into place, divided by the pivot (every entry, the
 * pivot itself included, by the saved pivot value), and for every other row
 * r the multiple f = a[r][p] of it is subtracted as a[r][c] - f * a[p][c]
 * (product and difference rounded separately).  A zero, NaN or infinite
 * pivot makes the block singular: ORC_ERR_ARG.  A repeated (row, column)
 * entry of A keeps its last value in D.
 */
int orc_bjacobi_blocks(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, int bs,
                       double* D, double* E)
{
    if (n < 0 || bs < 1 || bs > 32) return ORC_ERR_ARG;
    double a[32 * 32], inv[32 * 32];
    for (int64_t b0 = 0; b0 < n; b0 += bs) {
        const int m = (int)((n - b0) < bs ? (n - b0) : bs);
        for (int k = 0; k < m * m; ++k) { a[k] = 0.0; inv[k] = 0.0; }
        for (int r = 0; r < m; ++r) {
            for (int64_t k = rowptr[b0 + r]; k < rowptr[b0 + r + 1]; ++k) {
                const int64_t c = (int64_t)col[k] - b0;
                if (c >= 0 && c < m) a[r * m + c] = val[k];
            }
            inv[r * m + r] = 1.0;
        }
        for (int r = 0; r < m; ++r)
            for (int j = 0; j < bs; ++j) D[(b0 + r) * bs + j] = j < m ? a[r * m + j] : 0.0;
        for (int p = 0; p < m; ++p) {
            int piv = p;
            double big = fabs(a[p * m + p]);
            for (int r = p + 1; r < m; ++r)
                if (fabs(a[r * m + p]) > big) { big = fabs(a[r * m + p]); piv = r; }
            if (!(big > 0.0) || !finite(big)) return ORC_ERR_ARG;
            if (piv != p) {
                for (int c = 0; c < m; ++c) {
                    double t = a[p * m + c]; a[p * m + c] = a[piv * m + c]; a[piv * m + c] = t;
                    t = inv[p * m + c]; inv[p * m + c] = inv[piv * m + c]; inv[piv * m + c] = t;
                }
            }
            const double d = a[p * m + p];
            for (int c = 0; c < m; ++c) {
                a[p * m + c] = a[p * m + c] / d;
                inv[p * m + c] = inv[p * m + c] / d;
            }
            for (int r = 0; r < m; ++r) {
                if (r == p) continue;
                const double f = a[r * m + p];
                for (int c = 0; c < m; ++c) {
                    a[r * m + c] = a[r * m + c] - f * a[p * m + c];
                    inv[r * m + c] = inv[r * m + c] - f * inv[p * m + c];
                }
            }
        }
        for (int r = 0; r < m; ++r)
            for (int j = 0; j < bs; ++j) E[(b0 + r) * bs + j] = j < m ? inv[r * m + j] : 0.0;
    }
    return ORC_OK;
}

/* z = M v block by block (M = D or E as stored by orc_bjacobi_blocks):
 * z_i = sum over the block's columns j of M[i][j] v[b0 + j], accumulated with
 * fma in column order starting from zero.  z must not overlap v. */
void orc_bjacobi_apply(int64_t n, int bs, const double* M, const double* v, double* z)
{
    ORC_ROWS
    for (int64_t i = 0; i < n; ++i) {
        const int64_t b0 = i - i % bs;
        const int m = (int)((n - b0) < bs ? (n - b0) : bs);
        double acc = 0.0;
        for (int j = 0; j < m; ++j) acc = fma(M[i * bs + j], v[b0 + j], acc);
        z[i] = acc;
    }
}

typedef struct {
    int64_t n;
    const int64_t* rowptr; const int32_t* col; const double* val;
    int bs;
    const double* E;
    double* z;
} orc_bj_ctx;

/* y = (A M^-1) x: z = E x block by block, then y = A z */
static void mv_bjacobi(void* ctx, const double* x, double* y)
{
    orc_bj_ctx* c = (orc_bj_ctx*)ctx;
    orc_bjacobi_apply(c->n, c->bs, c->E, x, c->z);
    orc_spmv(c->n, c->rowptr, c->col, c->val, c->z, y);
}
static double dot_bjacobi(void* ctx, const double* x, const double* y)
{
    return orc_dot(((const orc_bj_ctx*)ctx)->n, x, y);
}

int orc_solve_bjacobi(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, int bs,
                      const double* b, double* x, const orc_opts* o,
                      double* hist, int hist_cap, int* hist_len, double* scal_hist, orc_result* res)
{
    memset(res, 0, sizeof(*res));
    if (hist_len) *hist_len = 0;
    if (n < 0 || bs < 1 || bs > 32) { res->status = ORC_ERR_ARG; return ORC_ERR_ARG; }
    const size_t nn = (size_t)(n > 0 ? n : 1);
    double* D = (double*)calloc(nn * (size_t)bs, sizeof(double));
    double* E = (double*)calloc(nn * (size_t)bs, sizeof(double));
    double* y = (double*)calloc(nn, sizeof(double));
    double* z = (double*)calloc(nn, sizeof(double));
    int st = orc_bjacobi_blocks(n, rowptr, col, val, bs, D, E);
    if (st != ORC_OK) {
        res->status = st;
    } else {
        orc_bjacobi_apply(n, bs, D, x, y);            /* y_0 = M x_0 */
        orc_bj_ctx c = {n, rowptr, col, val, bs, E, z};
        orc_ws w;
        memset(&w, 0, sizeof(w));
        w.n = n; w.b = b;
        w.mv = mv_bjacobi; w.dot = dot_bjacobi; w.ctx = &c;
        st = solve_runs(&w, y, o, hist, hist_cap, hist_len, scal_hist, NULL, NULL, res);
        orc_bjacobi_apply(n, bs, E, y, x);            /* x = M^-1 y */
    }
    free(D); free(E); free(y); free(z);
    return st;
}
