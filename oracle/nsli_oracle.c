/*
 * nsli_oracle.c -- plain, slow, double-precision CPU restatement of the
 * pseudo-projection method (AP and ModAP) of Sokolinsky & Sokolinskaya,
 * "Scalable Parallel Algorithm for Solving Non-stationary Systems of Linear
 * Inequalities" (Lobachevskii J. Math., 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header, table or constant
 * with the CUDA path and includes nothing from it.
 *
 * Every loop is sequential and in the order the paper states the operation:
 * rows i = 0..m-1 ascending, columns j = 0..n-1 ascending, all arithmetic in
 * IEEE double (compile with -ffp-contract=off so no multiply-add is fused).
 *
 * Notation (Section 2):
 *   r_i      = <a_i, x> - b_i                      residual of inequality i
 *   rho+_i   = max(r_i, 0) / ||a_i||^2 * a_i       positive slice, Eq. 7
 *   y        = sum_i rho+_i                        Reduce(+, B), Section 3
 *   h        = number of non-zero slices           Eq. 8
 *   phi      = y / h                               Eq. 8 (Algorithm 1 step)
 *   psi      = lambda * y / ||y||                  Eq. 12 (ModAP step)
 *   eps-membership: for all i, r_i <= 0 or |r_i| / ||a_i|| < eps   Eq. 10
 *
 * Readings of the paper taken here (the paper is silent or its listings are
 * lost):
 *   - the relaxed Algorithm 1 step is x <- x - lambda * y / h (lambda = 1 is
 *     Eq. 8 exactly); the ModAP step is x <- x - lambda * y / ||y||;
 *   - a row with r_i == 0 is satisfied (h counts non-zero slices, Eq. 8);
 *   - the stopping test of an iteration is evaluated at the top of the
 *     iteration, on the Map at (x_k, b(k)); the iteration count is the number
 *     of x-updates performed;
 *   - the non-stationary data is the translated right-hand side
 *     b(k) = b0 + k * rho * (A v), one tick per iteration (Section 5 moves the
 *     polytope along a straight line before every iteration).
 *
 * Parity pins live in the tests (closed forms, brute force on 2-D/3-D
 * systems, Fejer monotonicity, the fixed point, library quantizers).
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

/* step rules */
#define ORACLE_RULE_RELAXED 0 /* x <- x - lambda * y / h        (Eq. 8)  */
#define ORACLE_RULE_MODAP   1 /* x <- x - lambda * y / ||y||    (Eq. 12) */

/* stopping rules */
#define ORACLE_STOP_NONE        0 /* run to max_iter; h == 0 gives a zero step */
#define ORACLE_STOP_STEP        1 /* ||x_{k+1} - x_k|| < eps                  */
#define ORACLE_STOP_EPSMEM      2 /* Eq. 10: max_i r_i / ||a_i|| < eps        */
#define ORACLE_STOP_MAXVIOL_REL 3 /* max_i r_i <= eps * max_i |b_i|           */

/* what one iteration did */
#define ORACLE_IT_STEPPED   0 /* an x-update was performed, no stop         */
#define ORACLE_IT_CONVERGED 1 /* stop test passed at the top; x unchanged   */
#define ORACLE_IT_STEP_STOP 2 /* x-update performed, then ||dx|| < eps      */

/* solve status */
#define ORACLE_OK            0
#define ORACLE_NOT_CONVERGED 1

/* ||a_i||^2 for every row (Section 2, reflection vector denominator).
 * Returns the number of zero rows (the paper assumes a_i != 0). */
int64_t oracle_norms2(int64_t m, int64_t n, const double *A, double *n2)
{
    int64_t zero_rows = 0;
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double a = A[i * n + j];
            s = s + a * a;
        }
        n2[i] = s;
        if (s == 0.0)
            zero_rows = zero_rows + 1;
    }
    return zero_rows;
}

/* b_i(k) = b0_i + k * rho * Av_i: translation of the polytope by k*rho*v
 * (Section 5; one tick per iteration). */
void oracle_tick_b(int64_t m, const double *b0, const double *Av, double rho,
                   int64_t k, double *b)
{
    double t = (double)k * rho;
    for (int64_t i = 0; i < m; ++i) {
        double shift = 0.0;
        if (Av != NULL)
            shift = t * Av[i];
        b[i] = b0[i] + shift;
    }
}

/* Map (Eq. 13, each element gives rho+_i of Eq. 7) followed by
 * Reduce(+, B) (Section 3).  Outputs
 *   y[n]      sum of the positive slices,
 *   *h        number of rows with r_i > 0,
 *   *maxviol  max_i r_i,
 *   *maxnorm  max_i r_i / ||a_i||,
 *   *maxb     max_i |b_i|,
 *   r[m]      the residuals (optional, may be NULL). */
void oracle_map_reduce(int64_t m, int64_t n, const double *A, const double *b,
                       const double *n2, const double *x, double *y,
                       int64_t *h, double *maxviol, double *maxnorm,
                       double *maxb, double *r)
{
    for (int64_t j = 0; j < n; ++j)
        y[j] = 0.0;
    int64_t count = 0;
    double mv = -INFINITY, mn = -INFINITY, mb = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        const double *a = A + i * n;
        double dot = 0.0;
        for (int64_t j = 0; j < n; ++j)
            dot = dot + a[j] * x[j];
        double ri = dot - b[i];
        if (r != NULL)
            r[i] = ri;
        if (ri > mv)
            mv = ri;
        double rn = ri / sqrt(n2[i]);
        if (rn > mn)
            mn = rn;
        if (fabs(b[i]) > mb)
            mb = fabs(b[i]);
        if (ri > 0.0) {
            /* positive slice of the reflection vector, Eq. 7 */
            double c = ri / n2[i];
            for (int64_t j = 0; j < n; ++j)
                y[j] = y[j] + c * a[j];
            count = count + 1;
        }
    }
    *h = count;
    *maxviol = mv;
    *maxnorm = mn;
    *maxb = mb;
}

/* The same Map and Reduce for a matrix held as binary32 values: each entry is
 * widened to double before use, so the arithmetic is that of
 * oracle_map_reduce on the exact values (used for large systems, where a
 * double copy of A would not fit beside the binary32 one). */
void oracle_map_reduce_f32(int64_t m, int64_t n, const float *A,
                           const double *b, const double *n2, const double *x,
                           double *y, int64_t *h, double *maxviol,
                           double *maxnorm, double *maxb, double *r)
{
    for (int64_t j = 0; j < n; ++j)
        y[j] = 0.0;
    int64_t count = 0;
    double mv = -INFINITY, mn = -INFINITY, mb = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        const float *a = A + i * n;
        double dot = 0.0;
        for (int64_t j = 0; j < n; ++j)
            dot = dot + (double)a[j] * x[j];
        double ri = dot - b[i];
        if (r != NULL)
            r[i] = ri;
        if (ri > mv)
            mv = ri;
        double rn = ri / sqrt(n2[i]);
        if (rn > mn)
            mn = rn;
        if (fabs(b[i]) > mb)
            mb = fabs(b[i]);
        if (ri > 0.0) {
            double c = ri / n2[i];
            for (int64_t j = 0; j < n; ++j)
                y[j] = y[j] + c * (double)a[j];
            count = count + 1;
        }
    }
    *h = count;
    *maxviol = mv;
    *maxnorm = mn;
    *maxb = mb;
}

/* ||a_i||^2 of binary32 rows, accumulated in double. */
int64_t oracle_norms2_f32(int64_t m, int64_t n, const float *A, double *n2)
{
    int64_t zero_rows = 0;
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double a = (double)A[i * n + j];
            s = s + a * a;
        }
        n2[i] = s;
        if (s == 0.0)
            zero_rows = zero_rows + 1;
    }
    return zero_rows;
}

/* The same Map and Reduce for A in compressed-row form: row i holds the
 * entries val[e] at columns ci[e], e = rp[i] .. rp[i+1]-1, columns
 * ascending.  Each sum runs over the stored entries of a row in column
 * order, which is the order of oracle_map_reduce with the zero entries left
 * out (adding a zero product changes no sum). */
void oracle_map_reduce_csr(int64_t m, int64_t n, const int64_t *rp,
                           const int32_t *ci, const double *val,
                           const double *b, const double *n2, const double *x,
                           double *y, int64_t *h, double *maxviol,
                           double *maxnorm, double *maxb, double *r)
{
    for (int64_t j = 0; j < n; ++j)
        y[j] = 0.0;
    int64_t count = 0;
    double mv = -INFINITY, mn = -INFINITY, mb = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double dot = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            dot = dot + val[e] * x[ci[e]];
        double ri = dot - b[i];
        if (r != NULL)
            r[i] = ri;
        if (ri > mv)
            mv = ri;
        double rn = ri / sqrt(n2[i]);
        if (rn > mn)
            mn = rn;
        if (fabs(b[i]) > mb)
            mb = fabs(b[i]);
        if (ri > 0.0) {
            double c = ri / n2[i];
            for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
                y[ci[e]] = y[ci[e]] + c * val[e];
            count = count + 1;
        }
    }
    *h = count;
    *maxviol = mv;
    *maxnorm = mn;
    *maxb = mb;
}

/* ||a_i||^2 of compressed rows; returns the number of zero rows. */
int64_t oracle_norms2_csr(int64_t m, const int64_t *rp, const double *val,
                          double *n2)
{
    int64_t zero_rows = 0;
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            s = s + val[e] * val[e];
        n2[i] = s;
        if (s == 0.0)
            zero_rows = zero_rows + 1;
    }
    return zero_rows;
}

static int stop_test_passes(int stop, double eps, double maxviol,
                            double maxnorm, double maxb)
{
    if (stop == ORACLE_STOP_EPSMEM)
        return maxnorm < eps; /* Eq. 10 over all rows */
    if (stop == ORACLE_STOP_MAXVIOL_REL)
        return maxviol <= eps * maxb;
    return 0;
}

/* The decision and the step of one iteration, given the Reduce's outputs at
 * (x_k, b(k)): the top-of-iteration test (Eq. 10 or max r_i <= eps max|b|,
 * h == 0 meaning x in M), then the relaxed step x <- x - lambda y / h
 * (Eq. 8) or the fixed-length step x <- x - lambda y / ||y|| (Eq. 12).
 * x[n] is updated in place when a step is taken; stats as for
 * oracle_iteration (stats[0..3] already hold h and the maxima). */
static int decide_and_step(int64_t n, double *x, const double *y, int64_t h,
                           double maxviol, double maxnorm, double maxb,
                           double lambda, int rule, int stop, double eps,
                           int force_step, double *stats)
{
    stats[4] = 0.0;
    stats[5] = 0.0;

    double ynorm2 = 0.0;
    for (int64_t j = 0; j < n; ++j)
        ynorm2 = ynorm2 + y[j] * y[j];
    double ynorm = sqrt(ynorm2);
    stats[5] = ynorm;

    if (!force_step) {
        if (stop != ORACLE_STOP_NONE && h == 0)
            return ORACLE_IT_CONVERGED; /* x lies in M(t): phi = 0 */
        if (stop_test_passes(stop, eps, maxviol, maxnorm, maxb))
            return ORACLE_IT_CONVERGED;
    }

    /* step: relaxed Eq. 8 or fixed-length Eq. 12 */
    double dx2 = 0.0;
    if (h > 0) {
        double s;
        if (rule == ORACLE_RULE_MODAP)
            s = (ynorm > 0.0) ? lambda / ynorm : 0.0;
        else
            s = lambda / (double)h;
        for (int64_t j = 0; j < n; ++j) {
            double d = s * y[j];
            x[j] = x[j] - d;
            dx2 = dx2 + d * d;
        }
    }
    stats[4] = sqrt(dx2);
    if (stop == ORACLE_STOP_STEP && stats[4] < eps)
        return ORACLE_IT_STEP_STOP;
    return ORACLE_IT_STEPPED;
}

/* One iteration of Algorithm 1 / ModAP at tick k (the order of the ModAP-on-
 * lists description in Section 3: Map, Reduce, step, data update, test; the
 * test of step k+1 is evaluated here at the top of iteration k+1).
 *
 * x[n] is updated in place when a step is taken; work[n] receives y.
 * stats[0..5] = h, maxviol, maxnorm, maxb, ||dx||, ||y||.
 * force_step != 0 skips the top-of-iteration test (used after a rejected
 * candidate).  Returns one of ORACLE_IT_*. */
int oracle_iteration(int64_t m, int64_t n, const double *A, const double *b0,
                     const double *Av, double rho, int64_t k,
                     const double *n2, double *x, double lambda, int rule,
                     int stop, double eps, int force_step, double *work,
                     double *b_scratch, double *r_out, double *stats)
{
    int64_t h;
    double maxviol, maxnorm, maxb;
    oracle_tick_b(m, b0, Av, rho, k, b_scratch);
    oracle_map_reduce(m, n, A, b_scratch, n2, x, work, &h, &maxviol, &maxnorm,
                      &maxb, r_out);
    stats[0] = (double)h;
    stats[1] = maxviol;
    stats[2] = maxnorm;
    stats[3] = maxb;
    return decide_and_step(n, x, work, h, maxviol, maxnorm, maxb, lambda, rule,
                           stop, eps, force_step, stats);
}

/* The exchange of ModAPL (Section 3, the list form split into sublists, one
 * per worker): worker w = 0..R-1 has run the Map and a local Reduce over its
 * own contiguous block of rows at (x_k, b(k)) and produced (y_w, h_w, and its
 * maxima).  The global Reduce adds the y_w in worker order w = 0, 1, ...,
 * R-1 (sequentially, element by element), adds the h_w and takes the maxima;
 * then the decision and the step are those of oracle_iteration.  ys holds
 * the R vectors y_w row-major (R x n); hs, maxviols, maxnorms, maxbs hold R
 * values each.  x[n] is updated in place; y_out[n] receives the global y;
 * stats as for oracle_iteration.  Returns one of ORACLE_IT_*. */
int oracle_combine_step(int64_t R, int64_t n, const double *ys,
                        const int64_t *hs, const double *maxviols,
                        const double *maxnorms, const double *maxbs,
                        double *x, double lambda, int rule, int stop,
                        double eps, int force_step, double *y_out,
                        double *stats)
{
    int64_t h = 0;
    double mv = -INFINITY, mn = -INFINITY, mb = 0.0;
    for (int64_t j = 0; j < n; ++j)
        y_out[j] = 0.0;
    for (int64_t w = 0; w < R; ++w) {
        const double *yw = ys + w * n;
        for (int64_t j = 0; j < n; ++j)
            y_out[j] = y_out[j] + yw[j];
        h = h + hs[w];
        if (maxviols[w] > mv)
            mv = maxviols[w];
        if (maxnorms[w] > mn)
            mn = maxnorms[w];
        if (maxbs[w] > mb)
            mb = maxbs[w];
    }
    stats[0] = (double)h;
    stats[1] = mv;
    stats[2] = mn;
    stats[3] = mb;
    return decide_and_step(n, x, y_out, h, mv, mn, mb, lambda, rule, stop, eps,
                           force_step, stats);
}

/* The whole iterative process: iterations at ticks k0, k0+1, ... until the
 * stopping rule holds or max_iter x-updates have been made.
 * out[0..7] = status, iterations, final tick, h, maxviol, maxnorm, maxb,
 * last ||dx||.  work must hold n + m doubles. */
void oracle_solve(int64_t m, int64_t n, const double *A, const double *b0,
                  const double *Av, double rho, int64_t k0, const double *n2,
                  double *x, double lambda, int rule, int stop, double eps,
                  int64_t max_iter, double *work, double *out)
{
    double stats[6] = {0, 0, 0, 0, 0, 0};
    double *y = work;
    double *bk = work + n;
    int64_t it = 0;
    int status = ORACLE_NOT_CONVERGED;
    double last_dx = 0.0;
    for (;;) {
        int64_t k = k0 + it;
        if (it == max_iter) {
            /* evaluate the test once more at the final point, no step */
            oracle_tick_b(m, b0, Av, rho, k, bk);
            int64_t h;
            oracle_map_reduce(m, n, A, bk, n2, x, y, &h, &stats[1], &stats[2],
                              &stats[3], NULL);
            stats[0] = (double)h;
            if ((stop != ORACLE_STOP_NONE && h == 0) ||
                stop_test_passes(stop, eps, stats[1], stats[2], stats[3]))
                status = ORACLE_OK;
            else
                status = ORACLE_NOT_CONVERGED;
            break;
        }
        int code = oracle_iteration(m, n, A, b0, Av, rho, k, n2, x, lambda,
                                    rule, stop, eps, 0, y, bk, NULL, stats);
        if (code == ORACLE_IT_CONVERGED) {
            status = ORACLE_OK;
            break;
        }
        it = it + 1;
        last_dx = stats[4];
        if (code == ORACLE_IT_STEP_STOP) {
            status = ORACLE_OK;
            break;
        }
    }
    out[0] = (double)status;
    out[1] = (double)it;
    out[2] = (double)(k0 + it);
    out[3] = stats[0];
    out[4] = stats[1];
    out[5] = stats[2];
    out[6] = stats[3];
    out[7] = last_dx;
}

/* ---- storage formats: the exact values the stored matrix holds ---------- */

/* Round a binary32 value to the nearest bfloat16 (8-bit exponent, 7 stored
 * mantissa bits), ties to even, from the format's definition: keep the upper
 * 16 bits of the binary32 encoding after adding half of the dropped unit
 * plus the parity of the kept part. */
static float round_to_bf16(float v)
{
    uint32_t u;
    memcpy(&u, &v, sizeof u);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu) != 0u) {
        u = u | 0x00400000u; /* quiet NaN */
    } else {
        uint32_t keep_lsb = (u >> 16) & 1u;
        u = u + 0x7fffu + keep_lsb;
    }
    u = u & 0xffff0000u;
    float r;
    memcpy(&r, &u, sizeof r);
    return r;
}

void oracle_quantize_bf16(int64_t count, const float *in, float *out)
{
    for (int64_t i = 0; i < count; ++i)
        out[i] = round_to_bf16(in[i]);
}

/* Round a finite real to the nearest FP8 E4M3 value (bias 7, 3 mantissa
 * bits, no infinities, largest finite 448, subnormal quantum 2^-9), ties to
 * even, saturating at +-448. */
static double round_to_e4m3(double v)
{
    double a = fabs(v);
    double quantum;
    if (a < ldexp(1.0, -6)) {
        quantum = ldexp(1.0, -9); /* subnormal spacing */
    } else {
        int e2;
        frexp(a, &e2);   /* a = f * 2^e2, f in [0.5, 1) */
        int e = e2 - 1;  /* floor(log2 a) */
        if (e > 8)
            e = 8;
        quantum = ldexp(1.0, e - 3);
    }
    double q = nearbyint(a / quantum) * quantum; /* ties to even */
    if (q > 448.0)
        q = 448.0;
    return (v < 0.0) ? -q : q;
}

/* Per-row FP8 E4M3 storage with a power-of-two row scale: s_i is the
 * smallest power of two with max_j |a_ij| / s_i <= 448, the stored code is
 * e4m3(a_ij / s_i) and the represented value is code * s_i (exact in binary32
 * for these inputs).  A zero row gets s_i = 1. */
void oracle_quantize_e4m3_rows(int64_t m, int64_t n, const float *in,
                               float *out, float *scale)
{
    for (int64_t i = 0; i < m; ++i) {
        double amax = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double a = fabs((double)in[i * n + j]);
            if (a > amax)
                amax = a;
        }
        int e = 0;
        if (amax > 0.0) {
            int e2;
            frexp(amax, &e2);
            e = e2 - 10; /* safely below the answer, then walk up */
            while (ldexp(amax, -e) > 448.0)
                e = e + 1;
            while (ldexp(amax, -(e - 1)) <= 448.0)
                e = e - 1;
        }
        double s = ldexp(1.0, e);
        scale[i] = (float)s;
        for (int64_t j = 0; j < n; ++j) {
            double q = round_to_e4m3((double)in[i * n + j] / s);
            out[i * n + j] = (float)(q * s);
        }
    }
}
