/*
 * oracle/cqk_oracle.c -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, sequential, FP64 CPU oracle for the continuous quadratic knapsack
 * problem (CQK) of Secchin & Silva, "Parallel Newton methods for the continuous
 * quadratic knapsack problem: A Jacobi and Gauss-Seidel tale" (arXiv 2603.15910):
 *
 *     min  1/2 x'Dx - a'x   s.t.  b'x = r,  l <= x <= u,   D = diag(d), d > 0, b > 0.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  It shares no code, header or constant with the
 * CUDA library in paper_2603_15910_b300/.
 *
 * Every routine follows the paper's definitions and algorithms in the paper's
 * order and notation; nothing is blocked, fused or reordered.  Floating point is
 * IEEE FP64 (compiled with -ffp-contract=off, no fast-math).  Sums that the
 * method defines over all n variables are accumulated in `long double` (x87
 * extended precision) so that the oracle is at least as accurate as the method.
 *
 * Routines (paper reference in brackets):
 *   cqko_x              x_i(lambda)                                  [Sec. 2.1, eq. (xopt)]
 *   cqko_phi            phi(lambda), phi'_+(lambda), phi'_-(lambda)  [eq. (opt), eq. (phideriv)]
 *   cqko_lambda0        multiplier ignoring the bounds               [eq. (CQKlambda0)]
 *   cqko_breakpoint     closest breakpoint right / left of lambda    [Sec. 2.1 breakpoints; Alg. 1]
 *   cqko_newton         semismooth Newton with secant safeguard      [Alg. 1; stopping criteria of Sec. 4]
 *   cqko_solve_sort     exact solve by sorting breakpoints           [definition: phi(lambda*) = r]
 *   cqko_condat_init    Condat's multiplier initialisation           [Alg. 2]
 *   cqko_lambda0_warm   eq. (CQKlambda0) over J = {l < xbar < u}      [Sec. 2, start from a primal estimate]
 *   cqko_condat_chunks  Alg. 2 per chunk, union of the J's           [Sec. 4, parallel lambda_0; eq. (lambdaJ)]
 *   cqko_condat_chunks_warm  the same on I = supp(xbar)              [Sec. 3.3 warm start]
 *   cqko_condat         Condat's projection onto the simplex         [Alg. 3]
 *   cqko_newton_simplex specialised Newton for the simplex           [Alg. 4; Theorem 3.1]
 *   cqko_project_simplex_sort  sort-based simplex projection         [textbook closed form, cited in Sec. 1]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/*
 * Threads of the loops over all n variables (the phi evaluations of eq. (opt) and
 * eq. (phideriv), eq. (CQKlambda0), the breakpoint search, the per-chunk Alg. 2 scans of
 * Sec. 4).  1, the default, is the plain sequential oracle that every test uses.  More
 * threads (when compiled with OpenMP) give the paper's CPU Jacobi form of the same method
 * (Sec. 4: the map-reduce split over threads), used only to time the all-core CPU
 * baseline; the rounding order of the sums then depends on the thread count.
 */
static int g_threads = 1;
void cqko_set_threads(int t) { g_threads = t > 1 ? t : 1; }
int cqko_get_threads(void) { return g_threads; }

/* status values returned by the oracle (its own numbering) */
#define ORC_OK 0
#define ORC_INFEASIBLE 1
#define ORC_MAXITER 2
#define ORC_BAD_INPUT 3

/* which test stopped the Newton loop */
#define STOPR_NONE 0
#define STOPR_EXACT 1    /* phi(lambda_k) == r                                  (Alg. 1 / Alg. 4)        */
#define STOPR_RESID 2    /* |phi - r| < eps^{3/4} (sum |b_i x_i| + |r|)          (Sec. 4 criterion 1)     */
#define STOPR_STEP 3     /* |(phi - r)/phi'| < eps^{3/4}                        (Sec. 4 criterion 2)     */
#define STOPR_SAME 4     /* lambda_{k+1} == lambda_k                            (Sec. 4 criterion 2)     */
#define STOPR_BRACKET 5  /* upper - lower < eps^{3/4} max(|upper|, |lower|)      (Sec. 4 criterion 3)     */
#define STOPR_BELOW 6    /* phi(lambda_k) <= r for k >= 1                       (Alg. 4)                 */

/* ------------------------------------------------------------------------- */
/* eq. (xopt): x_i(lambda) = max{l_i, min{u_i, (b_i lambda + a_i)/d_i}}       */
static double x_i(double lam, double a, double b, double d, double l, double u) {
    double t = (b * lam + a) / d;
    return fmax(l, fmin(u, t));
}

void cqko_x(int64_t n, const double* a, const double* b, const double* d, const double* l,
            const double* u, double lam, double* x) {
    for (int64_t i = 0; i < n; i++) x[i] = x_i(lam, a[i], b[i], d[i], l[i], u[i]);
}

/* Breakpoints of Sec. 2.1: lower_i = (d_i l_i - a_i)/b_i, upper_i = (d_i u_i - a_i)/b_i. */
static double brk_lower(double a, double b, double d, double l) { return (d * l - a) / b; }
static double brk_upper(double a, double b, double d, double u) { return (d * u - a) / b; }

/*
 * eq. (opt) and eq. (phideriv):
 *   out[0] = phi(lambda)     = sum_i b_i x_i(lambda)
 *   out[1] = phi'_+(lambda)  = sum over {lower_i <= lambda < upper_i} of b_i^2/d_i
 *   out[2] = phi'_-(lambda)  = sum over {lower_i <  lambda <= upper_i} of b_i^2/d_i
 *   out[3] = sum_i |b_i x_i(lambda)|   (the scale of stopping criterion 1, Sec. 4)
 */
void cqko_phi(int64_t n, const double* a, const double* b, const double* d, const double* l,
              const double* u, double lam, double* out) {
    long double phi = 0.0L, dp = 0.0L, dm = 0.0L, absbx = 0.0L;
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1) reduction(+ : phi, dp, dm, absbx)
    for (int64_t i = 0; i < n; i++) {
        double xi = x_i(lam, a[i], b[i], d[i], l[i], u[i]);
        double lo = brk_lower(a[i], b[i], d[i], l[i]);
        double up = brk_upper(a[i], b[i], d[i], u[i]);
        double w = b[i] * b[i] / d[i];
        phi += (long double)b[i] * (long double)xi;
        absbx += fabsl((long double)b[i] * (long double)xi);
        if (lo <= lam && lam < up) dp += w;
        if (lo < lam && lam <= up) dm += w;
    }
    out[0] = (double)phi;
    out[1] = (double)dp;
    out[2] = (double)dm;
    out[3] = (double)absbx;
}

/* eq. (CQKlambda0) with J = {1..n}: lambda_0 = (r - s)/q, s = sum b_i a_i/d_i, q = sum b_i^2/d_i. */
double cqko_lambda0(int64_t n, const double* a, const double* b, const double* d, double r) {
    long double s = 0.0L, q = 0.0L;
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1) reduction(+ : s, q)
    for (int64_t i = 0; i < n; i++) {
        s += (long double)(b[i] * a[i] / d[i]);
        q += (long double)(b[i] * b[i] / d[i]);
    }
    return (double)(((long double)r - s) / q);
}

/*
 * Start from a primal estimate xbar (Sec. 2, after eq. (CQKlambda0)): the same
 * formula with J = {i : l_i < xbar_i < u_i}, the variables that xbar leaves free;
 * when that set is empty xbar is discarded and J = {1..n}.
 */
double cqko_lambda0_warm(int64_t n, const double* a, const double* b, const double* d,
                         const double* l, const double* u, const double* xbar, double r) {
    long double s = 0.0L, q = 0.0L;
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        if (l[i] < xbar[i] && xbar[i] < u[i]) {
            s += (long double)(b[i] * a[i] / d[i]);
            q += (long double)(b[i] * b[i] / d[i]);
            m++;
        }
    }
    if (m == 0) return cqko_lambda0(n, a, b, d, r);
    return (double)(((long double)r - s) / q);
}

/*
 * Closest finite breakpoint strictly to the right (dir > 0) or strictly to the
 * left (dir < 0) of lam, over both families lower_i and upper_i (Alg. 1, the
 * branches where the needed lateral derivative vanishes).  Returns 0 and sets
 * *found = 0 when there is none.
 */
double cqko_breakpoint(int64_t n, const double* a, const double* b, const double* d,
                       const double* l, const double* u, double lam, int dir, int* found) {
    double best = dir > 0 ? INFINITY : -INFINITY;
    int any = 0;
#pragma omp parallel num_threads(g_threads) if (g_threads > 1)
    {
        double tbest = dir > 0 ? INFINITY : -INFINITY;
        int tfound = 0;
#pragma omp for nowait
        for (int64_t i = 0; i < n; i++) {
            double c[2] = {brk_lower(a[i], b[i], d[i], l[i]), brk_upper(a[i], b[i], d[i], u[i])};
            for (int k = 0; k < 2; k++) {
                if (!isfinite(c[k])) continue;
                if (dir > 0 && c[k] > lam && c[k] < tbest) { tbest = c[k]; tfound = 1; }
                if (dir < 0 && c[k] < lam && c[k] > tbest) { tbest = c[k]; tfound = 1; }
            }
        }
#pragma omp critical
        {
            if (tfound && (!any || (dir > 0 ? tbest < best : tbest > best))) best = tbest;
            any |= tfound;
        }
    }
    *found = any;
    return *found ? best : 0.0;
}

/*
 * Alg. 1 (semismooth Newton for CQK) from lambda_0 = lam0, with the three
 * stopping tests of Sec. 4 (eps34 = machine-eps^{3/4}).
 *
 *  - Each pass evaluates phi, phi'_+, phi'_- and sum|b x| at lambda_k.
 *  - phi < r: lower <- lambda_k; Newton step with phi'_+ if it is positive and
 *    lands strictly left of upper, secant step otherwise; if phi'_+ = 0, the
 *    closest breakpoint right of lower (none: infeasible).  phi > r symmetric.
 *  - Secant step: zero of the line through (lower, phi(lower)) and
 *    (upper, phi(upper)).
 *  - Criterion 1 is tested on phi(lambda_k); criterion 2 on the Newton step
 *    computed from lambda_k (its size, or lambda_{k+1} == lambda_k); criterion 3
 *    on the bracket after it has been updated with lambda_k.
 *
 * Outputs: lam_out = lambda_k at the stop (x = x(lambda_k)); evals = number of
 * phi evaluations; bpsearch = number of breakpoint searches; nsecant = number of
 * secant steps; stop = STOPR_*;
 * step_out = the Newton step available at the stop from lambda_k inside the
 * bracket (0 if none) -- used by the final-step variant of the tests;
 * trace (nullable, >= max_iter entries) = lambda_0 .. lambda_k.
 */
int cqko_newton(int64_t n, const double* a, const double* b, const double* d, const double* l,
                const double* u, double r, double lam0, int max_iter, double eps34,
                double* lam_out, int* evals, int* bpsearch, int* nsecant, int* stop, double* step_out,
                double* trace) {
    double lower = -INFINITY, upper = INFINITY, phi_lower = NAN, phi_upper = NAN;
    double lam = lam0;
    double f[4];
    *evals = 0; *bpsearch = 0; *nsecant = 0; *stop = STOPR_NONE; *step_out = 0.0; *lam_out = lam;
    for (int k = 0; k < max_iter; k++) {
        if (trace) trace[k] = lam;
        cqko_phi(n, a, b, d, l, u, lam, f);
        (*evals)++;
        double phi = f[0], dplus = f[1], dminus = f[2], absbx = f[3];
        double g = phi - r;
        *lam_out = lam;
        if (g == 0.0) { *stop = STOPR_EXACT; return ORC_OK; }
        if (fabs(g) < eps34 * (absbx + fabs(r))) {
            *stop = STOPR_RESID;
            double s = g < 0 ? (dplus > 0 ? -g / dplus : 0.0) : (dminus > 0 ? -g / dminus : 0.0);
            double t = lam + s;
            if (g < 0 && !(t < upper)) s = 0.0;
            if (g > 0 && !(t > lower)) s = 0.0;
            *step_out = s;
            return ORC_OK;
        }
        double next;
        int newton = 0;
        if (g < 0) {
            lower = lam; phi_lower = phi;
            if (dplus > 0) {
                double step = -g / dplus;
                if (fabs(step) < eps34) { *stop = STOPR_STEP; *step_out = step; return ORC_OK; }
                double t = lam + step;
                if (t < upper) { next = t; newton = 1; }
                else { next = lower - (phi_lower - r) * (upper - lower) / (phi_upper - phi_lower); (*nsecant)++; }
            } else {
                int found;
                (*bpsearch)++;
                next = cqko_breakpoint(n, a, b, d, l, u, lower, +1, &found);
                if (!found) { *stop = STOPR_NONE; return ORC_INFEASIBLE; }
            }
        } else {
            upper = lam; phi_upper = phi;
            if (dminus > 0) {
                double step = -g / dminus;
                if (fabs(step) < eps34) { *stop = STOPR_STEP; *step_out = step; return ORC_OK; }
                double t = lam + step;
                if (t > lower) { next = t; newton = 1; }
                else { next = lower - (phi_lower - r) * (upper - lower) / (phi_upper - phi_lower); (*nsecant)++; }
            } else {
                int found;
                (*bpsearch)++;
                next = cqko_breakpoint(n, a, b, d, l, u, upper, -1, &found);
                if (!found) { *stop = STOPR_NONE; return ORC_INFEASIBLE; }
            }
        }
        (void)newton;
        if (upper - lower < eps34 * fmax(fabs(upper), fabs(lower))) { *stop = STOPR_BRACKET; return ORC_OK; }
        if (next == lam) { *stop = STOPR_SAME; return ORC_OK; }
        lam = next;
    }
    return ORC_MAXITER;
}

/* ------------------------------------------------------------------------- */
/* Exact solve from the definition: phi is piecewise linear and non-decreasing
 * (Sec. 2.1), so lambda* with phi(lambda*) = r lies on a segment between two
 * consecutive breakpoints (or on an unbounded end segment).  Sort the finite
 * breakpoints, bisect over them evaluating phi directly, and interpolate on the
 * bracketing segment.  O(n log n).  Returns ORC_INFEASIBLE when r lies outside
 * [b'l, b'u].  On success x = x(lambda*). */
static int cmp_double(const void* p, const void* q) {
    double x = *(const double*)p, y = *(const double*)q;
    return (x > y) - (x < y);
}

static double phi_only(int64_t n, const double* a, const double* b, const double* d,
                       const double* l, const double* u, double lam) {
    long double s = 0.0L;
    for (int64_t i = 0; i < n; i++) s += (long double)b[i] * (long double)x_i(lam, a[i], b[i], d[i], l[i], u[i]);
    return (double)s;
}

/* On an open interval between consecutive breakpoints every variable keeps one
 * status (at l, at u, or free), so phi(lambda) = sum_L b l + sum_U b u +
 * sum_F b (a + lambda b)/d there, and phi(lambda) = r gives the closed form
 * lambda = (r - sum_L b l - sum_U b u - sum_F b a/d) / sum_F b^2/d
 * (eq. (CQKlambda0) with J = F and the fixed variables moved to the right-hand
 * side).  The statuses are read at an interior point m of the interval.
 * Returns 0 when the interval has no free variable (phi is flat there). */
static int segment_lambda(int64_t n, const double* a, const double* b, const double* d,
                          const double* l, const double* u, double r, double m, double* lam) {
    long double fixed = 0.0L, s = 0.0L, q = 0.0L;
    for (int64_t i = 0; i < n; i++) {
        double lo = brk_lower(a[i], b[i], d[i], l[i]), up = brk_upper(a[i], b[i], d[i], u[i]);
        if (m <= lo) fixed += (long double)b[i] * l[i];
        else if (m >= up) fixed += (long double)b[i] * u[i];
        else {
            s += (long double)(b[i] * a[i] / d[i]);
            q += (long double)(b[i] * b[i] / d[i]);
        }
    }
    if (!(q > 0.0L)) return 0;
    *lam = (double)(((long double)r - fixed - s) / q);
    return 1;
}

int cqko_solve_sort(int64_t n, const double* a, const double* b, const double* d, const double* l,
                    const double* u, double r, double* lam_out, double* x) {
    /* feasibility: r must lie in [sum b_i l_i, sum b_i u_i] */
    long double lo_sum = 0.0L, up_sum = 0.0L;
    int lo_inf = 0, up_inf = 0;
    for (int64_t i = 0; i < n; i++) {
        if (isinf(l[i])) lo_inf = 1; else lo_sum += (long double)b[i] * l[i];
        if (isinf(u[i])) up_inf = 1; else up_sum += (long double)b[i] * u[i];
    }
    if ((!lo_inf && (long double)r < lo_sum) || (!up_inf && (long double)r > up_sum)) return ORC_INFEASIBLE;

    double* bp = (double*)malloc(sizeof(double) * (size_t)(2 * n + 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        double c0 = brk_lower(a[i], b[i], d[i], l[i]), c1 = brk_upper(a[i], b[i], d[i], u[i]);
        if (isfinite(c0)) bp[m++] = c0;
        if (isfinite(c1)) bp[m++] = c1;
    }
    double lam = 0.0;
    int ok = 1;
    if (m == 0) {
        /* no finite breakpoint: every variable is free for every lambda */
        ok = segment_lambda(n, a, b, d, l, u, r, 0.0, &lam);
    } else {
        qsort(bp, (size_t)m, sizeof(double), cmp_double);
        double plo = phi_only(n, a, b, d, l, u, bp[0]);
        double phi_hi = phi_only(n, a, b, d, l, u, bp[m - 1]);
        if (r == plo) lam = bp[0];
        else if (r == phi_hi) lam = bp[m - 1];
        else if (r < plo) {
            /* left end segment (-inf, bp[0]) */
            ok = segment_lambda(n, a, b, d, l, u, r, bp[0] - (fabs(bp[0]) + 1.0), &lam);
        } else if (r > phi_hi) {
            /* right end segment (bp[m-1], +inf) */
            ok = segment_lambda(n, a, b, d, l, u, r, bp[m - 1] + (fabs(bp[m - 1]) + 1.0), &lam);
        } else {
            /* bisection over the sorted breakpoints; invariant phi(bp[lo]) < r < phi(bp[hi]) */
            int64_t lo = 0, hi = m - 1;
            int exact = 0;
            while (hi - lo > 1) {
                int64_t mid = lo + (hi - lo) / 2;
                double pm = phi_only(n, a, b, d, l, u, bp[mid]);
                if (pm == r) { lam = bp[mid]; exact = 1; break; }
                if (pm < r) lo = mid; else hi = mid;
            }
            if (!exact) {
                double mid = bp[lo] + 0.5 * (bp[hi] - bp[lo]);
                ok = segment_lambda(n, a, b, d, l, u, r, mid, &lam);
                /* rounding can push the closed form a hair outside the segment */
                if (ok) lam = fmin(fmax(lam, bp[lo]), bp[hi]);
            }
        }
    }
    free(bp);
    if (!ok) return ORC_INFEASIBLE;
    *lam_out = lam;
    if (x) cqko_x(n, a, b, d, l, u, lam, x);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/*
 * Alg. 2 (initialise lambda, simplex projection) on the ordered index subset
 * I = (idx[0], ..., idx[p-1]).  y_i is read as |y_i| when l1 != 0 and the
 * membership test y + lambda > 0 becomes min{|y|, |y| + lambda} > 0 (Sec. 3.2,
 * the strengthened test before Lemma 3.2).  J is kept as its running sum and
 * size; the multiplier is always lambda_J = (r - sum_J y)/|J| (eq. (lambdaJ)).
 * J~ (the sets dropped on restarts) is kept as an ordered list.
 * Outputs: *jsum = sum_{j in J} y_j, *jcount = |J|.  Returns lambda_J.
 */
static double yv(const double* y, int64_t i, int l1) { return l1 ? fabs(y[i]) : y[i]; }
static int passes(double yi, double lam, int l1) {
    return l1 ? (fmin(yi, yi + lam) > 0.0) : (yi + lam > 0.0);
}

double cqko_condat_init(const double* y, const int64_t* idx, int64_t p, double r, int l1,
                        double* jsum, int64_t* jcount, int64_t* scratch /* 2p entries */,
                        double* trace /* nullable: lambda after each scanned entry, first loop */) {
    int64_t* Jlist = scratch;       /* members of J, in order of insertion  */
    int64_t* Jt = scratch + p;      /* J~, in order of insertion            */
    int64_t nJ = 0, nJt = 0;
    double S = 0.0;
    double lam;
    if (p == 0) { *jsum = 0.0; *jcount = 0; return NAN; }
    Jlist[nJ++] = idx[0];
    S = yv(y, idx[0], l1);
    lam = r - S;
    if (trace) trace[0] = lam;
    for (int64_t j = 1; j < p; j++) {
        double yj = yv(y, idx[j], l1);
        if (passes(yj, lam, l1)) {
            lam = (r - S - yj) / (double)(nJ + 1);
            if (lam < r - yj) {
                Jlist[nJ++] = idx[j];
                S += yj;
            } else {
                for (int64_t k = 0; k < nJ; k++) Jt[nJt++] = Jlist[k];
                nJ = 0;
                Jlist[nJ++] = idx[j];
                S = yj;
                lam = r - yj;
            }
        }
        if (trace) trace[j] = lam;
    }
    for (int64_t k = 0; k < nJt; k++) {
        double yj = yv(y, Jt[k], l1);
        if (passes(yj, lam, l1)) {
            lam = (r - S - yj) / (double)(nJ + 1);
            Jlist[nJ++] = Jt[k];
            S += yj;
        }
    }
    *jsum = S;
    *jcount = nJ;
    return lam;
}

/*
 * Parallel initial multiplier of Sec. 4: each worker runs Alg. 2 on its own
 * subset I of the variables and lambda_0 follows from eq. (lambdaJ) on the union
 * of the returned J's, using the per-chunk partial sums.
 * The subsets are the chunks of a fixed partition: variable i belongs to chunk
 * ((i + shift) / tile) mod nchunks and every chunk is scanned in increasing i
 * (shift places the first tile boundary; 0 for a problem that starts a tile).
 * Outputs: lambda_0, the union's sum and size.
 */
double cqko_condat_chunks(int64_t n, const double* y, double r, int l1, int64_t tile,
                          int64_t nchunks, int64_t shift, double* usum, int64_t* ucount) {
    int64_t ntiles = (n + shift + tile - 1) / tile;
    int64_t maxp = ((ntiles + nchunks - 1) / nchunks) * tile;
    long double S = 0.0L;
    int64_t C = 0;
#pragma omp parallel num_threads(g_threads) if (g_threads > 1) reduction(+ : S, C)
    {
        int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxp > 0 ? maxp : 1));
        int64_t* scratch = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * (maxp > 0 ? maxp : 1)));
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < nchunks; c++) {
            int64_t p = 0;
            for (int64_t t = c; t < ntiles; t += nchunks)
                for (int64_t i = t * tile - shift; i < (t + 1) * tile - shift && i < n; i++)
                    if (i >= 0) idx[p++] = i;
            if (p == 0) continue;
            double js; int64_t jc;
            cqko_condat_init(y, idx, p, r, l1, &js, &jc, scratch, NULL);
            S += js;
            C += jc;
        }
        free(idx);
        free(scratch);
    }
    *usum = (double)S;
    *ucount = C;
    return (double)(((long double)r - S) / (long double)C);
}

/*
 * Warm start of Sec. 3.3: Alg. 2 run on I = supp(xbar) = {i : xbar_i > 0} (l1 ball:
 * xbar_i != 0), here per chunk of the same partition as cqko_condat_chunks (an element
 * outside the support is skipped by its chunk's scan).  When no chunk keeps an element
 * (J_+ empty) the multiplier is max{r/n, -y_1} as the paper sets it (l1 ball: |y_1|).
 */
double cqko_condat_chunks_warm(int64_t n, const double* y, const double* xbar, double r, int l1,
                               int64_t tile, int64_t nchunks, int64_t shift, double* usum,
                               int64_t* ucount) {
    int64_t ntiles = (n + shift + tile - 1) / tile;
    int64_t maxp = ((ntiles + nchunks - 1) / nchunks) * tile;
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(maxp > 0 ? maxp : 1));
    int64_t* scratch = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * (maxp > 0 ? maxp : 1)));
    long double S = 0.0L;
    int64_t C = 0;
    for (int64_t c = 0; c < nchunks; c++) {
        int64_t p = 0;
        for (int64_t t = c; t < ntiles; t += nchunks)
            for (int64_t i = t * tile - shift; i < (t + 1) * tile - shift && i < n; i++)
                if (i >= 0 && (l1 ? xbar[i] != 0.0 : xbar[i] > 0.0)) idx[p++] = i;
        if (p == 0) continue;
        double js; int64_t jc;
        cqko_condat_init(y, idx, p, r, l1, &js, &jc, scratch, NULL);
        S += js;
        C += jc;
    }
    free(idx);
    free(scratch);
    *usum = (double)S;
    *ucount = C;
    if (C == 0) {
        double y1 = l1 ? fabs(y[0]) : y[0];
        return fmax(r / (double)n, -y1);
    }
    return (double)(((long double)r - S) / (long double)C);
}

/*
 * Alg. 3 (Condat's projection onto the simplex {x >= 0, sum x = r}): lambda and
 * J from Alg. 2 with I = {1..n}, then repeatedly drop j in J with
 * y_j + lambda <= 0, updating lambda = lambda_J of eq. (lambdaJ) after each drop,
 * until J no longer changes; x = max{0, y + lambda}.  Returns lambda.
 */
double cqko_condat(int64_t n, const double* y, double r, double* x) {
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* scratch = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * (n > 0 ? n : 1)));
    for (int64_t i = 0; i < n; i++) idx[i] = i;
    double S; int64_t nJ;
    /* Alg. 2 leaves J in scratch[0 .. nJ) */
    double lam = cqko_condat_init(y, idx, n, r, 0, &S, &nJ, scratch, NULL);
    int64_t* J = scratch;
    int changed = 1;
    while (changed) {
        changed = 0;
        int64_t keep = 0;
        for (int64_t k = 0; k < nJ; k++) {
            int64_t j = J[k];
            int64_t size_after = keep + (nJ - k - 1);
            if (y[j] + lam <= 0.0 && size_after > 0) {
                /* drop j: J <- J \ {j}; lambda <- lambda_J of the smaller J */
                S -= y[j];
                lam = (r - S) / (double)size_after;
                changed = 1;
            } else {
                J[keep++] = j;
            }
        }
        nJ = keep;
    }
    if (x) for (int64_t i = 0; i < n; i++) x[i] = fmax(0.0, y[i] + lam);
    free(idx);
    free(scratch);
    return lam;
}

/* ------------------------------------------------------------------------- */
/* Simplex specialisation of eq. (opt) and eq. (phideriv) (proof of Theorem 3.1):
 * phi(lambda) = sum max{0, y_i + lambda}, phi'_+ = #{-y_i <= lambda}, phi'_- = #{-y_i < lambda}.
 * y is read as |y| when l1 != 0 (Sec. 3.2). */
static void phi_simplex(int64_t n, const double* y, int l1, double lam, double* out) {
    long double phi = 0.0L;
    int64_t dp = 0, dm = 0;
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1) reduction(+ : phi, dp, dm)
    for (int64_t i = 0; i < n; i++) {
        double yi = yv(y, i, l1);
        phi += (long double)fmax(0.0, yi + lam);
        if (-yi <= lam) dp++;
        if (-yi < lam) dm++;
    }
    out[0] = (double)phi;
    out[1] = (double)dp;
    out[2] = (double)dm;
}

/*
 * Alg. 4 (semismooth Newton for the projection onto the r-simplex) from lam0,
 * with stopping criteria 2 and 3 of Sec. 4 (criterion 1 is not used for the
 * simplex), for y (or |y| when l1 != 0).
 *  line 1: lambda_0 <- max{lambda_0, min_i(-y_i)}
 *  k = 0: stop if phi = r; one Newton step with phi'_+ if phi < r, else phi'_-
 *  k >= 1: stop if phi(lambda_k) <= r; otherwise a Newton step with phi'_-.
 * Outputs as cqko_newton (trace, when given, receives lambda_0 .. lambda_k).
 */
int cqko_newton_simplex(int64_t n, const double* y, double r, int l1, double lam0, int max_iter,
                        double eps34, double* lam_out, int* evals, int* stop, double* trace) {
    double ymin = INFINITY;
#pragma omp parallel for num_threads(g_threads) if (g_threads > 1) reduction(min : ymin)
    for (int64_t i = 0; i < n; i++) { double v = -yv(y, i, l1); if (v < ymin) ymin = v; }
    double lam = fmax(lam0, ymin);
    double lower = -INFINITY, upper = INFINITY;
    double f[3];
    *evals = 0; *stop = STOPR_NONE; *lam_out = lam;
    for (int k = 0; k < max_iter; k++) {
        if (trace) trace[k] = lam;
        phi_simplex(n, y, l1, lam, f);
        (*evals)++;
        double g = f[0] - r;
        *lam_out = lam;
        double step;
        if (k == 0) {
            if (g == 0.0) { *stop = STOPR_EXACT; return ORC_OK; }
            if (g < 0) { lower = lam; step = -g / f[1]; }
            else { upper = lam; step = -g / f[2]; }
        } else {
            if (g <= 0.0) { *stop = STOPR_BELOW; return ORC_OK; }
            upper = lam;
            step = -g / f[2];
        }
        if (upper - lower < eps34 * fmax(fabs(upper), fabs(lower))) { *stop = STOPR_BRACKET; return ORC_OK; }
        if (fabs(step) < eps34) { *stop = STOPR_STEP; return ORC_OK; }
        double next = lam + step;
        if (next == lam) { *stop = STOPR_SAME; return ORC_OK; }
        lam = next;
    }
    return ORC_MAXITER;
}

/* Textbook sort-based projection onto {x >= 0, sum x = r} (Held-Wolfe-Crowder;
 * Duchi et al. 2008, cited in Sec. 1): sort y decreasingly, rho = the largest j
 * with y_(j) - (sum_{i<=j} y_(i) - r)/j > 0, lambda* = (r - sum_{i<=rho} y_(i))/rho,
 * x = max{0, y + lambda*}.  Returns lambda*. */
static int cmp_desc(const void* p, const void* q) {
    double x = *(const double*)p, y = *(const double*)q;
    return (x < y) - (x > y);
}

double cqko_project_simplex_sort(int64_t n, const double* y, double r, double* x) {
    double* s = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(s, y, sizeof(double) * (size_t)n);
    qsort(s, (size_t)n, sizeof(double), cmp_desc);
    long double cum = 0.0L, cum_rho = 0.0L;
    int64_t rho = 0;
    for (int64_t j = 0; j < n; j++) {
        cum += s[j];
        if ((long double)s[j] - (cum - r) / (long double)(j + 1) > 0.0L) { rho = j + 1; cum_rho = cum; }
    }
    double lam = (double)(((long double)r - cum_rho) / (long double)rho);
    if (x) for (int64_t i = 0; i < n; i++) x[i] = fmax(0.0, y[i] + lam);
    free(s);
    return lam;
}
