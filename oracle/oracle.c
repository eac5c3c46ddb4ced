/*
 * oracle.c -- plain, slow FP64 CPU reference for the 2D Laplace solvers compared
 * in "A Comparison of SOR, ADI and Multigrid Methods for Solving Partial
 * Differential Equations" (arXiv 2208.02427).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load or call this library. It shares no code with the
 * CUDA path and is never a fallback for it.
 *
 * Every routine follows one passage of the paper, in the paper's order and
 * notation; where the paper is silent or garbled the reading taken is stated
 * beside the code. Build with -ffp-contract=off: the only fused multiply-adds
 * are the explicit fma() calls, so every value is rounded exactly as written.
 *
 * Readings fixed here (the paper is ambiguous or garbled on these):
 *  - Eq. 2 / Eq. 11 print dx^2 under the y-difference; the y-difference is taken
 *    over dy^2, which is what the beta = dx/dy of Eq. 5 implies.
 *  - Division by d = 2(1+beta^2) is a multiplication by the double nearest 1/d
 *    (exact when beta = 1, where 1/d = 1/4).
 *  - The beta^2 term of the neighbour sum is fused into the final addition:
 *    fma(beta^2, N + S, E + W). For beta = 1 this equals (E + W) + (N + S).
 *  - Eq. 7 prints u^k for psi^k; Eq. 8 misses a parenthesis and its boundary
 *    terms; Eq. 10's coefficients are garbled and are re-derived below from
 *    Eq. 7 solved implicitly along the line.
 *  - Restriction and interpolation operators are not named by the paper; full
 *    weighting and bilinear interpolation are used. Coarse levels keep beta and
 *    double both spacings, and carry the correction equation of Eq. 15 in the
 *    scaled form (E+W) + b2 (N+S) - d e + q = 0 with q = 4 FW(r_fine).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define AT(a, m, i, j) ((a)[(size_t)(j) * (size_t)(m) + (size_t)(i)])

static void coefficients(double beta, double* b2, double* d)
{
    *b2 = beta * beta;
    *d = 2.0 * (1.0 + *b2);
}

/* Neighbour sum of Eq. 5: psi_{i+1,j} + psi_{i-1,j} + beta^2 (psi_{i,j+1} + psi_{i,j-1}). */
static double neighbour_sum(const double* p, int m, int i, int j, double b2)
{
    double ew = AT(p, m, i - 1, j) + AT(p, m, i + 1, j);
    double ns = AT(p, m, i, j - 1) + AT(p, m, i, j + 1);
    return fma(b2, ns, ew);
}

/* The same sum for beta = 1 with the four terms paired the other way, west with south and
 * east with north: (psi_{i-1,j} + psi_{i,j-1}) + (psi_{i+1,j} + psi_{i,j+1}). Eq. 5 fixes no
 * order of its additions; this one differs from neighbour_sum only in rounding. */
static double neighbour_sum_diagonal(const double* p, int m, int i, int j)
{
    double ws = AT(p, m, i - 1, j) + AT(p, m, i, j - 1);
    double en = AT(p, m, i + 1, j) + AT(p, m, i, j + 1);
    return ws + en;
}

static double neighbour_sum_ordered(const double* p, int m, int i, int j, double b2, int order)
{
    return order == ORA_SUM_DIAGONAL ? neighbour_sum_diagonal(p, m, i, j)
                                     : neighbour_sum(p, m, i, j, b2);
}

/* ------------------------------------------------------------------------- */
/* Residual, Eqs. 11-12. R = L(psi) is scaled by dx^2 so that it reads
 * r = (E + W) + beta^2 (N + S) - d psi, plus the source term q of a coarse level
 * (V-cycle steps 4-5: L(dpsi) + R = 0). r is defined on interior nodes only.  */
void ora_defect(int m, int n, double beta, const double* psi, const double* q, double* r)
{
    double b2, d;
    coefficients(beta, &b2, &d);
    memset(r, 0, sizeof(double) * (size_t)m * (size_t)n);
    for (int j = 1; j < n - 1; ++j)
        for (int i = 1; i < m - 1; ++i) {
            double s = neighbour_sum(psi, m, i, j, b2);
            if (q) s = s + AT(q, m, i, j);
            AT(r, m, i, j) = fma(-d, AT(psi, m, i, j), s);
        }
}

double ora_defect_norm_l2(int m, int n, double beta, const double* psi, const double* q)
{
    double b2, d, acc = 0.0;
    coefficients(beta, &b2, &d);
    for (int j = 1; j < n - 1; ++j)
        for (int i = 1; i < m - 1; ++i) {
            double s = neighbour_sum(psi, m, i, j, b2);
            if (q) s = s + AT(q, m, i, j);
            double r = fma(-d, AT(psi, m, i, j), s);
            acc += r * r;
        }
    return sqrt(acc);
}

/* ------------------------------------------------------------------------- */
/* Jacobi, Eq. 5: every point from the old iterate. */
void ora_jacobi_sweep(int m, int n, double beta, const double* in, double* out)
{
    double b2, d;
    coefficients(beta, &b2, &d);
    double inv_d = 1.0 / d;
    memcpy(out, in, sizeof(double) * (size_t)m * (size_t)n); /* ring */
    for (int j = 1; j < n - 1; ++j)
        for (int i = 1; i < m - 1; ++i)
            AT(out, m, i, j) = neighbour_sum(in, m, i, j, b2) * inv_d;
}

/* Visit order of a point sweep: lexicographic (Eq. 6: i-1 and j-1 already new)
 * or red-black (all i+j even, then all i+j odd). */
static int colour_count(int ordering) { return ordering == ORA_RB ? 2 : 1; }
static int visits(int ordering, int colour, int i, int j)
{
    return ordering == ORA_RB ? ((i + j) & 1) == colour : 1;
}

/* Gauss-Seidel, Eq. 6 (source q on coarse levels), neighbour sum in order sum_order. */
int ora_gs_sweep_ordered(int m, int n, double beta, int ordering, int sum_order, double* psi,
                         const double* q)
{
    double b2, d;
    coefficients(beta, &b2, &d);
    if (sum_order == ORA_SUM_DIAGONAL && b2 != 1.0) return -1;
    double inv_d = 1.0 / d;
    for (int c = 0; c < colour_count(ordering); ++c)
        for (int j = 1; j < n - 1; ++j)
            for (int i = 1; i < m - 1; ++i) {
                if (!visits(ordering, c, i, j)) continue;
                double s = neighbour_sum_ordered(psi, m, i, j, b2, sum_order);
                if (q) s = s + AT(q, m, i, j);
                AT(psi, m, i, j) = s * inv_d;
            }
    return 0;
}

void ora_gs_sweep(int m, int n, double beta, int ordering, double* psi, const double* q)
{
    ora_gs_sweep_ordered(m, n, beta, ordering, ORA_SUM_PAPER, psi, q);
}

/* SOR, Eq. 7: psi^{k+1} = (1 - w) psi^k + w * (Gauss-Seidel value of Eq. 6). */
int ora_sor_sweep_ordered(int m, int n, double beta, double w, int ordering, int sum_order,
                          double* psi, const double* q)
{
    double b2, d;
    coefficients(beta, &b2, &d);
    if (sum_order == ORA_SUM_DIAGONAL && b2 != 1.0) return -1;
    double inv_d = 1.0 / d, one_minus_w = 1.0 - w;
    for (int c = 0; c < colour_count(ordering); ++c)
        for (int j = 1; j < n - 1; ++j)
            for (int i = 1; i < m - 1; ++i) {
                if (!visits(ordering, c, i, j)) continue;
                double s = neighbour_sum_ordered(psi, m, i, j, b2, sum_order);
                if (q) s = s + AT(q, m, i, j);
                double gs = s * inv_d;
                AT(psi, m, i, j) = fma(w, gs, one_minus_w * AT(psi, m, i, j));
            }
    return 0;
}

void ora_sor_sweep(int m, int n, double beta, double w, int ordering, double* psi,
                   const double* q)
{
    ora_sor_sweep_ordered(m, n, beta, w, ordering, ORA_SUM_PAPER, psi, q);
}

/* ------------------------------------------------------------------------- */
/* Thomas algorithm for tridiagonal systems (named in the Introduction and used by
 * SLOR): forward elimination, then back substitution. cp, dp: work of length N. */
void ora_thomas(int N, const double* a, const double* b, const double* c, const double* d,
                double* x, double* cp, double* dp)
{
    cp[0] = N > 1 ? c[0] / b[0] : 0.0;
    dp[0] = d[0] / b[0];
    for (int i = 1; i < N; ++i) {
        double den = b[i] - a[i] * cp[i - 1];
        cp[i] = i < N - 1 ? c[i] / den : 0.0;
        dp[i] = (d[i] - a[i] * dp[i - 1]) / den;
    }
    x[N - 1] = dp[N - 1];
    for (int i = N - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
}

/* Value of the field at position k (0..len+1) of line `line` in direction dir:
 * dir 0 walks row j = line along i, dir 1 walks column i = line along j. */
static double* line_at(double* psi, int m, int dir, int line, int k)
{
    return dir == 0 ? &AT(psi, m, k, line) : &AT(psi, m, line, k);
}

/* One line of SLOR (Eqs. 8-10). Along the line the coupling is `off`
 * (1 for x-lines, beta^2 for y-lines); the two neighbouring lines enter the
 * right-hand side with weight `cross` (beta^2 for x-lines, 1 for y-lines).
 *  form A (Eq. 8 then Eq. 9):
 *     -off x_{k-1} + d x_k - off x_{k+1} = cross (P_k + Q_k),  psi <- psi + w (x - psi)
 *  form B (Eq. 10 re-derived from Eq. 7 made implicit along the line):
 *     -w off x_{k-1} + d x_k - w off x_{k+1} = d (1 - w) psi_k + w cross (P_k + Q_k),  psi <- x
 * P, Q are the current values on the neighbouring lines; the two Dirichlet ends of
 * the line move to the right-hand side of the first and last equations. */
static void relax_line(int m, int n, double b2, double d, double w, int form, int dir, int line,
                       double* psi, double* a, double* b, double* c, double* rhs, double* x,
                       double* cp, double* dp)
{
    int len = dir == 0 ? m - 2 : n - 2;
    double off = dir == 0 ? 1.0 : b2;
    double cross = dir == 0 ? b2 : 1.0;
    double coupling = form == ORA_FORM_A ? off : w * off;
    for (int k = 1; k <= len; ++k) {
        double nb = dir == 0 ? AT(psi, m, k, line - 1) + AT(psi, m, k, line + 1)
                             : AT(psi, m, line - 1, k) + AT(psi, m, line + 1, k);
        double here = *line_at(psi, m, dir, line, k);
        double r = form == ORA_FORM_A ? cross * nb : d * (1.0 - w) * here + w * (cross * nb);
        if (k == 1) r += coupling * *line_at(psi, m, dir, line, 0);
        if (k == len) r += coupling * *line_at(psi, m, dir, line, len + 1);
        a[k - 1] = -coupling;
        b[k - 1] = d;
        c[k - 1] = -coupling;
        rhs[k - 1] = r;
    }
    ora_thomas(len, a, b, c, rhs, x, cp, dp);
    for (int k = 1; k <= len; ++k) {
        double* p = line_at(psi, m, dir, line, k);
        *p = form == ORA_FORM_A ? *p + w * (x[k - 1] - *p) : x[k - 1];
    }
    (void)n;
}

void ora_line_sweep(int m, int n, double beta, double w, int form, int dir, int line_order,
                    double* psi)
{
    double b2, d;
    coefficients(beta, &b2, &d);
    int lines = dir == 0 ? n - 2 : m - 2;
    int len = dir == 0 ? m - 2 : n - 2;
    double* work = (double*)malloc(sizeof(double) * 7 * (size_t)len);
    double *a = work, *b = a + len, *c = b + len, *rhs = c + len, *x = rhs + len, *cp = x + len,
           *dp = cp + len;
    if (line_order == ORA_LINES_ZEBRA) {
        for (int start = 1; start <= 2; ++start) /* odd lines, then even lines */
            for (int l = start; l <= lines; l += 2)
                relax_line(m, n, b2, d, w, form, dir, l, psi, a, b, c, rhs, x, cp, dp);
    } else {
        for (int l = 1; l <= lines; ++l)
            relax_line(m, n, b2, d, w, form, dir, l, psi, a, b, c, rhs, x, cp, dp);
    }
    free(work);
}

/* ADI: one cycle is a sweep by rows followed by a sweep by columns. */
void ora_adi_iteration(int m, int n, double beta, double w, int form, int line_order, double* psi)
{
    ora_line_sweep(m, n, beta, w, form, 0, line_order, psi);
    ora_line_sweep(m, n, beta, w, form, 1, line_order, psi);
}

/* ------------------------------------------------------------------------- */
/* V-cycle step 3/6: restrict the fine residual by full weighting,
 * FW(r)(I,J) = [4 r(2I,2J) + 2 (edge neighbours) + (corner neighbours)] / 16,
 * and scale it to the coarse equation: the coarse spacing is twice the fine one,
 * so q_c = (2h)^2 FW(R) = 4 FW(r) with r = h^2 R. */
void ora_restrict_fw(int mf, int nf, const double* rf, double* qc)
{
    int mc = (mf - 1) / 2 + 1, nc = (nf - 1) / 2 + 1;
    memset(qc, 0, sizeof(double) * (size_t)mc * (size_t)nc);
    for (int J = 1; J < nc - 1; ++J)
        for (int I = 1; I < mc - 1; ++I) {
            int i = 2 * I, j = 2 * J;
            double centre = AT(rf, mf, i, j);
            double edges = (AT(rf, mf, i - 1, j) + AT(rf, mf, i + 1, j)) +
                           (AT(rf, mf, i, j - 1) + AT(rf, mf, i, j + 1));
            double corners = (AT(rf, mf, i - 1, j - 1) + AT(rf, mf, i + 1, j - 1)) +
                             (AT(rf, mf, i - 1, j + 1) + AT(rf, mf, i + 1, j + 1));
            AT(qc, mc, I, J) = 0.25 * ((4.0 * centre + 2.0 * edges) + corners);
        }
}

/* V-cycle steps 8 and 10: interpolate the coarse correction bilinearly and add it
 * (Eq. 13: psi = dpsi + psi^k). Coincident nodes copy, edge midpoints average two
 * coarse values, cell centres average four. Coarse ring values are zero. */
void ora_prolong_add(int mc, int nc, const double* ec, int mf, int nf, double* uf)
{
    (void)nc;
    for (int j = 1; j < nf - 1; ++j)
        for (int i = 1; i < mf - 1; ++i) {
            int I = i / 2, J = j / 2;
            double e;
            if (!(i & 1) && !(j & 1))
                e = AT(ec, mc, I, J);
            else if ((i & 1) && !(j & 1))
                e = 0.5 * (AT(ec, mc, I, J) + AT(ec, mc, I + 1, J));
            else if (!(i & 1) && (j & 1))
                e = 0.5 * (AT(ec, mc, I, J) + AT(ec, mc, I, J + 1));
            else
                e = 0.25 * ((AT(ec, mc, I, J) + AT(ec, mc, I + 1, J)) +
                            (AT(ec, mc, I, J + 1) + AT(ec, mc, I + 1, J + 1)));
            AT(uf, mf, i, j) = AT(uf, mf, i, j) + e;
        }
}

/* V-cycle step 7 solved exactly: Gaussian elimination with partial pivoting on
 * the dense 5-point system d u_k - (interior neighbours) = q_k + (ring neighbours),
 * unknowns numbered k = (j-1)(m-2) + (i-1). Returns 0, or -1 if too large. */
int ora_coarse_direct(int m, int n, double beta, double* u, const double* q)
{
    double b2, d;
    coefficients(beta, &b2, &d);
    int mi = m - 2, ni = n - 2, N = mi * ni;
    if (N <= 0) return 0;
    if (N > 4096) return -1;
    double* A = (double*)calloc((size_t)N * (size_t)N, sizeof(double));
    double* rhs = (double*)malloc(sizeof(double) * (size_t)N);
    if (!A || !rhs) { free(A); free(rhs); return -1; }
    for (int j = 1; j <= ni; ++j)
        for (int i = 1; i <= mi; ++i) {
            int k = (j - 1) * mi + (i - 1);
            double r = q ? AT(q, m, i, j) : 0.0;
            A[(size_t)k * N + k] = d;
            const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
            for (int t = 0; t < 4; ++t) {
                int ii = i + di[t], jj = j + dj[t];
                double wgt = t < 2 ? 1.0 : b2;
                if (ii >= 1 && ii <= mi && jj >= 1 && jj <= ni)
                    A[(size_t)k * N + (size_t)((jj - 1) * mi + (ii - 1))] = -wgt;
                else
                    r += wgt * AT(u, m, ii, jj);
            }
            rhs[k] = r;
        }
    for (int col = 0; col < N; ++col) {
        int piv = col;
        for (int row = col + 1; row < N; ++row)
            if (fabs(A[(size_t)row * N + col]) > fabs(A[(size_t)piv * N + col])) piv = row;
        if (piv != col) {
            for (int t = 0; t < N; ++t) {
                double tmp = A[(size_t)col * N + t];
                A[(size_t)col * N + t] = A[(size_t)piv * N + t];
                A[(size_t)piv * N + t] = tmp;
            }
            double tmp = rhs[col]; rhs[col] = rhs[piv]; rhs[piv] = tmp;
        }
        for (int row = col + 1; row < N; ++row) {
            double f = A[(size_t)row * N + col] / A[(size_t)col * N + col];
            if (f == 0.0) continue;
            for (int t = col; t < N; ++t) A[(size_t)row * N + t] -= f * A[(size_t)col * N + t];
            rhs[row] -= f * rhs[col];
        }
    }
    for (int row = N - 1; row >= 0; --row) {
        double s = rhs[row];
        for (int t = row + 1; t < N; ++t) s -= A[(size_t)row * N + t] * rhs[t];
        rhs[row] = s / A[(size_t)row * N + row];
    }
    for (int j = 1; j <= ni; ++j)
        for (int i = 1; i <= mi; ++i) AT(u, m, i, j) = rhs[(j - 1) * mi + (i - 1)];
    free(A);
    free(rhs);
    return 0;
}

/* V-cycle step 7 as printed: Gauss-Seidel "till convergence", i.e. until a sweep
 * leaves every value unchanged (or a generous cap is hit). */
static void coarse_gs(int m, int n, double beta, int ordering, double* u, const double* q)
{
    size_t sz = (size_t)m * (size_t)n;
    double* prev = (double*)malloc(sizeof(double) * sz);
    for (int s = 0; s < 1000000; ++s) {
        memcpy(prev, u, sizeof(double) * sz);
        ora_gs_sweep(m, n, beta, ordering, u, q);
        double change = 0.0, big = 0.0;
        for (size_t k = 0; k < sz; ++k) {
            change = fmax(change, fabs(u[k] - prev[k]));
            big = fmax(big, fabs(u[k]));
        }
        if (change <= 1e-16 * big) break;
    }
    free(prev);
}

int ora_mg_levels(int m, int n, int coarsest_min, int max_levels)
{
    if (coarsest_min < 3) coarsest_min = 3;
    int levels = 1;
    while ((max_levels <= 0 || levels < max_levels) && (m - 1) % 2 == 0 && (n - 1) % 2 == 0 &&
           (m - 1) / 2 + 1 >= coarsest_min && (n - 1) / 2 + 1 >= coarsest_min) {
        m = (m - 1) / 2 + 1;
        n = (n - 1) / 2 + 1;
        ++levels;
    }
    return levels;
}

typedef struct { int m, n; double *u, *q, *r; } level;

static void smooth(level* L, const double* q, double beta, const ora_params* p)
{
    if (p->w == 1.0)
        ora_gs_sweep(L->m, L->n, beta, p->ordering, L->u, q);
    else
        ora_sor_sweep(L->m, L->n, beta, p->w, p->ordering, L->u, q);
}

/* The 11 steps of the V-cycle ("Multigrid Method (V-Cycle)"), for any number of
 * levels: smooth nu1 times, restrict the residual, solve the coarse correction
 * equation recursively (exactly on the coarsest level), interpolate and add the
 * correction, smooth nu2 times. Level 0 is the Laplace problem itself (q = 0);
 * deeper levels carry the correction with a zero ring and zero initial guess. */
static int vcycle(level* lv, int l, int nl, double beta, const ora_params* p)
{
    level* L = &lv[l];
    const double* q = l == 0 ? NULL : L->q;
    if (l == nl - 1) {
        if (p->coarse == ORA_COARSE_GS) {
            coarse_gs(L->m, L->n, beta, p->ordering, L->u, q);
            return 0;
        }
        return ora_coarse_direct(L->m, L->n, beta, L->u, q);
    }
    for (int s = 0; s < p->nu1; ++s) smooth(L, q, beta, p);
    ora_defect(L->m, L->n, beta, L->u, q, L->r);
    level* C = &lv[l + 1];
    ora_restrict_fw(L->m, L->n, L->r, C->q);
    memset(C->u, 0, sizeof(double) * (size_t)C->m * (size_t)C->n);
    int rc = vcycle(lv, l + 1, nl, beta, p);
    if (rc) return rc;
    ora_prolong_add(C->m, C->n, C->u, L->m, L->n, L->u);
    for (int s = 0; s < p->nu2; ++s) smooth(L, q, beta, p);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Solver loop: iterate until the stopping rule holds (Eq. 16 for MAXDELTA, or the
 * L2 norm of the residual of Eq. 12) or max_iter is reached. */
int ora_solve(int m, int n, double dx, double dy, double* psi, const ora_params* p, long* iters,
              double* r0, double* rfinal, double* hist, long hist_len)
{
    if (m < 3 || n < 3 || !(dx > 0.0) || !(dy > 0.0) || !p || p->check_every < 1 ||
        p->max_iter < 0 || !(p->tol >= 0.0))
        return -1;
    if (p->method < ORA_JACOBI || p->method > ORA_MG) return -1;
    if (p->sum_order != ORA_SUM_PAPER && p->sum_order != ORA_SUM_DIAGONAL) return -1;
    if (p->sum_order == ORA_SUM_DIAGONAL &&
        ((p->method != ORA_GS && p->method != ORA_SOR) || dx != dy))
        return -1;
    double beta = dx / dy;
    size_t sz = (size_t)m * (size_t)n;
    double* prev = (double*)malloc(sizeof(double) * sz);
    double* tmp = (double*)malloc(sizeof(double) * sz);
    level* lv = NULL;
    int nl = 0;
    if (p->method == ORA_MG) {
        nl = ora_mg_levels(m, n, p->coarsest_min, p->max_levels);
        lv = (level*)calloc((size_t)nl, sizeof(level));
        int mm = m, nn = n;
        for (int l = 0; l < nl; ++l) {
            lv[l].m = mm;
            lv[l].n = nn;
            size_t s = (size_t)mm * (size_t)nn;
            lv[l].u = l == 0 ? psi : (double*)calloc(s, sizeof(double));
            lv[l].q = (double*)calloc(s, sizeof(double));
            lv[l].r = (double*)calloc(s, sizeof(double));
            mm = (mm - 1) / 2 + 1;
            nn = (nn - 1) / 2 + 1;
        }
    }
    double nr0 = ora_defect_norm_l2(m, n, beta, psi, NULL);
    *r0 = nr0;
    int status = 1;
    long k = 0;
    if ((p->norm == ORA_NORM_L2_REL && nr0 == 0.0) ||
        (p->norm == ORA_NORM_L2_ABS && nr0 <= p->tol))
        status = 0;
    long nh = 0;
    while (status == 1 && k < p->max_iter) {
        ++k;
        int check = (k % p->check_every) == 0 || k == p->max_iter;
        if (check && p->norm == ORA_NORM_MAXDELTA) memcpy(prev, psi, sizeof(double) * sz);
        switch (p->method) {
        case ORA_JACOBI:
            ora_jacobi_sweep(m, n, beta, psi, tmp);
            memcpy(psi, tmp, sizeof(double) * sz);
            break;
        case ORA_GS: ora_gs_sweep_ordered(m, n, beta, p->ordering, p->sum_order, psi, NULL); break;
        case ORA_SOR:
            ora_sor_sweep_ordered(m, n, beta, p->w, p->ordering, p->sum_order, psi, NULL);
            break;
        case ORA_SLOR: ora_line_sweep(m, n, beta, p->w, p->form, 0, p->line_order, psi); break;
        case ORA_ADI: ora_adi_iteration(m, n, beta, p->w, p->form, p->line_order, psi); break;
        case ORA_MG:
            if (vcycle(lv, 0, nl, beta, p)) { status = -2; goto done; }
            break;
        }
        if (!check) continue;
        double val;
        int conv;
        if (p->norm == ORA_NORM_MAXDELTA) {
            val = 0.0;
            for (size_t t = 0; t < sz; ++t) {
                double dlt = fabs(psi[t] - prev[t]);
                if (isnan(dlt)) { val = dlt; break; } /* a NaN anywhere is divergence */
                if (dlt > val) val = dlt;
            }
            conv = val <= p->tol;
        } else {
            double nr = ora_defect_norm_l2(m, n, beta, psi, NULL);
            val = p->norm == ORA_NORM_L2_REL ? nr / nr0 : nr;
            conv = p->norm == ORA_NORM_L2_REL ? nr <= p->tol * nr0 : nr <= p->tol;
        }
        if (hist && nh < hist_len) hist[nh++] = val;
        if (!isfinite(val)) status = 2;
        else if (conv) status = 0;
    }
done:
    *iters = k;
    *rfinal = ora_defect_norm_l2(m, n, beta, psi, NULL);
    if (lv) {
        for (int l = 0; l < nl; ++l) {
            if (l > 0) free(lv[l].u);
            free(lv[l].q);
            free(lv[l].r);
        }
        free(lv);
    }
    free(prev);
    free(tmp);
    return status;
}
