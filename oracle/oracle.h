/*
 * oracle.h -- plain, slow FP64 CPU reference for the 2D Laplace solvers compared
 * in "A Comparison of SOR, ADI and Multigrid Methods for Solving Partial
 * Differential Equations" (arXiv 2208.02427).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load or call this library. It shares no code, header,
 * table or helper with the CUDA path, and it is never a fallback for it.
 *
 * Layout: a field is a dense row-major array psi[j*m + i]; i = 0..m-1 runs along
 * x (contiguous), j = 0..n-1 along y. The outer ring holds Dirichlet data and is
 * never written by any routine here. beta = dx/dy, b2 = beta*beta,
 * d = 2(1 + b2) (the diagonal of Eq. 5).
 */
#ifndef LAPLACE_ORACLE_H
#define LAPLACE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* point-iteration orderings */
enum { ORA_LEX = 0,   /* j outer, i inner, both ascending (Eq. 6 as printed) */
       ORA_RB = 1 };  /* red (i+j even) then black (i+j odd) */

/* line orderings */
enum { ORA_LINES_SUCCESSIVE = 0, /* lines 1,2,3,... (SLOR as printed) */
       ORA_LINES_ZEBRA = 1 };    /* odd lines first, then even lines */

/* line relaxation forms */
enum { ORA_FORM_A = 0,   /* SLORA: Thomas on Eq. 8, then relax with Eq. 9 */
       ORA_FORM_B = 1 }; /* SLORB: relaxation inside the line system, Eq. 10 */

/* methods for ora_solve */
enum { ORA_JACOBI = 0, ORA_GS = 1, ORA_SOR = 2, ORA_SLOR = 3, ORA_ADI = 4, ORA_MG = 5 };

/* stopping norms */
enum { ORA_NORM_L2_REL = 0,   /* ||r(psi^k)||_2 <= tol * ||r(psi^0)||_2 */
       ORA_NORM_L2_ABS = 1,   /* ||r(psi^k)||_2 <= tol */
       ORA_NORM_MAXDELTA = 2 };/* max |psi^k - psi^(k-1)| <= tol, Eq. 16 */

/* rounding order of the 4-term neighbour sum of Eqs. 5-7 (the paper writes the sum and fixes
 * no order; both orders are the same sum) */
enum { ORA_SUM_PAPER = 0,     /* (E + W) + beta^2 (N + S), as the equation is printed */
       ORA_SUM_DIAGONAL = 1 };/* (W + S) + (E + N), beta = 1 only */

/* coarsest-level solver for the V-cycle */
enum { ORA_COARSE_DIRECT = 0,   /* Gaussian elimination with partial pivoting */
       ORA_COARSE_GS = 1 };     /* Gauss-Seidel until the update stops changing */

typedef struct {
    int method;        /* ORA_JACOBI .. ORA_MG */
    int ordering;      /* ORA_LEX / ORA_RB for GS, SOR and the MG smoother */
    int line_order;    /* ORA_LINES_* for SLOR and ADI */
    int form;          /* ORA_FORM_A / ORA_FORM_B for SLOR and ADI */
    double w;          /* relaxation factor (SOR, SLOR, ADI; MG smoother) */
    int norm;          /* ORA_NORM_* */
    double tol;        /* stopping tolerance */
    long max_iter;     /* iteration (or V-cycle) cap */
    int check_every;   /* test the stopping rule every this many iterations (>=1) */
    int nu1, nu2;      /* MG pre/post smoothing sweeps */
    int coarsest_min;  /* MG: coarsen while both coarse sides stay >= this */
    int max_levels;    /* MG: 0 = as many as the sizes allow */
    int coarse;        /* ORA_COARSE_* */
    int sum_order;     /* ORA_SUM_* for the GS and SOR methods (beta = 1 for DIAGONAL) */
} ora_params;

/* ---- building blocks (each cites the passage it follows) ---- */

/* Scaled defect r = dx^2 * L(psi) (+ q), Eqs. 11-12, on interior nodes; 0 on the ring. */
void ora_defect(int m, int n, double beta, const double* psi, const double* q, double* r);
double ora_defect_norm_l2(int m, int n, double beta, const double* psi, const double* q);

/* One Jacobi sweep, Eq. 5, from `in` to `out` (ring copied). */
void ora_jacobi_sweep(int m, int n, double beta, const double* in, double* out);
/* One Gauss-Seidel sweep, Eq. 6 (with source q when non-NULL), in place. */
void ora_gs_sweep(int m, int n, double beta, int ordering, double* psi, const double* q);
/* One SOR sweep, Eq. 7 (with source q when non-NULL), in place. */
void ora_sor_sweep(int m, int n, double beta, double w, int ordering, double* psi, const double* q);
/* The same two sweeps with the neighbour sum in order sum_order (ORA_SUM_*; DIAGONAL needs
 * beta = 1 and returns -1 otherwise, leaving psi unchanged). */
int ora_gs_sweep_ordered(int m, int n, double beta, int ordering, int sum_order, double* psi,
                         const double* q);
int ora_sor_sweep_ordered(int m, int n, double beta, double w, int ordering, int sum_order,
                          double* psi, const double* q);

/* Thomas algorithm: a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i], i = 0..N-1. */
void ora_thomas(int N, const double* a, const double* b, const double* c, const double* d,
                double* x, double* cp, double* dp);
/* One sweep of line relaxation over all x-lines (rows, dir=0) or y-lines (columns,
 * dir=1), Eqs. 8-10, in the given line order and form. */
void ora_line_sweep(int m, int n, double beta, double w, int form, int dir, int line_order,
                    double* psi);
/* One ADI iteration: all x-lines, then all y-lines (ADI subsection). */
void ora_adi_iteration(int m, int n, double beta, double w, int form, int line_order, double* psi);

/* Multigrid transfer operators (V-cycle steps 3, 6, 8, 10). */
void ora_restrict_fw(int mf, int nf, const double* rf, double* qc);
void ora_prolong_add(int mc, int nc, const double* ec, int mf, int nf, double* uf);
/* Exact solve of the 5-point system (E+W) + b2 (N+S) - d u + q = 0 with the ring
 * of u as Dirichlet data (V-cycle step 7 solved to convergence). */
int ora_coarse_direct(int m, int n, double beta, double* u, const double* q);
/* Number of levels the V-cycle uses for an m x n grid. */
int ora_mg_levels(int m, int n, int coarsest_min, int max_levels);

/* ---- driver ---- */

/* Iterate `method` on psi (ring = Dirichlet data, interior = initial guess) until
 * the stopping rule holds or max_iter is reached. Returns 0 converged, 1 reached
 * max_iter, 2 non-finite, <0 argument error. *iters = iterations done; r0 / rfinal
 * = initial / final ||r||_2; hist (may be NULL, length hist_len) receives the
 * stopping-rule value after every checked iteration. */
int ora_solve(int m, int n, double dx, double dy, double* psi, const ora_params* p,
              long* iters, double* r0, double* rfinal, double* hist, long hist_len);

#ifdef __cplusplus
}
#endif
#endif
