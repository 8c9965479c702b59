/*
 * pd_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for the
 * ground state of the general pairing Hamiltonian in the seniority-zero basis
 * (Liu & Qi, "PairDiag", Comput. Phys. Commun.).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code with the
 * CUDA path.  Its route: the basis in the order of Sec. 3.1 (ascending
 * integers, Table 1), generated by the textbook successor of k-subsets in
 * colexicographic order; binary search (Sec. 3.2)
 * to locate each scattered state, the explicit diagonal (Eq. "diagonal") and
 * off-diagonal elements (Sec. 3.3), Lanczos (Algorithm 2) with full
 * Gram-Schmidt reorthogonalisation and restart from the ground Ritz vector
 * (Sec. 3.4), and cyclic Jacobi for the small tridiagonal matrix.
 *
 * Conventions: bit p of a state is orbit p (orbit 0 = lowest bit); G is
 * Omega x Omega row-major, G[a*omega+b] = V_ab (real symmetric, Sec. 4.1);
 * indices are 0-based (the paper's are 1-based).
 *
 * The optional OpenMP pragma only distributes independent rows of H*x over
 * threads; every row is computed by the same serial code.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Eq. (extcmn): C(n,m) = n!/(m!(n-m)!) for n >= m >= 0, and 0 for n < m.
 * Built by Pascal's rule, which is exact in uint64 for n <= 63. */
uint64_t orc_binom(int n, int m)
{
    if (n < 0 || m < 0 || m > n || n > 63) return 0;
    uint64_t row[64];
    memset(row, 0, sizeof row);
    row[0] = 1;
    for (int i = 1; i <= n; ++i)
        for (int j = i; j >= 1; --j) row[j] += row[j - 1];
    return row[m];
}

/* Successor of a basis state: the next larger word with the same number of
 * set bits.  A state with N pairs is the subset {c_1 < c_2 < ... < c_N} of its
 * occupied orbits, and ascending integer order (Sec. 3.1, Table 1) is the
 * colexicographic order of these subsets.  Its successor is the textbook rule
 * for stepping through combinations in that order (D. E. Knuth, The Art of
 * Computer Programming, Vol. 4A, Sec. 7.2.1.3, Algorithm L, "lexicographic
 * combinations" of the reversed sequence c_N ... c_1): take the smallest j
 * for which c_j + 1 is not c_{j+1} (with c_{N+1} taken as 64, above every
 * orbit), raise c_j by one and put c_1 .. c_{j-1} back at 0 .. j-2.
 * Returns 0 when no successor fits in 64 bits (and for s = 0). */
uint64_t orc_next_state(uint64_t s)
{
    int c[65];
    int n = 0;
    for (int p = 0; p < 64; ++p)        /* the occupied orbits, ascending */
        if (s >> p & 1ull) c[n++] = p;
    if (n == 0) return 0;
    c[n] = 64;
    int j = 0;
    while (j < n && c[j] + 1 == c[j + 1]) ++j;
    if (c[j] + 1 >= 64) return 0;       /* the last word of 64-bit states */
    c[j] += 1;
    for (int i = 0; i < j; ++i) c[i] = i;
    uint64_t t = 0;
    for (int i = 0; i < n; ++i) t |= 1ull << c[i];
    return t;
}

/* Sec. 3.1: the basis is every Omega-bit word with N set bits, in ascending
 * order, produced by the successor above from the minimum 2^N-1 up to the maximum
 * (2^N-1) << (Omega-N).  Returns the number written (C(Omega,N)). */
int64_t orc_build_basis(int omega, int n, uint64_t *out)
{
    if (omega < 1 || omega > 62 || n < 0 || n > omega) return -1;
    uint64_t lo = (n == 0) ? 0ull : ((1ull << n) - 1ull);
    uint64_t hi = lo << (omega - n);
    int64_t count = 0, cap = (int64_t)orc_binom(omega, n);
    uint64_t s = lo;
    for (;;) {
        out[count++] = s;
        if (s == hi) break;
        if (count == cap) return -3;    /* the walk overran C(Omega,N): inconsistent */
        s = orc_next_state(s);
    }
    return count;
}

/* Sec. 3.2: binary search of a state in the ascending basis; -1 if absent. */
int64_t orc_search(const uint64_t *basis, int64_t dim, uint64_t s)
{
    int64_t lo = 0, hi = dim - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (basis[mid] == s) return mid;
        if (basis[mid] < s) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* Sec. 3.2 hash: f = 1 + sum_j C(O_j - 1, j), O_j the 1-based orbit number of
 * the j-th occupied orbit (counting from the lowest bit).  Returns f (1-based). */
uint64_t orc_hash(uint64_t s)
{
    uint64_t f = 1;
    int j = 0;
    for (int p = 0; p < 64; ++p) {
        if (s >> p & 1ull) {
            ++j;
            int O = p + 1;
            f += orc_binom(O - 1, j);
        }
    }
    return f;
}

/* Eq. (diagonal): H_ii = sum over occupied orbits p of (2 e_p + V_pp). */
double orc_diag(uint64_t s, int omega, const double *e, const double *G)
{
    double d = 0.0;
    for (int p = 0; p < omega; ++p)
        if (s >> p & 1ull) d += 2.0 * e[p] + G[p * omega + p];
    return d;
}

/* Sec. 3.3: y = H x computed on the fly.  For every basis state |i> and every
 * pair (O occupied, E empty), |j> = S+_E S-_O |i> is located by binary search
 * and contributes <i|H|j> = V_EO x_j; the diagonal follows Eq. (diagonal). */
void orc_hx(int omega, const double *e, const double *G, const uint64_t *basis,
            int64_t dim, const double *x, double *y)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < dim; ++i) {
        uint64_t s = basis[i];
        double acc = orc_diag(s, omega, e, G) * x[i];
        for (int o = 0; o < omega; ++o) {
            if (!(s >> o & 1ull)) continue;
            for (int q = 0; q < omega; ++q) {
                if (s >> q & 1ull) continue;
                uint64_t t = (s & ~(1ull << o)) | (1ull << q);
                int64_t j = orc_search(basis, dim, t);
                acc += G[q * omega + o] * x[j];
            }
        }
        y[i] = acc;
    }
}

/* H*x on a truncated space (Sec. 3.5).  basis lists the kept states in
 * ascending order; a scattered state missing from it is dropped, so the
 * operator is the principal submatrix of H on the kept states.  Each kept
 * target is located by binary search, as the paper does once the space is no
 * longer complete. */
void orc_hx_sub(int omega, const double *e, const double *G, const uint64_t *basis,
                int64_t dim, const double *x, double *y)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < dim; ++i) {
        uint64_t s = basis[i];
        double acc = orc_diag(s, omega, e, G) * x[i];
        for (int o = 0; o < omega; ++o) {
            if (!(s >> o & 1ull)) continue;
            for (int q = 0; q < omega; ++q) {
                if (s >> q & 1ull) continue;
                uint64_t t = (s & ~(1ull << o)) | (1ull << q);
                int64_t j = orc_search(basis, dim, t);
                if (j < 0) continue;                 /* excluded by the truncation */
                acc += G[q * omega + o] * x[j];
            }
        }
        y[i] = acc;
    }
}

/* The same product restricted to selected rows: y[r] = (H x)[rows[r]]. */
void orc_hx_rows(int omega, const double *e, const double *G, const uint64_t *basis,
                 int64_t dim, const double *x, const int64_t *rows, int64_t nrows,
                 double *y)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        uint64_t s = basis[i];
        double acc = orc_diag(s, omega, e, G) * x[i];
        for (int o = 0; o < omega; ++o) {
            if (!(s >> o & 1ull)) continue;
            for (int q = 0; q < omega; ++q) {
                if (s >> q & 1ull) continue;
                uint64_t t = (s & ~(1ull << o)) | (1ull << q);
                int64_t j = orc_search(basis, dim, t);
                acc += G[q * omega + o] * x[j];
            }
        }
        y[r] = acc;
    }
}

/* Monopole_Min / Monopole_Max / Posit_Min: extreme diagonal elements. */
void orc_monopole(int omega, const double *e, const double *G, const uint64_t *basis,
                  int64_t dim, double *dmin, double *dmax, int64_t *pos_min)
{
    double lo = INFINITY, hi = -INFINITY;
    int64_t pos = 0;
    for (int64_t i = 0; i < dim; ++i) {
        double d = orc_diag(basis[i], omega, e, G);
        if (d < lo) { lo = d; pos = i; }
        if (d > hi) hi = d;
    }
    *dmin = lo; *dmax = hi; *pos_min = pos;
}

/* Cyclic Jacobi eigen-decomposition of a dense symmetric n x n matrix
 * (row-major, overwritten).  Each rotation zeroes one off-diagonal pair
 * (p,q) with the stable tangent t = sgn(tau)/(|tau| + sqrt(1+tau^2)),
 * tau = (a_qq - a_pp)/(2 a_pq).  On return w holds the eigenvalues and the
 * columns of V (row-major n x n) the eigenvectors. */
void orc_jacobi(int n, double *A, double *w, double *V)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double a2 = A[i * n + j] * A[i * n + j];
                tot += a2;
                if (i != j) off += a2;
            }
        if (off == 0.0 || off <= 1e-32 * tot) break;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                /* A <- J^T A J with J the rotation in the (p,q) plane */
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

static double dotp(const double *a, const double *b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Lowest eigenpair of T = tridiag(beta, alpha, beta) of size m via Jacobi. */
static void tridiag_ground(int m, const double *alpha, const double *beta,
                           double *theta, double *svec, double *theta2)
{
    double *A = calloc((size_t)m * m, sizeof(double));
    double *V = malloc((size_t)m * m * sizeof(double));
    double *w = malloc((size_t)m * sizeof(double));
    for (int i = 0; i < m; ++i) {
        A[i * m + i] = alpha[i];
        if (i + 1 < m) A[i * m + i + 1] = A[(i + 1) * m + i] = beta[i];
    }
    orc_jacobi(m, A, w, V);
    int k = 0;
    for (int i = 1; i < m; ++i) if (w[i] < w[k]) k = i;
    double second = INFINITY;
    for (int i = 0; i < m; ++i) if (i != k && w[i] < second) second = w[i];
    *theta = w[k];
    *theta2 = second;
    for (int i = 0; i < m; ++i) svec[i] = V[i * m + k];
    free(A); free(V); free(w);
}

/*
 * Restarted Lanczos for the lowest eigenpair (Algorithm 2 and Sec. 3.4).
 *
 * Each cycle starts from q_1 = v/||v|| and runs up to m = min(window, dim)
 * steps of Algorithm 2; after each step the new vector is orthogonalised
 * against every stored Lanczos vector by classical Gram-Schmidt, twice.  The
 * lowest Ritz pair of the tridiagonal L comes from Jacobi; the cycle restarts
 * from the ground Ritz vector.  Convergence (Sec. 5.1): at the first step of a
 * cycle, alpha_1 is the Rayleigh quotient of the restart vector and beta_1 the
 * norm of its residual; the solve stops once |beta_1/alpha_1| <= tol.
 * A step whose beta is below 1e-13 times the running size of L ends the
 * cycle early (an invariant subspace has been found).
 *
 * mode 0 = restarted; mode 1 = a single Krylov space without restart (the
 * Ritz value is returned, and rel_res reports its residual).
 *
 * v: in = start vector (dim), out = normalised ground-state vector.
 * Returns 0 on convergence, 1 if max_restarts was reached, <0 on bad input.
 */
int orc_lanczos_ground(int omega, int n, const double *e, const double *G,
                       int window, double tol, int max_restarts, int mode,
                       double *v, double *e0, int *iters_out, int *restarts_out,
                       double *rel_res_out, double *gap_out)
{
    if (omega < 1 || omega > 62 || n < 0 || n > omega || window < 1) return -1;
    int64_t dim = (int64_t)orc_binom(omega, n);
    uint64_t *basis = malloc((size_t)dim * sizeof(uint64_t));
    if (orc_build_basis(omega, n, basis) != dim) { free(basis); return -2; }
    int m = window < dim ? window : (int)dim;
    double *Q = malloc((size_t)m * dim * sizeof(double));
    double *p = malloc((size_t)dim * sizeof(double));
    double *alpha = malloc((size_t)m * sizeof(double));
    double *beta = malloc((size_t)m * sizeof(double));
    double *svec = malloc((size_t)m * sizeof(double));
    int iters = 0, restarts = 0, status = 1;
    double theta = 0.0, theta2 = INFINITY, rel = INFINITY;

    for (int cycle = 0; cycle <= max_restarts; ++cycle) {
        double nv = sqrt(dotp(v, v, dim));
        for (int64_t k = 0; k < dim; ++k) Q[k] = v[k] / nv;
        int used = 0;
        double tnorm = 0.0;
        for (int i = 0; i < m; ++i) {
            double *qi = Q + (int64_t)i * dim;
            orc_hx(omega, e, G, basis, dim, qi, p);
            ++iters;
            alpha[i] = dotp(qi, p, dim);
            for (int64_t k = 0; k < dim; ++k) {
                p[k] -= alpha[i] * qi[k];
                if (i > 0) p[k] -= beta[i - 1] * Q[(int64_t)(i - 1) * dim + k];
            }
            if (i == 0) {
                /* Sec. 5.1 convergence measure for the restart vector */
                double b1 = sqrt(dotp(p, p, dim));
                rel = (b1 == 0.0) ? 0.0 : b1 / fabs(alpha[0]);
                theta = alpha[0];
                if (mode == 0 && rel <= tol) { status = 0; used = 0; break; }
            }
            for (int pass = 0; pass < 2; ++pass)
                for (int j = 0; j <= i; ++j) {
                    double *qj = Q + (int64_t)j * dim;
                    double c = dotp(qj, p, dim);
                    for (int64_t k = 0; k < dim; ++k) p[k] -= c * qj[k];
                }
            beta[i] = sqrt(dotp(p, p, dim));
            used = i + 1;
            double rowsz = fabs(alpha[i]) + beta[i] + (i > 0 ? beta[i - 1] : 0.0);
            if (rowsz > tnorm) tnorm = rowsz;
            if (i + 1 == m || beta[i] <= 1e-13 * tnorm) break;
            double *qn = Q + (int64_t)(i + 1) * dim;
            for (int64_t k = 0; k < dim; ++k) qn[k] = p[k] / beta[i];
        }
        if (status == 0) {             /* converged: v = q_1 */
            for (int64_t k = 0; k < dim; ++k) v[k] = Q[k];
            break;
        }
        tridiag_ground(used, alpha, beta, &theta, svec, &theta2);
        for (int64_t k = 0; k < dim; ++k) {
            double s = 0.0;
            for (int j = 0; j < used; ++j) s += svec[j] * Q[(int64_t)j * dim + k];
            v[k] = s;
        }
        if (mode == 1) {               /* Mode = 1: return this Krylov space's ground state */
            double nn = sqrt(dotp(v, v, dim));
            for (int64_t k = 0; k < dim; ++k) v[k] /= nn;
            orc_hx(omega, e, G, basis, dim, v, p);
            double r2 = 0.0;
            for (int64_t k = 0; k < dim; ++k) { double d = p[k] - theta * v[k]; r2 += d * d; }
            rel = sqrt(r2) / fabs(theta);
            status = 0;
            break;
        }
        if (cycle < max_restarts) ++restarts;
    }
    *e0 = theta;
    *iters_out = iters;
    *restarts_out = restarts;
    *rel_res_out = rel;
    *gap_out = theta2 - theta;
    free(basis); free(Q); free(p); free(alpha); free(beta); free(svec);
    return status;
}
