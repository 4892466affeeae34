/*
 * FP64 CPU oracle for the dense Kohn-Sham solver path (Cholesky -> standard form ->
 * eigendecomposition -> back-substitution -> occupation -> density matrices).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, loads or calls this
 * file; only the tests, the package's smoke check and the benchmark's CPU-baseline leg
 * use it. It shares no code, header or constant with the CUDA implementation.
 *
 * Every routine is the plain textbook definition written out in binary64, column-major
 * storage (element (i,j) of an n-by-n matrix at a[i + j*n]), with no blocking. The
 * eigendecomposition of the standard-form matrix is cyclic Jacobi (Jacobi 1846, in the
 * form given by Golub & Van Loan, "Matrix Computations", sec. 8.5) with the round-robin
 * ordering of Brent & Luk (1985), so the n/2 rotations of one round are independent.
 * The method of the paper (two-stage tridiagonalisation) reaches the same eigenpairs up
 * to rounding, so the oracle uses the simplest correct algorithm instead.
 *
 * Citations refer to Yu et al., "ELSI: A Unified Software Interface for Kohn-Sham
 * Electronic Structure Solvers" (arXiv:1705.11191).
 *
 * Pins (tests/test_oracle_pins.py): tight-binding chain closed form, commuting
 * generalized chain closed form, 2x2 quadratic, brute force against LAPACK on small
 * cases, and the invariants Tr(PS)=N_el, PSP=2P, Tr(PH)=Tr(WS)=sum f*eps.
 */
#define _DEFAULT_SOURCE
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define A_(a, n, i, j) ((a)[(size_t)(i) + (size_t)(j) * (size_t)(n)])

/* ------------------------------------------------------------------------------------
 * Cholesky factorisation S = L L^T (Eq. 8, "eq:cholesky", sec. 3.1).
 * Plain left-looking column algorithm. L is written to l (lower triangle, zeros above).
 * Returns 0 on success, or j+1 when the j-th pivot is not positive (S not positive
 * definite in working precision).
 * ---------------------------------------------------------------------------------- */
int orc_cholesky(int n, const double *s, double *l)
{
    memset(l, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int j = 0; j < n; ++j) {
        double d = A_(s, n, j, j);
        for (int k = 0; k < j; ++k) d -= A_(l, n, j, k) * A_(l, n, j, k);
        if (!(d > 0.0)) return j + 1;
        double ljj = sqrt(d);
        A_(l, n, j, j) = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A_(s, n, i, j);
            for (int k = 0; k < j; ++k) v -= A_(l, n, i, k) * A_(l, n, j, k);
            A_(l, n, i, j) = v / ljj;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Standard form H~ = L^{-1} H L^{-T} (Eq. 9, "eq:after_cholesky", sec. 3.1).
 * Step 1: Y = L^{-1} H by forward substitution on every column of H.
 * Step 2: H~ = L^{-1} Y^T (H~ is symmetric, so H~ = (Y L^{-T})^T = L^{-1} Y^T).
 * The result is symmetrised, (X + X^T)/2, to remove rounding asymmetry.
 * ---------------------------------------------------------------------------------- */
static void forward_subst_cols(int n, const double *l, double *b)
{
    /* Solve L x = b for every column of b, in place. */
#pragma omp parallel for schedule(static)
    for (int c = 0; c < n; ++c) {
        double *x = b + (size_t)c * (size_t)n;
        for (int i = 0; i < n; ++i) {
            double v = x[i];
            for (int k = 0; k < i; ++k) v -= A_(l, n, i, k) * x[k];
            x[i] = v / A_(l, n, i, i);
        }
    }
}

void orc_standard_form(int n, const double *h, const double *l, double *ht)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    memcpy(y, h, sizeof(double) * (size_t)n * (size_t)n);
    forward_subst_cols(n, l, y); /* y = L^{-1} H */
    for (int j = 0; j < n; ++j)  /* ht = y^T */
        for (int i = 0; i < n; ++i) A_(ht, n, i, j) = A_(y, n, j, i);
    forward_subst_cols(n, l, ht); /* ht = L^{-1} y^T */
    for (int j = 0; j < n; ++j)
        for (int i = j + 1; i < n; ++i) {
            double m = 0.5 * (A_(ht, n, i, j) + A_(ht, n, j, i));
            A_(ht, n, i, j) = m;
            A_(ht, n, j, i) = m;
        }
    free(y);
}

/* ------------------------------------------------------------------------------------
 * Cyclic Jacobi eigendecomposition of a symmetric matrix A (n x n, overwritten).
 * On return w[i] = A[i,i] (eigenvalues, unsorted) and V holds the eigenvectors as
 * columns. One sweep = n-1 rounds (n even; odd n gets a dummy index) of the round-robin
 * tournament; in each round every pair (p,q) gets one rotation J_pq chosen so that
 * (J^T A J)_pq = 0:
 *     theta = (a_qq - a_pp) / (2 a_pq),  t = sign(theta) / (|theta| + sqrt(1+theta^2)),
 *     c = 1/sqrt(1+t^2),  s = t c.
 * The rotations of one round act on disjoint index pairs, so they are all computed
 * from the same A and applied together: A <- J^T A J, V <- V J.
 * A rotation is skipped when a_pq is negligible: |a_pq| <= 8 eps sqrt(|a_pp a_qq|)
 * (the relative criterion of Demmel & Veselic 1992) or |a_pq| <= 2 eps ||A||_F / sqrt(n).
 * Returns the number of sweeps used, or -1 if max_sweeps passed without convergence.
 * ---------------------------------------------------------------------------------- */
int orc_jacobi(int n, double *a, double *w, double *v, int max_sweeps)
{
    const double eps = 2.220446049250313e-16;
    memset(v, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i = 0; i < n; ++i) A_(v, n, i, i) = 1.0;
    if (n == 1) { w[0] = a[0]; return 0; }

    double fro = 0.0;
    for (size_t i = 0; i < (size_t)n * (size_t)n; ++i) fro += a[i] * a[i];
    fro = sqrt(fro);
    /* entries below the rounding level of the whole matrix (a few eps ||A||_F per row)
     * cannot be reduced by a rotation either; this matters for (near-)zero eigenvalues */
    const double abs_tol = 2.0 * eps * fro / sqrt((double)n);
    /* A rotation on a pair whose off-diagonal entry is already at the rounding level of
     * its diagonal entries cannot reduce it further; with exactly degenerate eigenvalues
     * (the real form of a complex Hermitian matrix has every eigenvalue twice) such
     * rotations would repeat forever. The skip rule therefore allows 8 eps. */
    const double rel_tol = 8.0 * eps;

    const int m = (n % 2) ? n + 1 : n; /* tournament size, one dummy player if n odd */
    int *pp = (int *)malloc(sizeof(int) * (size_t)(m / 2));
    int *qq = (int *)malloc(sizeof(int) * (size_t)(m / 2));
    double *cs = (double *)malloc(sizeof(double) * (size_t)(m / 2));
    double *sn = (double *)malloc(sizeof(double) * (size_t)(m / 2));
    int *ring = (int *)malloc(sizeof(int) * (size_t)m);

    int sweep;
    for (sweep = 1; sweep <= max_sweeps; ++sweep) {
        long rotations = 0;
        for (int i = 0; i < m; ++i) ring[i] = i;
        for (int round = 0; round < m - 1; ++round) {
            /* pairs of this round: ring[i] vs ring[m-1-i] */
            int np = 0;
            for (int i = 0; i < m / 2; ++i) {
                int p = ring[i], q = ring[m - 1 - i];
                if (p > q) { int t = p; p = q; q = t; }
                if (q >= n) continue; /* dummy player */
                double apq = A_(a, n, p, q);
                double app = A_(a, n, p, p), aqq = A_(a, n, q, q);
                if (fabs(apq) <= abs_tol || fabs(apq) <= rel_tol * sqrt(fabs(app * aqq))) continue;
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                double c = 1.0 / sqrt(1.0 + t * t);
                pp[np] = p; qq[np] = q; cs[np] = c; sn[np] = t * c; ++np;
            }
            rotations += np;
            /* A <- A J (columns p, q of every pair) and V <- V J */
#pragma omp parallel for schedule(static)
            for (int r = 0; r < np; ++r) {
                int p = pp[r], q = qq[r];
                double c = cs[r], s = sn[r];
                double *ap = a + (size_t)p * n, *aq = a + (size_t)q * n;
                double *vp = v + (size_t)p * n, *vq = v + (size_t)q * n;
                for (int i = 0; i < n; ++i) {
                    double x = ap[i], y = aq[i];
                    ap[i] = c * x - s * y;
                    aq[i] = s * x + c * y;
                    double xv = vp[i], yv = vq[i];
                    vp[i] = c * xv - s * yv;
                    vq[i] = s * xv + c * yv;
                }
            }
            /* A <- J^T A (rows p, q of every pair) */
#pragma omp parallel for schedule(static)
            for (int j = 0; j < n; ++j) {
                double *col = a + (size_t)j * n;
                for (int r = 0; r < np; ++r) {
                    int p = pp[r], q = qq[r];
                    double c = cs[r], s = sn[r];
                    double x = col[p], y = col[q];
                    col[p] = c * x - s * y;
                    col[q] = s * x + c * y;
                }
            }
            /* rotate the tournament: ring[0] fixed, others shift by one */
            int last = ring[m - 1];
            for (int i = m - 1; i > 1; --i) ring[i] = ring[i - 1];
            ring[1] = last;
        }
        if (rotations == 0) break;
    }
    for (int i = 0; i < n; ++i) w[i] = A_(a, n, i, i);
    free(pp); free(qq); free(cs); free(sn); free(ring);
    return (sweep > max_sweeps) ? -1 : sweep;
}

/* ------------------------------------------------------------------------------------
 * Stable ascending sort of eigenpairs (eigenvalues "in ascending order", sec. 4.4,
 * elsi_ev_real). Insertion sort on an index array: ties keep their input order.
 * w (n) and the columns of v (n x n) are permuted together.
 * ---------------------------------------------------------------------------------- */
void orc_sort_eigenpairs(int n, double *w, double *v)
{
    int *idx = (int *)malloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 1; i < n; ++i) {
        int key = idx[i], j = i - 1;
        while (j >= 0 && w[idx[j]] > w[key]) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = key;
    }
    double *w2 = (double *)malloc(sizeof(double) * (size_t)n);
    double *v2 = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
    for (int j = 0; j < n; ++j) {
        w2[j] = w[idx[j]];
        memcpy(v2 + (size_t)j * n, v + (size_t)idx[j] * n, sizeof(double) * (size_t)n);
    }
    memcpy(w, w2, sizeof(double) * (size_t)n);
    memcpy(v, v2, sizeof(double) * (size_t)n * (size_t)n);
    free(idx); free(w2); free(v2);
}

/* ------------------------------------------------------------------------------------
 * Back-substitution c = L^{-T} c~ (Eq. 9: c~ = L^* c), for the first k columns of vt.
 * Plain backward substitution with L^T (upper triangular).
 * ---------------------------------------------------------------------------------- */
void orc_back_substitute(int n, int k, const double *l, const double *vt, double *c)
{
#pragma omp parallel for schedule(static)
    for (int col = 0; col < k; ++col) {
        const double *b = vt + (size_t)col * n;
        double *x = c + (size_t)col * n;
        for (int i = n - 1; i >= 0; --i) {
            double s = b[i];
            for (int r = i + 1; r < n; ++r) s -= A_(l, n, r, i) * x[r]; /* (L^T)_{i r} = L_{r i} */
            x[i] = s / A_(l, n, i, i);
        }
    }
}

/* ------------------------------------------------------------------------------------
 * Occupation numbers and chemical potential (sec. 4.4, elsi_dm_real; Eqs. 14-15 and
 * 17-18, "eq:fermi_dirac", "eq:n_electron", "eq:gaussian", "eq:erf").
 *
 * eps: the k lowest eigenvalues, ascending. Spin factor g = 2 (spin-unpolarised),
 * so each f lies in [0, 2]: f_l = g * phi((eps_l - mu)/kT).
 *   scheme 0: integer (aufbau) occupation: states filled in ascending order with g
 *             electrons each until n_el is reached (the last one may be partial).
 *   scheme 1: Gaussian broadening, phi(x) = (1 - erf(x))/2.
 *   scheme 2: Fermi-Dirac broadening, phi(x) = 1/(1 + e^x).
 * For schemes 1-2 mu is found by bisection: start from [eps_min, eps_max], widen by
 * 1 Ha at either end until N(lo) <= n_el <= N(hi), then halve until
 * |N(mid) - n_el| <= occ_accuracy, at most mu_max_steps halvings. If that is not met,
 * mu = hi is taken and the surplus N(hi) - n_el >= 0 is removed starting from the
 * highest occupied state downwards (each f clamped at 0), so sum f = n_el exactly.
 * Returns 0, or -1 for invalid arguments / an unreachable electron count.
 * ---------------------------------------------------------------------------------- */
/* Occupation fraction for x = (eps - mu) / kT. Schemes (sec. 4.5, broadening_scheme):
 * 1 Gaussian, 0.5 erfc(x); 2 Fermi-Dirac (Eq. 14); 3 Methfessel-Paxton of order 0 (the
 * Gaussian); 4 Methfessel-Paxton of order 1 (Methfessel & Paxton, Phys. Rev. B 40, 3616
 * (1989): S_N(x) = 0.5 erfc(x) + sum_{n=1..N} A_n H_{2n-1}(x) exp(-x^2),
 * A_n = (-1)^n / (n! 4^n sqrt(pi)), H the physicists' Hermite polynomials; for N = 1,
 * A_1 H_1(x) = -x / (2 sqrt(pi))). */
static double occ_phi(int scheme, double x)
{
    if (scheme == 1 || scheme == 3) return 0.5 * erfc(x);
    if (scheme == 4) return 0.5 * erfc(x) - x * exp(-x * x) / (2.0 * sqrt(M_PI));
    /* Fermi-Dirac in a form that does not overflow */
    if (x > 0.0) { double e = exp(-x); return e / (1.0 + e); }
    return 1.0 / (1.0 + exp(x));
}

static double occ_count(int k, const double *eps, int scheme, double kt, double mu, double g)
{
    double s = 0.0;
    for (int l = 0; l < k; ++l) s += g * occ_phi(scheme, (eps[l] - mu) / kt);
    return s;
}

int orc_occupation(int k, const double *eps, double n_el, int scheme, double kt,
                   double occ_accuracy, int mu_max_steps, double *f, double *mu_out)
{
    const double g = 2.0;
    if (k <= 0 || n_el < 0.0 || n_el > g * k) return -1;
    if (scheme == 0) {
        double left = n_el;
        for (int l = 0; l < k; ++l) {
            double take = left >= g ? g : (left > 0.0 ? left : 0.0);
            f[l] = take;
            left -= take;
        }
        /* mu reported as the highest (partially) occupied level */
        int top = 0;
        for (int l = 0; l < k; ++l) if (f[l] > 0.0) top = l;
        *mu_out = eps[top];
        return 0;
    }
    if (!(kt > 0.0) || scheme < 1 || scheme > 4) return -1;
    double lo = eps[0], hi = eps[k - 1];
    for (int it = 0; it < 1000 && occ_count(k, eps, scheme, kt, lo, g) > n_el; ++it) lo -= 1.0;
    for (int it = 0; it < 1000 && occ_count(k, eps, scheme, kt, hi, g) < n_el; ++it) hi += 1.0;
    double mu = hi;
    int converged = 0;
    for (int step = 0; step < mu_max_steps; ++step) {
        double mid = 0.5 * (lo + hi);
        double nm = occ_count(k, eps, scheme, kt, mid, g);
        if (fabs(nm - n_el) <= occ_accuracy) { mu = mid; converged = 1; break; }
        if (nm < n_el) lo = mid; else hi = mid;
    }
    if (!converged) mu = hi;
    for (int l = 0; l < k; ++l) f[l] = g * occ_phi(scheme, (eps[l] - mu) / kt);
    if (!converged) {
        double surplus = 0.0;
        for (int l = 0; l < k; ++l) surplus += f[l];
        surplus -= n_el;
        for (int l = k - 1; l >= 0 && surplus > 0.0; --l) {
            double take = f[l] < surplus ? f[l] : surplus;
            f[l] -= take;
            surplus -= take;
        }
    }
    *mu_out = mu;
    return 0;
}

/* ------------------------------------------------------------------------------------
 * One chemical potential for several problems (k-points and spin channels). Sec. 4.4
 * states that the electron count of the bisection is summed over k-points, spin
 * channels and states. Entry j (of m, in any order) has eigenvalue eps[j] and weight
 * wt[j] >= 0 (the weight of the problem it belongs to); the electron count is
 * sum_j wt[j] f_j with f_j in [0, g].
 *   Integer occupation: aufbau, levels in ascending order of eigenvalue; a level is the
 *   set of entries with exactly equal eigenvalues, and the top level shares the
 *   electrons left in proportion to the weights. mu = eigenvalue of the top level that
 *   receives electrons (the lowest eigenvalue when n_el = 0).
 *   Smeared occupation: bisection as in orc_occupation with the weighted count. When it
 *   stalls, mu = hi and the surplus is removed from the levels in descending order, a
 *   whole level at a time, the last one scaled by a common factor.
 * Returns 0, or -1 for invalid arguments.
 * ---------------------------------------------------------------------------------- */
static const double *g_sort_key;
static int cmp_by_key(const void *a, const void *b)
{
    int i = *(const int *)a, j = *(const int *)b;
    if (g_sort_key[i] < g_sort_key[j]) return -1;
    if (g_sort_key[i] > g_sort_key[j]) return 1;
    return (i > j) - (i < j);
}

static double wocc_count(int m, const double *eps, const double *wt, int scheme, double kt,
                         double mu, double g)
{
    double s = 0.0;
    for (int j = 0; j < m; ++j) s += wt[j] * g * occ_phi(scheme, (eps[j] - mu) / kt);
    return s;
}

int orc_occupation_weighted(int m, const double *eps, const double *wt, double n_el,
                            int scheme, double kt, double occ_accuracy, int mu_max_steps,
                            double *f, double *mu_out)
{
    const double g = 2.0;
    if (m <= 0 || n_el < 0.0) return -1;
    double wsum = 0.0;
    for (int j = 0; j < m; ++j) {
        if (!(wt[j] >= 0.0)) return -1;
        wsum += wt[j];
    }
    if (n_el > g * wsum * (1.0 + 1e-14)) return -1;
    int *ord = (int *)malloc(sizeof(int) * (size_t)m);
    for (int j = 0; j < m; ++j) ord[j] = j;
    g_sort_key = eps;
    qsort(ord, (size_t)m, sizeof(int), cmp_by_key); /* ascending eigenvalue */
    if (scheme == 0) {
        double left = n_el;
        double mu = eps[ord[0]];
        for (int a = 0; a < m;) {
            int b = a;
            double wl = 0.0;
            while (b < m && eps[ord[b]] == eps[ord[a]]) wl += wt[ord[b++]];
            double fl;
            if (left <= 0.0) fl = 0.0;
            else if (left >= g * wl) fl = g;
            else fl = left / wl;
            if (left > 0.0) mu = eps[ord[a]];
            for (int c = a; c < b; ++c) f[ord[c]] = fl;
            left -= fl * wl;
            a = b;
        }
        *mu_out = mu;
        free(ord);
        return 0;
    }
    if (!(kt > 0.0) || scheme < 1 || scheme > 4) { free(ord); return -1; }
    double lo = eps[ord[0]], hi = eps[ord[m - 1]];
    for (int it = 0; it < 1000 && wocc_count(m, eps, wt, scheme, kt, lo, g) > n_el; ++it) lo -= 1.0;
    for (int it = 0; it < 1000 && wocc_count(m, eps, wt, scheme, kt, hi, g) < n_el; ++it) hi += 1.0;
    double mu = hi;
    int converged = 0;
    for (int step = 0; step < mu_max_steps; ++step) {
        double mid = 0.5 * (lo + hi);
        double nm = wocc_count(m, eps, wt, scheme, kt, mid, g);
        if (fabs(nm - n_el) <= occ_accuracy) { mu = mid; converged = 1; break; }
        if (nm < n_el) lo = mid; else hi = mid;
    }
    if (!converged) mu = hi;
    for (int j = 0; j < m; ++j) f[j] = g * occ_phi(scheme, (eps[j] - mu) / kt);
    if (!converged) {
        double surplus = -n_el;
        for (int j = 0; j < m; ++j) surplus += wt[j] * f[j];
        double removed = 0.0;
        for (int b = m; b > 0 && surplus > 0.0;) {
            int a = b - 1;
            while (a > 0 && eps[ord[a - 1]] == eps[ord[b - 1]]) --a;
            double gl = 0.0;
            for (int c = a; c < b; ++c) gl += wt[ord[c]] * f[ord[c]];
            if (removed + gl >= surplus) {
                double keep = (gl > 0.0) ? 1.0 - (surplus - removed) / gl : 0.0;
                for (int c = a; c < b; ++c) f[ord[c]] *= keep;
                break;
            }
            for (int c = a; c < b; ++c) f[ord[c]] = 0.0;
            removed += gl;
            b = a;
        }
    }
    *mu_out = mu;
    free(ord);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Weighted outer-product sum D = sum_l w_l c_l c_l^T over the first k columns of c.
 * With w = f this is the density matrix (Eq. 7, "eq:density_matrix", sec. 2);
 * with w = f*eps it is the energy-weighted density matrix W.
 * Plain triple loop.
 * ---------------------------------------------------------------------------------- */
void orc_weighted_outer(int n, int k, const double *c, const double *w, double *d)
{
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += w[l] * A_(c, n, i, l) * A_(c, n, j, l);
            A_(d, n, i, j) = s;
        }
}

/* ------------------------------------------------------------------------------------
 * Full pipeline (sec. 3.1 and sec. 4.4): eigenvalues of (H, S) ascending (all n), the
 * first k eigenvectors (S-orthonormal), occupations, P, W and the band energy
 * E = sum_l f_l eps_l ("energy corresponding to the occupied eigenstates").
 * unit_ovlp != 0 skips the Cholesky (S = I, "overlap_is_unit", sec. 4.5).
 * Any of p, w_mat, f may be NULL to skip that output.
 * Returns 0; j+1 (>0) for a non-positive Cholesky pivot j; -1 Jacobi non-convergence;
 * -2 occupation failure.
 * ---------------------------------------------------------------------------------- */
int orc_solve(int n, int k, const double *h, const double *s, int unit_ovlp,
              double n_el, int scheme, double kt, double occ_accuracy, int mu_max_steps,
              double *eval, double *c, double *f, double *p, double *w_mat,
              double *energy, double *mu)
{
    size_t nn = (size_t)n * (size_t)n;
    double *l = (double *)malloc(sizeof(double) * nn);
    double *ht = (double *)malloc(sizeof(double) * nn);
    double *v = (double *)malloc(sizeof(double) * nn);
    int rc = 0;
    if (unit_ovlp) {
        memset(l, 0, sizeof(double) * nn);
        for (int i = 0; i < n; ++i) A_(l, n, i, i) = 1.0;
        for (size_t i = 0; i < nn; ++i) ht[i] = h[i];
        for (int j = 0; j < n; ++j)
            for (int i = j + 1; i < n; ++i) {
                double m = 0.5 * (A_(ht, n, i, j) + A_(ht, n, j, i));
                A_(ht, n, i, j) = m; A_(ht, n, j, i) = m;
            }
    } else {
        rc = orc_cholesky(n, s, l);
        if (rc) goto done;
        orc_standard_form(n, h, l, ht);
    }
    if (orc_jacobi(n, ht, eval, v, 60) < 0) { rc = -1; goto done; }
    orc_sort_eigenpairs(n, eval, v);
    orc_back_substitute(n, k, l, v, c);
    if (f || p || w_mat || energy) {
        double *ff = (double *)malloc(sizeof(double) * (size_t)k);
        double muv = 0.0;
        if (orc_occupation(k, eval, n_el, scheme, kt, occ_accuracy, mu_max_steps, ff, &muv)) {
            free(ff); rc = -2; goto done;
        }
        if (f) memcpy(f, ff, sizeof(double) * (size_t)k);
        if (mu) *mu = muv;
        double e = 0.0;
        for (int i = 0; i < k; ++i) e += ff[i] * eval[i];
        if (energy) *energy = e;
        if (p) orc_weighted_outer(n, k, c, ff, p);
        if (w_mat) {
            double *fe = (double *)malloc(sizeof(double) * (size_t)k);
            for (int i = 0; i < k; ++i) fe[i] = ff[i] * eval[i];
            orc_weighted_outer(n, k, c, fe, w_mat);
            free(fe);
        }
        free(ff);
    }
done:
    free(l); free(ht); free(v);
    return rc;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
