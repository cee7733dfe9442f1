/*
 * oracle.c -- plain, slow, obviously-correct FP64 CPU reference for the hot
 * path of "Xabclib: A Fully Auto-tuned Sparse Iterative Solver" (Katagiri et
 * al.): CRS sparse matrix-vector multiply inside the restarted Krylov solvers
 * GMRES(m) and BiCGStab, the four re-orthogonalisations and the accuracy
 * policy that picks one (Sec. 3.2.2, 3.3.2), the restart-frequency rule (Eq. 1,
 * Fig. 2, Sec. 4.3), and the pieces the GPU library adds around them (FP32-inside-FP64 iterative
 * refinement, matrix features, and a small MLP with analytic gradients).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline / reference arm may load it.  The CUDA library
 * never calls it and shares no code, header, table or helper with it.
 *
 * Style rules followed throughout:
 *   - one loop per mathematical sum, ascending index order, no blocking,
 *     fusion or reordering beyond what the stated definition says;
 *   - FP64 everywhere except where a routine's whole point is FP32 arithmetic
 *     (the inner solve of the mixed-precision refinement), which says so;
 *   - CRS is 0-based: rowptr[n+1], col[nnz], val[nnz], columns ascending.
 *
 * Return codes match the library's meaning: 0 ok, -4 not converged within the
 * iteration limit, -5 numerical breakdown.
 *
 * Parity pins (which independent facts each routine is checked against) are
 * listed in the test files; every routine here has at least one.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The same source is also compiled with -fopenmp for the benchmark's
 * all-cores CPU baseline (the paper's row-parallel decomposition, U1 of
 * Sec. 3.2.2, run over the host's cores).  ORC_PAR marks the row loop of the
 * SpMV and the streaming vector loops of the solvers; ORC_PAR_SUM a dot
 * product.  Without -fopenmp both expand to nothing: the single-thread build
 * the tests check is exactly the plain loops.  In the OpenMP build the dot
 * products are summed in per-thread pieces, so its results differ by
 * rounding; it is used for timing only. */
#ifdef _OPENMP
#include <omp.h>
#define ORC_STR_(x) #x
#define ORC_PAR _Pragma("omp parallel for schedule(static)")
#define ORC_PAR_SUM(v) _Pragma(ORC_STR_(omp parallel for schedule(static) reduction(+:v)))
#else
#define ORC_PAR
#define ORC_PAR_SUM(v)
#endif

/* Threads the loops above use (1 in the single-thread build). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORC_OK 0
#define ORC_ENOCONV (-4)
#define ORC_EBREAKDOWN (-5)
#define ORC_EFAULT (-7)

/* ------------------------------------------------------------------------ */
/* Sparse matrix-vector products                                              */
/* ------------------------------------------------------------------------ */

/* General CRS SpMV, y = alpha*A*x + beta*y (Sec. 3.2.2; CRS format Sec. 4.2).
 * For each row i: s = sum over k in [rowptr[i], rowptr[i+1]) of val[k]*x[col[k]],
 * accumulated in ascending k.  beta == 0 means y is not read (BLAS rule). */
void orc_spmv(int n, const int *rowptr, const int *col, const double *val,
              double alpha, const double *x, double beta, double *y)
{
    ORC_PAR
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++)
            s += val[k] * x[col[k]];
        y[i] = (beta == 0.0) ? alpha * s : alpha * s + beta * y[i];
    }
}

/* Symmetric SpMV from upper-triangle storage (Sec. 4.2: "the lower part of the
 * matrix is not stored"; S1-S3 of Sec. 3.2.2).  Each stored (i, j, u) with
 * j >= i contributes u*x[j] to row i and, when j != i, u*x[i] to row j, i.e.
 * y = alpha*(U + U^T - diag(U))*x + beta*y. */
void orc_spmv_sym(int n, const int *rowptr, const int *col, const double *val,
                  double alpha, const double *x, double beta, double *y)
{
    double *t = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int i = 0; i < n; i++) {
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int j = col[k];
            t[i] += val[k] * x[j];
            if (j != i)
                t[j] += val[k] * x[i];
        }
    }
    for (int i = 0; i < n; i++)
        y[i] = (beta == 0.0) ? alpha * t[i] : alpha * t[i] + beta * y[i];
    free(t);
}

/* FP32 CRS SpMV with FP32 accumulation (the inner product of the mixed
 * precision refinement: matrix, vector and sum all single precision). */
void orc_spmv_f32(int n, const int *rowptr, const int *col, const float *val,
                  float alpha, const float *x, float beta, float *y)
{
    for (int i = 0; i < n; i++) {
        float s = 0.0f;
        for (int k = rowptr[i]; k < rowptr[i + 1]; k++)
            s += val[k] * x[col[k]];
        y[i] = (beta == 0.0f) ? alpha * s : alpha * s + beta * y[i];
    }
}

/* Dense y = A x, A row-major m x n.  Used only to pin the sparse routines. */
void orc_dense_matvec(int m, int n, const double *A, const double *x, double *y)
{
    for (int i = 0; i < m; i++) {
        double s = 0.0;
        for (int j = 0; j < n; j++)
            s += A[(size_t)i * n + j] * x[j];
        y[i] = s;
    }
}

/* Dense LU with partial pivoting, solves A z = b in place (A row-major n x n
 * is overwritten by its factors, b by z).  Returns 0, or -1 if a pivot is 0.
 * Textbook Gaussian elimination; used only to pin the Krylov solvers. */
int orc_lu_solve(int n, double *A, double *b)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++) {
            double v = fabs(A[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        if (best == 0.0)
            return -1;
        if (p != k) {
            for (int j = 0; j < n; j++) {
                double t = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)p * n + j];
                A[(size_t)p * n + j] = t;
            }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int i = k + 1; i < n; i++) {
            double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            A[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; j++)
                A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
            b[i] -= l * b[k];
        }
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = b[i];
        for (int j = i + 1; j < n; j++)
            s -= A[(size_t)i * n + j] * b[j];
        b[i] = s / A[(size_t)i * n + i];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Vector helpers (plain loops)                                              */
/* ------------------------------------------------------------------------ */

static double dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    ORC_PAR_SUM(s)
    for (int i = 0; i < n; i++)
        s += a[i] * b[i];
    return s;
}

static double nrm2(int n, const double *a) { return sqrt(dot(n, a, a)); }

/* matvec by storage kind: 0 = general CRS, 1 = symmetric upper CRS */
static void matvec(int kind, int n, const int *rp, const int *ci, const double *v,
                   const double *x, double *y)
{
    if (kind == 1)
        orc_spmv_sym(n, rp, ci, v, 1.0, x, 0.0, y);
    else
        orc_spmv(n, rp, ci, v, 1.0, x, 0.0, y);
}

/* ------------------------------------------------------------------------ */
/* Restart-frequency auto-tuning (Sec. 3.2.1, Eq. 1; Fig. 2; Sec. 4.3)       */
/* ------------------------------------------------------------------------ */

/* MM ratio of Eq. (1): R(s,t) = max{r(z)} / min{r(z)} over z = s-t+1 .. s.
 * r is indexed 1-based as in the paper (r[z-1] holds r(z)).  Requires
 * 1 <= t <= s.  A zero minimum gives +inf. */
double orc_mm_ratio(const double *r, int s, int t)
{
    double mx = r[s - t], mn = r[s - t];
    for (int z = s - t + 1; z <= s; z++) {
        double v = r[z - 1];
        if (v > mx) mx = v;
        if (v < mn) mn = v;
    }
    return (mn == 0.0) ? INFINITY : mx / mn;
}

/* The judgement of OpenATI_DAFRT: over the I samples SAMP(1..I), a small MM
 * ratio means stagnation, so IRT = 1 ("increase the restart frequency") when
 * R(I, I) < theta, else IRT = 0.  theta is a library parameter (the paper
 * passes it through IATPARAM/RATPARAM without giving a value). */
int orc_dafrt(int I, const double *samp, double theta)
{
    return orc_mm_ratio(samp, I, I) < theta ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Arnoldi with modified Gram-Schmidt (Sec. 3.2.2, "MGS: the default")       */
/* ------------------------------------------------------------------------ */

/* ------------------------------------------------------------------------ */
/* Orthogonalisation of w against v_0..v_j (Sec. 3.2.2: the four             */
/* re-orthogonalisation implementations OpenATLib offers)                    */
/* ------------------------------------------------------------------------ */

#define ORC_MGS 0  /* modified Gram-Schmidt, the default                     */
#define ORC_CGS 1  /* classical Gram-Schmidt                                 */
#define ORC_DGKS 2 /* DGKS: classical Gram-Schmidt run two times             */
#define ORC_BCGS 3 /* blocked CGS: CGS inside a block, MGS between blocks    */
#define ORC_AUTO 4 /* accuracy policy (Sec. 3.3.2) chooses among the above   */

/* V holds v_0..v_j as rows of length n; on return w is orthogonalised and
 * h[0..j] holds the projection coefficients (h_ij of the Hessenberg column).
 *   MGS : for i = 0..j: h_i = (w, v_i); w -= h_i v_i           (w updated each time)
 *   CGS : h_i = (w, v_i) for all i with w fixed; then w -= sum_i h_i v_i
 *   DGKS: CGS, then CGS again on the result; h = first + second coefficients
 *   BCGS: the basis in consecutive blocks of bl vectors, taken in order; per
 *         block CGS against the current w, then w updated before the next
 *         block (bl = 4 in the solvers). */
static void orth(int ortho, int bl, int n, int j, const double *V, double *w, double *h)
{
    if (ortho == ORC_MGS) {
        for (int i = 0; i <= j; i++) {
            h[i] = dot(n, w, V + (size_t)i * n);
            ORC_PAR
            for (int q = 0; q < n; q++)
                w[q] -= h[i] * V[(size_t)i * n + q];
        }
        return;
    }
    if (ortho == ORC_CGS || ortho == ORC_DGKS) {
        double *h2 = (double *)malloc(sizeof(double) * (size_t)(j + 1));
        int passes = (ortho == ORC_DGKS) ? 2 : 1;
        for (int i = 0; i <= j; i++) h[i] = 0.0;
        for (int pass = 0; pass < passes; pass++) {
            for (int i = 0; i <= j; i++)
                h2[i] = dot(n, w, V + (size_t)i * n);
            for (int i = 0; i <= j; i++) {
                ORC_PAR
                for (int q = 0; q < n; q++)
                    w[q] -= h2[i] * V[(size_t)i * n + q];
                h[i] += h2[i];
            }
        }
        free(h2);
        return;
    }
    /* ORC_BCGS */
    for (int i0 = 0; i0 <= j; i0 += bl) {
        int i1 = i0 + bl - 1;
        if (i1 > j) i1 = j;
        for (int i = i0; i <= i1; i++)
            h[i] = dot(n, w, V + (size_t)i * n);
        for (int i = i0; i <= i1; i++) {
            ORC_PAR
            for (int q = 0; q < n; q++)
                w[q] -= h[i] * V[(size_t)i * n + q];
        }
    }
}

/* k steps of Arnoldi from v1 = v0/||v0|| with the given orthogonalisation
 * (block length bl for BCGS).  V is (m+1) x n (row j = v_{j+1}), H is
 * (m+1) x m row-major, both zero-filled here.  Per step j: w = A v_j,
 * orth(w) gives h_{0..j,j}, h_{j+1,j} = ||w||.  Stops early on breakdown
 * (h_{j+1,j} == 0).  Returns the number of steps. */
int orc_arnoldi_ortho(int n, int kind, const int *rp, const int *ci, const double *v,
                      const double *v0, int m, int ortho, int bl, double *V, double *H)
{
    memset(V, 0, sizeof(double) * (size_t)(m + 1) * n);
    memset(H, 0, sizeof(double) * (size_t)(m + 1) * m);
    double b = nrm2(n, v0);
    for (int i = 0; i < n; i++)
        V[i] = v0[i] / b;
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *h = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    int steps = 0;
    for (int j = 0; j < m; j++) {
        matvec(kind, n, rp, ci, v, V + (size_t)j * n, w);
        orth(ortho, bl, n, j, V, w, h);
        for (int i = 0; i <= j; i++)
            H[(size_t)i * m + j] = h[i];
        double hn = nrm2(n, w);
        H[(size_t)(j + 1) * m + j] = hn;
        steps = j + 1;
        if (hn == 0.0)
            break;
        for (int q = 0; q < n; q++)
            V[(size_t)(j + 1) * n + q] = w[q] / hn;
    }
    free(w);
    free(h);
    return steps;
}

/* Gram-Schmidt QR of the k columns of X (column-major n x k) with the given
 * orthogonalisation: column j is orthogonalised against q_0..q_{j-1} by
 * orth(), then normalised.  Q is column-major n x k, R column-major k x k
 * (upper triangular: R[i + j*k] = h_i for i < j, R[j + j*k] = norm).
 * Returns the number of columns before a zero norm (k if none). */
int orc_gs_qr(int n, int k, const double *X, int ortho, int bl, double *Q, double *R)
{
    memset(R, 0, sizeof(double) * (size_t)k * k);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *h = (double *)malloc(sizeof(double) * (size_t)(k > 0 ? k : 1));
    int done = k;
    for (int j = 0; j < k; j++) {
        memcpy(w, X + (size_t)j * n, sizeof(double) * (size_t)n);
        if (j > 0) {
            orth(ortho, bl, n, j - 1, Q, w, h);
            for (int i = 0; i < j; i++) R[i + (size_t)j * k] = h[i];
        }
        double nr = nrm2(n, w);
        R[j + (size_t)j * k] = nr;
        if (nr == 0.0) { done = j; break; }
        for (int q = 0; q < n; q++) Q[(size_t)j * n + q] = w[q] / nr;
    }
    free(w);
    free(h);
    return done;
}

/* Arnoldi with MGS (the default orthogonalisation). */
int orc_arnoldi(int n, int kind, const int *rp, const int *ci, const double *v,
                const double *v0, int m, double *V, double *H)
{
    return orc_arnoldi_ortho(n, kind, rp, ci, v, v0, m, ORC_MGS, 4, V, H);
}

/* The accuracy policy's choice (Sec. 3.3.2): MGS when the requested accuracy
 * is 1e-10 or tighter, else BCGS; DGKS once a fault convergence occurred. */
static int policy_ortho(double tol, int faulted)
{
    if (faulted) return ORC_DGKS;
    return tol <= 1e-10 ? ORC_MGS : ORC_BCGS;
}

/* ------------------------------------------------------------------------ */
/* ILU(0) preconditioner (the preconditioner of the paper's solver runs,     */
/* Sec. 4.3): incomplete LU with the sparsity pattern of A, general CRS.     */
/* ------------------------------------------------------------------------ */

/* Position of column j in row i (binary search over the sorted columns), or -1. */
static int find_col(const int *rp, const int *ci, int i, int j)
{
    int lo = rp[i], hi = rp[i + 1] - 1;
    while (lo <= hi) {
        int mid = lo + (hi - lo) / 2;
        if (ci[mid] == j) return mid;
        if (ci[mid] < j) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* lu = ILU(0) factors of A in A's pattern: the strictly lower part holds L
 * (unit diagonal not stored), the rest U.  Row by row (IKJ): for each stored
 * (i, k) with k < i, in ascending k: l_ik = a_ik / u_kk, then
 * a_ij -= l_ik u_kj for every stored (i, j) with j > k whose (k, j) is stored.
 * Returns ORC_EBREAKDOWN (-5) if a diagonal entry is missing or becomes 0. */
int orc_ilu0(int n, const int *rp, const int *ci, const double *va, double *lu)
{
    for (int p = 0; p < rp[n]; p++) lu[p] = va[p];
    for (int i = 0; i < n; i++) {
        for (int p = rp[i]; p < rp[i + 1] && ci[p] < i; p++) {
            int k = ci[p];
            int dk = find_col(rp, ci, k, k);
            if (dk < 0 || lu[dk] == 0.0) return ORC_EBREAKDOWN;
            lu[p] /= lu[dk];
            for (int q = p + 1; q < rp[i + 1]; q++) {
                int kq = find_col(rp, ci, k, ci[q]);
                if (kq >= 0) lu[q] -= lu[p] * lu[kq];
            }
        }
        int di = find_col(rp, ci, i, i);
        if (di < 0 || lu[di] == 0.0) return ORC_EBREAKDOWN;
    }
    return ORC_OK;
}

/* z = (LU)^{-1} r: forward substitution with the unit lower factor, then
 * backward substitution with the upper factor. */
void orc_ilu0_solve(int n, const int *rp, const int *ci, const double *lu, const double *r,
                    double *z)
{
    for (int i = 0; i < n; i++) {
        double s = r[i];
        for (int p = rp[i]; p < rp[i + 1] && ci[p] < i; p++) s -= lu[p] * z[ci[p]];
        z[i] = s;
    }
    for (int i = n - 1; i >= 0; i--) {
        double s = z[i], d = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; p++) {
            if (ci[p] > i) s -= lu[p] * z[ci[p]];
            else if (ci[p] == i) d = lu[p];
        }
        z[i] = s / d;
    }
}

/* ------------------------------------------------------------------------ */
/* Restarted GMRES(m) (Saad & Schultz; listed in Sec. 2.2, run in Sec. 4.3)  */
/* ------------------------------------------------------------------------ */

/* Breakdown threshold: after MGS, w is (in exact arithmetic) the component of
 * A v_j orthogonal to the basis, and ||A v_j||^2 = sum_i h_ij^2 + h_{j+1,j}^2.
 * A "happy" breakdown is declared when h_{j+1,j} <= 1e-14 of that length. */
#define ORC_BREAKDOWN_REL 1e-14

/*
 * GMRES(m) with MGS Arnoldi and Givens-rotation least squares, no
 * preconditioner, x in: initial guess, out: iterate.
 *
 *   kind:     0 general CRS, 1 symmetric upper CRS
 *   m:        initial restart length;  m_max: cap for the restart rule
 *   tol:      stop when ||b - A x|| / ||b|| <= tol (true residual)
 *   maxiter:  limit on Arnoldi steps (SpMVs inside cycles)
 *   dafrt:    1 = apply the restart-frequency rule: the true residual at every
 *             restart is a sample (Sec. 4.3: "in every restarting"); each time
 *             `window` samples are gathered (Fig. 2's judgement period I) the
 *             MM-ratio judgement runs, m += dm when it says IRT = 1 (Sec. 4.3:
 *             MSIZE+5), and the sample count resets (Fig. 2: K = 0).
 *   theta:    DAFRT threshold
 *
 * Fault convergence (Sec. 3.1, 3.3.2): each cycle stops on the implicit
 * residual |g_{k+1}|/||b|| <= tau.  If the true residual computed at the next
 * restart still exceeds tol, the cycle's claim was false: the fault counter
 * is incremented and the implicit threshold is narrowed, tau *= tol/res_true.
 *
 *   ortho:    ORC_MGS / ORC_CGS / ORC_DGKS / ORC_BCGS (block length 4), or
 *             ORC_AUTO: the accuracy policy of Sec. 3.3.2 (MGS for tol <= 1e-10,
 *             else BCGS; DGKS from the first fault convergence on).
 *   M:        ILU(0) factors from orc_ilu0 (general CRS only) for right
 *             preconditioning, Arnoldi on A M^{-1}: w = A (M^{-1} v_j) and
 *             x += M^{-1} (V y); NULL = no preconditioner.  Residuals stay
 *             those of A x = b.
 *   fault_check: 1 = the accuracy mechanism below; 0 = stop at the first
 *             claimed convergence and return ORC_EFAULT (-7) when the true
 *             residual misses tol (the time / memory / stable policies of
 *             Sec. 2.3.2 do not recompute the error).
 *
 * iinfo: [0] iterations, [1] restarts (cycles completed), [2] final m,
 *        [3] fault-convergence events, [4] orthogonalisation in use at exit.
 * dinfo: [0] last implicit relative residual, [1] true relative residual.
 * hist/mhist (may be NULL): true relative residual at the start of each cycle
 *        and the restart length m that cycle runs with, up to hist_cap entries.
 */
int orc_gmres(int n, int kind, const int *rp, const int *ci, const double *va,
              const double *b, double *x, int m, int m_max, double tol,
              int maxiter, int dafrt, double theta, int window, int dm, int ortho,
              int fault_check, const double *M, int *iinfo, double *dinfo, double *hist,
              int *mhist, int hist_cap)
{
    if (m_max < m) m_max = m;
    int iters = 0, restarts = 0, faults = 0, K = 0, claimed = 0, status = ORC_OK;
    int cur = (ortho == ORC_AUTO) ? policy_ortho(tol, 0) : ortho;
    double tau = tol, res_impl = 0.0, res_true = 0.0;
    double bnorm = nrm2(n, b);
    iinfo[0] = iinfo[1] = iinfo[3] = 0;
    iinfo[2] = m;
    iinfo[4] = cur;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        dinfo[0] = dinfo[1] = 0.0;
        return ORC_OK;
    }
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    double *V = (double *)malloc(sizeof(double) * (size_t)(m_max + 1) * n);
    double *H = (double *)malloc(sizeof(double) * (size_t)(m_max + 1) * m_max);
    double *cs = (double *)malloc(sizeof(double) * (size_t)m_max);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m_max);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m_max + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m_max);
    double *samp = (double *)malloc(sizeof(double) * (size_t)(window > 0 ? window : 1));
    double *hc = (double *)malloc(sizeof(double) * (size_t)(m_max + 1));
    double *tz = (double *)malloc(sizeof(double) * (size_t)n);

    for (;;) {
        /* r = b - A x, true residual */
        matvec(kind, n, rp, ci, va, x, r);
        ORC_PAR
        for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
        double beta = nrm2(n, r);
        res_true = beta / bnorm;
        if (hist && restarts < hist_cap) { hist[restarts] = res_true; mhist[restarts] = m; }
        if (res_true <= tol) { status = ORC_OK; break; }
        if (iters >= maxiter) { status = ORC_ENOCONV; break; }
        if (claimed && !fault_check) { faults++; status = ORC_EFAULT; break; }
        if (claimed) {
            faults++;
            tau *= tol / res_true;
            if (ortho == ORC_AUTO) cur = policy_ortho(tol, 1);
        }
        claimed = 0;
        if (dafrt && restarts > 0 && window > 0) {
            samp[K++] = res_true;
            if (K == window) {
                if (orc_dafrt(window, samp, theta)) {
                    m += dm;
                    if (m > m_max) m = m_max;
                }
                K = 0;
            }
        }
        if (mhist && restarts < hist_cap) mhist[restarts] = m; /* m this cycle uses */
        /* one cycle */
        ORC_PAR
        for (int i = 0; i < n; i++) V[i] = r[i] / beta;
        for (int i = 0; i <= m; i++) g[i] = 0.0;
        g[0] = beta;
        int k = 0, broke = 0;
        for (int j = 0; j < m; j++) {
            iters++;
            if (M) {
                orc_ilu0_solve(n, rp, ci, M, V + (size_t)j * n, tz);
                matvec(kind, n, rp, ci, va, tz, w);
            } else {
                matvec(kind, n, rp, ci, va, V + (size_t)j * n, w);
            }
            orth(cur, 4, n, j, V, w, hc);
            double len2 = 0.0;
            for (int i = 0; i <= j; i++) {
                H[(size_t)i * m_max + j] = hc[i];
                len2 += hc[i] * hc[i];
            }
            double hn = nrm2(n, w);
            H[(size_t)(j + 1) * m_max + j] = hn;
            len2 += hn * hn;
            /* previous rotations on column j */
            for (int i = 0; i < j; i++) {
                double a = H[(size_t)i * m_max + j], c = H[(size_t)(i + 1) * m_max + j];
                H[(size_t)i * m_max + j] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * m_max + j] = -sn[i] * a + cs[i] * c;
            }
            /* new rotation zeroing h_{j+1,j} */
            double a = H[(size_t)j * m_max + j];
            double rr = hypot(a, hn);
            if (rr == 0.0) { status = ORC_EBREAKDOWN; k = j; broke = 2; break; }
            cs[j] = a / rr;
            sn[j] = hn / rr;
            H[(size_t)j * m_max + j] = rr;
            H[(size_t)(j + 1) * m_max + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            res_impl = fabs(g[j + 1]) / bnorm;
            k = j + 1;
            if (hn <= ORC_BREAKDOWN_REL * sqrt(len2)) { broke = 1; break; }
            ORC_PAR
            for (int q = 0; q < n; q++)
                V[(size_t)(j + 1) * n + q] = w[q] / hn;
            if (res_impl <= tau) { claimed = 1; break; }
            if (iters >= maxiter) break;
        }
        if (broke == 2) break;
        if (broke == 1) claimed = 1;
        /* back substitution R y = g, then x += V y */
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int q = i + 1; q < k; q++)
                s -= H[(size_t)i * m_max + q] * y[q];
            y[i] = s / H[(size_t)i * m_max + i];
        }
        if (M) {
            for (int q = 0; q < n; q++) w[q] = 0.0;
            for (int i = 0; i < k; i++)
                for (int q = 0; q < n; q++)
                    w[q] += y[i] * V[(size_t)i * n + q];
            orc_ilu0_solve(n, rp, ci, M, w, tz);
            for (int q = 0; q < n; q++) x[q] += tz[q];
        } else {
            for (int i = 0; i < k; i++) {
                ORC_PAR
                for (int q = 0; q < n; q++)
                    x[q] += y[i] * V[(size_t)i * n + q];
            }
        }
        restarts++;
    }
    iinfo[0] = iters;
    iinfo[1] = restarts;
    iinfo[2] = m;
    iinfo[3] = faults;
    iinfo[4] = cur;
    dinfo[0] = res_impl;
    dinfo[1] = res_true;
    free(r); free(w); free(V); free(H); free(cs); free(sn); free(g); free(y); free(samp);
    free(hc); free(tz);
    return status;
}

/* ------------------------------------------------------------------------ */
/* BiCGStab (van der Vorst), no preconditioner (listed in Sec. 2.2, run in   */
/* Sec. 4.3).                                                                */
/* ------------------------------------------------------------------------ */

/*
 * One BiCGStab iteration (two SpMVs):
 *   rho' = (rhat, r); beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v)
 *   v = A p; alpha = rho' / (rhat, v); s = r - alpha v
 *   if ||s||/||b|| <= tau: x += alpha p, stop
 *   t = A s; omega = (t, s)/(t, t); x += alpha p + omega s; r = s - omega t
 *   rho = rho'; stop if ||r||/||b|| <= tau
 * With M (ILU(0) factors, general CRS) the iteration is right-preconditioned:
 * p^ = M^{-1} p and s^ = M^{-1} s replace p and s in the products with A and in
 * the update of x (x += alpha p^ + omega s^); residuals stay those of A x = b.
 * Breakdown (status -5) when rho', (rhat, v) or (t, t) is exactly zero, or omega
 * is zero without convergence.  The true residual is checked after every
 * claimed convergence; a false claim (fault convergence, Sec. 3.3.2) restarts
 * the recurrence from the true residual with tau *= tol/res_true.
 * iinfo: [0] iterations, [1] recurrence restarts, [3] fault events.
 * dinfo: [0] last recursive relative residual, [1] true relative residual.
 */
int orc_bicgstab(int n, int kind, const int *rp, const int *ci, const double *va,
                 const double *b, double *x, double tol, int maxiter, const double *M,
                 int *iinfo, double *dinfo)
{
    int iters = 0, restarts = 0, faults = 0, claimed = 0, status = ORC_OK;
    double tau = tol, res_rec = 0.0, res_true = 0.0;
    double bnorm = nrm2(n, b);
    iinfo[0] = iinfo[1] = iinfo[2] = iinfo[3] = 0;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        dinfo[0] = dinfo[1] = 0.0;
        return ORC_OK;
    }
    size_t bytes = sizeof(double) * (size_t)n;
    double *r = (double *)malloc(bytes), *rh = (double *)malloc(bytes);
    double *p = (double *)malloc(bytes), *v = (double *)malloc(bytes);
    double *s = (double *)malloc(bytes), *t = (double *)malloc(bytes);
    double *ph = (double *)malloc(bytes), *sh = (double *)malloc(bytes);
    for (;;) {
        matvec(kind, n, rp, ci, va, x, r);
        ORC_PAR
        for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
        res_true = nrm2(n, r) / bnorm;
        if (res_true <= tol) { status = ORC_OK; break; }
        if (iters >= maxiter) { status = ORC_ENOCONV; break; }
        if (claimed) { faults++; tau *= tol / res_true; restarts++; }
        else if (iters > 0) restarts++;
        claimed = 0;
        ORC_PAR
        for (int i = 0; i < n; i++) { rh[i] = r[i]; p[i] = 0.0; v[i] = 0.0; }
        double rho = 1.0, alpha = 1.0, omega = 1.0;
        int broke = 0;
        while (iters < maxiter) {
            iters++;
            double rho1 = dot(n, rh, r);
            if (rho1 == 0.0) { broke = 1; break; }
            double beta = (rho1 / rho) * (alpha / omega);
            ORC_PAR
            for (int i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            if (M) orc_ilu0_solve(n, rp, ci, M, p, ph);
            else {
                ORC_PAR
                for (int i = 0; i < n; i++) ph[i] = p[i];
            }
            matvec(kind, n, rp, ci, va, ph, v);
            double sigma = dot(n, rh, v);
            if (sigma == 0.0) { broke = 1; break; }
            alpha = rho1 / sigma;
            ORC_PAR
            for (int i = 0; i < n; i++) s[i] = r[i] - alpha * v[i];
            double sn = nrm2(n, s) / bnorm;
            if (sn <= tau) {
                for (int i = 0; i < n; i++) x[i] += alpha * ph[i];
                res_rec = sn;
                claimed = 1;
                break;
            }
            if (M) orc_ilu0_solve(n, rp, ci, M, s, sh);
            else {
                ORC_PAR
                for (int i = 0; i < n; i++) sh[i] = s[i];
            }
            matvec(kind, n, rp, ci, va, sh, t);
            double tt = dot(n, t, t);
            if (tt == 0.0) { broke = 1; break; }
            omega = dot(n, t, s) / tt;
            ORC_PAR
            for (int i = 0; i < n; i++) x[i] += alpha * ph[i] + omega * sh[i];
            ORC_PAR
            for (int i = 0; i < n; i++) r[i] = s[i] - omega * t[i];
            rho = rho1;
            res_rec = nrm2(n, r) / bnorm;
            if (res_rec <= tau) { claimed = 1; break; }
            if (omega == 0.0) { broke = 1; break; }
        }
        if (broke) {
            matvec(kind, n, rp, ci, va, x, r);
            for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
            res_true = nrm2(n, r) / bnorm;
            status = (res_true <= tol) ? ORC_OK : ORC_EBREAKDOWN;
            break;
        }
    }
    iinfo[0] = iters;
    iinfo[1] = restarts;
    iinfo[3] = faults;
    dinfo[0] = res_rec;
    dinfo[1] = res_true;
    free(r); free(rh); free(p); free(v); free(s); free(t); free(ph); free(sh);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Restarted Lanczos eigensolver for symmetric matrices (Sec. 2.2, 4.3:      */
/* OpenATI_EIGENSOLVE, restarted Lanczos), thick restart.                     */
/* ------------------------------------------------------------------------ */

/* Eigen-decomposition of the symmetric m x m matrix A (row-major, destroyed)
 * by cyclic Jacobi rotations until the off-diagonal mass is below 1e-30 of
 * the total: A = S diag(w) S^T, S row-major (column c = eigenvector c).
 * Eigenpairs are returned sorted by eigenvalue, largest first. */
void orc_sym_eig(int m, double *A, double *w, double *S)
{
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) S[i * m + j] = (i == j) ? 1.0 : 0.0;
    double tot = 0.0;
    for (int i = 0; i < m * m; i++) tot += A[i] * A[i];
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) off += 2.0 * A[p * m + q] * A[p * m + q];
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < m; p++)
            for (int q = p + 1; q < m; q++) {
                double apq = A[p * m + q];
                if (apq == 0.0) continue;
                /* rotation angle zeroing A[p][q]: tan(2t) = 2 apq / (aqq - app) */
                double tau = (A[q * m + q] - A[p * m + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
                for (int k = 0; k < m; k++) { /* A = A G (columns p, q) */
                    double akp = A[k * m + p], akq = A[k * m + q];
                    A[k * m + p] = c * akp - sn * akq;
                    A[k * m + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < m; k++) { /* A = G^T A (rows p, q) */
                    double apk = A[p * m + k], aqk = A[q * m + k];
                    A[p * m + k] = c * apk - sn * aqk;
                    A[q * m + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < m; k++) { /* S = S G */
                    double skp = S[k * m + p], skq = S[k * m + q];
                    S[k * m + p] = c * skp - sn * skq;
                    S[k * m + q] = sn * skp + c * skq;
                }
            }
    }
    for (int i = 0; i < m; i++) w[i] = A[i * m + i];
    /* sort descending (selection sort, columns of S follow) */
    for (int i = 0; i < m; i++) {
        int b = i;
        for (int j = i + 1; j < m; j++) if (w[j] > w[b]) b = j;
        if (b != i) {
            double t = w[i]; w[i] = w[b]; w[b] = t;
            for (int k = 0; k < m; k++) {
                double u = S[k * m + i]; S[k * m + i] = S[k * m + b]; S[k * m + b] = u;
            }
        }
    }
}

/*
 * The nev largest eigenvalues of a symmetric A (general CRS holding both
 * triangles, or upper storage with kind = 1) by restarted Lanczos with full
 * re-orthogonalisation (DGKS) and thick restart (Krylov-Schur form):
 *   - a cycle extends the orthonormal basis v_0..v_m by Lanczos steps
 *     w = A v_j, orthogonalised against every basis vector (the coefficients
 *     fill column j of the projected matrix T = V^T A V), v_{j+1} = w/||w||;
 *   - T (m x m, symmetrised) = S diag(theta) S^T; the residual of Ritz pair i
 *     is |beta_m S[m-1][i]| with beta_m = ||w|| of the last step;
 *   - if the nev largest Ritz values have residual <= tol |theta_i| the
 *     solve ends (the Ritz vectors V S[:, i] are the eigenvectors);
 *   - else the k = nev + (m - nev)/2 leading Ritz vectors are kept as the new
 *     v_0..v_{k-1}, v_m becomes v_k, and T restarts as diag(theta_0..k-1)
 *     with row / column k holding beta_m S[m-1][i] (the thick restart).
 * Restart rule (Eq. 1, Fig. 2, Sec. 4.3) when m_max > m: after every cycle
 * that does not converge, the largest relative residual of the wanted Ritz
 * pairs is a sample; every 5 samples the MM ratio decides (orc_dafrt with
 * theta) and m grows by 5 (capped at m_max) when the residuals stagnate.
 * v0: starting vector (n).  evals: nev values (largest first); evecs (may be
 * NULL): n x nev column-major; resid: nev Ritz residual norms.
 * iinfo: [0] Lanczos steps (SpMVs), [1] restarts, [2] final m.  Returns 0,
 * -4 (restart limit) or -5 (a zero vector: Krylov space exhausted before m
 * steps).
 */
int orc_lanczos(int n, int kind, const int *rp, const int *ci, const double *va, int nev,
                int m, int m_max, double theta, double tol, int maxrestart, const double *v0,
                double *evals, double *evecs, double *resid, int *iinfo)
{
    if (m_max < m) m_max = m;
    if (nev < 1 || m <= nev || m_max > n) return ORC_EBREAKDOWN;
    int mm = m_max; /* capacity */
    double *V = (double *)calloc((size_t)(mm + 1) * n, sizeof(double));
    double *T = (double *)calloc((size_t)(mm + 1) * (mm + 1), sizeof(double)); /* T[i*(mm+1)+j] */
    double *A = (double *)malloc(sizeof(double) * (size_t)mm * mm);
    double *S = (double *)malloc(sizeof(double) * (size_t)mm * mm);
    double *th = (double *)malloc(sizeof(double) * (size_t)mm);
    double *h = (double *)malloc(sizeof(double) * (size_t)(mm + 1));
    double *Y = (double *)malloc(sizeof(double) * (size_t)mm * n);
    double samp[5];
    int K = 0;
    double nb = nrm2(n, v0);
    for (int q = 0; q < n; q++) V[q] = v0[q] / nb;
    int k = 0, steps = 0, status = ORC_ENOCONV, restarts = 0;
    double beta = 0.0;
    for (;;) {
        for (int j = k; j < m; j++) {
            double *w = V + (size_t)(j + 1) * n;
            matvec(kind, n, rp, ci, va, V + (size_t)j * n, w);
            steps++;
            orth(ORC_DGKS, 4, n, j, V, w, h);
            for (int i = 0; i <= j; i++) T[i * (mm + 1) + j] = h[i];
            beta = nrm2(n, w);
            T[(j + 1) * (mm + 1) + j] = beta;
            if (beta == 0.0) { status = ORC_EBREAKDOWN; goto done; }
            for (int q = 0; q < n; q++) w[q] /= beta;
        }
        /* symmetrised projected matrix and its eigenpairs */
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++)
                A[i * m + j] = 0.5 * (T[i * (mm + 1) + j] + T[j * (mm + 1) + i]);
        orc_sym_eig(m, A, th, S);
        int conv = 1;
        for (int i = 0; i < nev; i++) {
            resid[i] = fabs(beta * S[(m - 1) * m + i]);
            evals[i] = th[i];
            if (resid[i] > tol * fabs(th[i])) conv = 0;
        }
        if (conv || restarts >= maxrestart) {
            status = conv ? ORC_OK : ORC_ENOCONV;
            if (evecs)
                for (int i = 0; i < nev; i++)
                    for (int q = 0; q < n; q++) {
                        double sum = 0.0;
                        for (int j = 0; j < m; j++) sum += V[(size_t)j * n + q] * S[j * m + i];
                        evecs[(size_t)i * n + q] = sum;
                    }
            break;
        }
        /* restart rule: the worst relative residual of the wanted pairs */
        if (m_max > m || K > 0) {
            double worst = 0.0;
            for (int i = 0; i < nev; i++) {
                double r = resid[i] / fabs(th[i]);
                if (r > worst) worst = r;
            }
            samp[K++] = worst;
            if (K == 5) {
                int grow = orc_dafrt(5, samp, theta);
                K = 0;
                if (grow && m < m_max) {
                    /* the thick restart below keeps k of the current m vectors;
                       the next cycle runs to the larger m */
                    int k2 = nev + (m - nev) / 2;
                    for (int i = 0; i < k2; i++)
                        for (int q = 0; q < n; q++) {
                            double sum = 0.0;
                            for (int j = 0; j < m; j++) sum += V[(size_t)j * n + q] * S[j * m + i];
                            Y[(size_t)i * n + q] = sum;
                        }
                    memcpy(V, Y, sizeof(double) * (size_t)k2 * n);
                    memcpy(V + (size_t)k2 * n, V + (size_t)m * n, sizeof(double) * (size_t)n);
                    for (int i = 0; i < (mm + 1) * (mm + 1); i++) T[i] = 0.0;
                    for (int i = 0; i < k2; i++) {
                        T[i * (mm + 1) + i] = th[i];
                        T[k2 * (mm + 1) + i] = beta * S[(m - 1) * m + i];
                    }
                    k = k2;
                    m = m + 5 > m_max ? m_max : m + 5;
                    restarts++;
                    continue;
                }
            }
        }
        /* thick restart with the k leading Ritz vectors */
        k = nev + (m - nev) / 2;
        for (int i = 0; i < k; i++)
            for (int q = 0; q < n; q++) {
                double sum = 0.0;
                for (int j = 0; j < m; j++) sum += V[(size_t)j * n + q] * S[j * m + i];
                Y[(size_t)i * n + q] = sum;
            }
        memcpy(V, Y, sizeof(double) * (size_t)k * n);
        memcpy(V + (size_t)k * n, V + (size_t)m * n, sizeof(double) * (size_t)n);
        for (int i = 0; i < (mm + 1) * (mm + 1); i++) T[i] = 0.0;
        for (int i = 0; i < k; i++) {
            T[i * (mm + 1) + i] = th[i];
            T[k * (mm + 1) + i] = beta * S[(m - 1) * m + i];
        }
        restarts++;
    }
done:
    iinfo[0] = steps;
    iinfo[1] = restarts;
    iinfo[2] = m;
    free(V); free(T); free(A); free(S); free(th); free(h); free(Y);
    return status;
}

/* ------------------------------------------------------------------------ */
/* FP32-inside-FP64 iterative refinement with GMRES(m) as the inner solver.   */
/* The paper's accuracy policy deliberately avoids refinement (Sec. 3.3.1);  */
/* this is the library's precision extension, written as the textbook        */
/* refinement loop: r = b - A x (FP64); solve A d = r/||r|| approximately in */
/* FP32; x += ||r|| d (FP64).                                                */
/* ------------------------------------------------------------------------ */

static float sdot(int n, const float *a, const float *b)
{
    float s = 0.0f;
    for (int i = 0; i < n; i++)
        s += a[i] * b[i];
    return s;
}

/* Inner FP32 GMRES(m) from d = 0 on A32 d = r32: SpMV, basis and inner
 * products (accumulated) in FP32; Hessenberg, Givens rotations and the small
 * least-squares solve in FP64; d += V y in FP32.  Stops when the implicit
 * residual relative to ||r32|| is <= tol_in or after maxit steps.
 * Returns the number of Arnoldi steps taken (status -5 on breakdown is folded
 * into an early return; the outer loop tests the true residual anyway). */
int orc_gmres_f32_inner(int n, const int *rp, const int *ci, const float *va,
                        const float *r32, float *d, int m, double tol_in, int maxit)
{
    int iters = 0;
    double rb = sqrt((double)sdot(n, r32, r32));
    for (int i = 0; i < n; i++) d[i] = 0.0f;
    if (rb == 0.0) return 0;
    float *rin = (float *)malloc(sizeof(float) * (size_t)n);
    float *w = (float *)malloc(sizeof(float) * (size_t)n);
    float *V = (float *)malloc(sizeof(float) * (size_t)(m + 1) * n);
    double *H = (double *)malloc(sizeof(double) * (size_t)(m + 1) * m);
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    int done = 0;
    while (!done && iters < maxit) {
        orc_spmv_f32(n, rp, ci, va, 1.0f, d, 0.0f, rin);
        for (int i = 0; i < n; i++) rin[i] = r32[i] - rin[i];
        double beta = sqrt((double)sdot(n, rin, rin));
        if (beta / rb <= tol_in || beta == 0.0) break;
        for (int i = 0; i < n; i++) V[i] = (float)(rin[i] / beta);
        for (int i = 0; i <= m; i++) g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; j++) {
            iters++;
            orc_spmv_f32(n, rp, ci, va, 1.0f, V + (size_t)j * n, 0.0f, w);
            double len2 = 0.0;
            for (int i = 0; i <= j; i++) {
                double h = (double)sdot(n, w, V + (size_t)i * n);
                H[(size_t)i * m + j] = h;
                len2 += h * h;
                float hf = (float)h;
                for (int q = 0; q < n; q++)
                    w[q] -= hf * V[(size_t)i * n + q];
            }
            double hn = sqrt((double)sdot(n, w, w));
            len2 += hn * hn;
            H[(size_t)(j + 1) * m + j] = hn;
            for (int i = 0; i < j; i++) {
                double a = H[(size_t)i * m + j], c = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * c;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            double a = H[(size_t)j * m + j];
            double rr = hypot(a, hn);
            if (rr == 0.0) { done = 1; break; }
            cs[j] = a / rr;
            sn[j] = hn / rr;
            H[(size_t)j * m + j] = rr;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            if (hn <= ORC_BREAKDOWN_REL * sqrt(len2)) { done = 1; break; }
            for (int q = 0; q < n; q++)
                V[(size_t)(j + 1) * n + q] = (float)((double)w[q] / hn);
            if (fabs(g[j + 1]) / rb <= tol_in) { done = 1; break; }
            if (iters >= maxit) break;
        }
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int q = i + 1; q < k; q++)
                s -= H[(size_t)i * m + q] * y[q];
            y[i] = s / H[(size_t)i * m + i];
        }
        for (int i = 0; i < k; i++) {
            float yi = (float)y[i];
            for (int q = 0; q < n; q++)
                d[q] += yi * V[(size_t)i * n + q];
        }
    }
    free(rin); free(w); free(V); free(H); free(cs); free(sn); free(g); free(y);
    return iters;
}

/*
 * Mixed-precision iterative refinement (the FP32-inside-FP64 extension of the
 * GMRES(m) solver; no counterpart in the paper, whose accuracy policy keeps
 * the whole solve in FP64).  Each outer step: r = b - A x in FP64; stop when
 * ||r|| / ||b|| <= tol or after max_outer steps; solve float(A) d =
 * float(r / ||r||) by FP32 GMRES(m) to tol_in; x += ||r|| * double(d).
 * Nothing else: no switch to FP64 GMRES when the steps stagnate.
 * iinfo: [0] total inner iterations, [1] outer steps.  dinfo: [1] true
 * relative residual at exit.
 */
int orc_gmres_ir(int n, const int *rp, const int *ci, const double *va,
                 const double *b, double *x, int m, double tol, double tol_in,
                 int maxit_in, int max_outer, int *iinfo, double *dinfo)
{
    for (int i = 0; i < 6; i++) iinfo[i] = 0;
    dinfo[0] = dinfo[1] = 0.0;
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) {
        for (int i = 0; i < n; i++) x[i] = 0.0;
        return ORC_OK;
    }
    int nnz = rp[n];
    float *va32 = (float *)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    for (int k = 0; k < nnz; k++) va32[k] = (float)va[k];
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    float *r32 = (float *)malloc(sizeof(float) * (size_t)n);
    float *d = (float *)malloc(sizeof(float) * (size_t)n);
    int status = ORC_OK, outer = 0, inner_total = 0;
    double res = 0.0;
    for (;;) {
        /* outer step: FP64 residual r = b - A x */
        orc_spmv(n, rp, ci, va, 1.0, x, 0.0, r);
        for (int i = 0; i < n; i++) r[i] = b[i] - r[i];
        double rn = nrm2(n, r);
        res = rn / bnorm;
        if (res <= tol) { status = ORC_OK; break; }
        if (outer >= max_outer) { status = ORC_ENOCONV; break; }
        /* inner: FP32 GMRES on float(A) d = float(r / ||r||) to tol_in */
        for (int i = 0; i < n; i++) r32[i] = (float)(r[i] / rn);
        inner_total += orc_gmres_f32_inner(n, rp, ci, va32, r32, d, m, tol_in, maxit_in);
        /* update: x += ||r|| * double(d) */
        for (int i = 0; i < n; i++) x[i] += rn * (double)d[i];
        outer++;
    }
    iinfo[0] = inner_total;
    iinfo[1] = outer;
    dinfo[1] = res;
    free(va32); free(r); free(r32); free(d);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Matrix features (inputs of the learned tuner)                             */
/* ------------------------------------------------------------------------ */

/*
 * raw[0] n, raw[1] nnz, raw[2] mean row length, raw[3] population variance of
 * row lengths, raw[4] max row length, raw[5] bandwidth max |i - j| over stored
 * entries, raw[6] symmetry flag: 1 when stored as upper triangle (sym_upper),
 * else 1 iff pattern and values equal their transpose exactly.
 * feat[8] (network input): ln(1+n), ln(1+nnz), ln(1+mean), ln(1+var),
 * ln(1+max), ln(1+bandwidth), sym, ln(1+max) - ln(1+mean).
 */
void orc_features(int n, const int *rp, const int *ci, const double *va,
                  int sym_upper, double *raw, double *feat)
{
    int nnz = rp[n];
    double mean = n > 0 ? (double)nnz / n : 0.0;
    double var = 0.0, mx = 0.0, bw = 0.0;
    for (int i = 0; i < n; i++) {
        double L = rp[i + 1] - rp[i];
        var += (L - mean) * (L - mean);
        if (L > mx) mx = L;
        for (int k = rp[i]; k < rp[i + 1]; k++) {
            double d = fabs((double)(ci[k] - i));
            if (d > bw) bw = d;
        }
    }
    var = n > 0 ? var / n : 0.0;
    int sym = 1;
    if (!sym_upper) {
        /* every (i, j, v) must have a stored (j, i, v): search row j */
        for (int i = 0; i < n && sym; i++) {
            for (int k = rp[i]; k < rp[i + 1] && sym; k++) {
                int j = ci[k], found = 0;
                for (int q = rp[j]; q < rp[j + 1]; q++)
                    if (ci[q] == i) { found = (va[q] == va[k]); break; }
                if (!found) sym = 0;
            }
        }
    }
    raw[0] = n; raw[1] = nnz; raw[2] = mean; raw[3] = var; raw[4] = mx; raw[5] = bw;
    raw[6] = sym;
    feat[0] = log1p((double)n);
    feat[1] = log1p((double)nnz);
    feat[2] = log1p(mean);
    feat[3] = log1p(var);
    feat[4] = log1p(mx);
    feat[5] = log1p(bw);
    feat[6] = sym;
    feat[7] = log1p(mx) - log1p(mean);
}

/* ------------------------------------------------------------------------ */
/* Tuner MLP: d_in -> h1 (ReLU) -> h2 (ReLU) -> sum(heads) logits,           */
/* softmax cross-entropy per head, Adam.  FP64 reference of the GPU's FP32   */
/* kernels.  Parameter blob: W1[h1][d_in], b1[h1], W2[h2][h1], b2[h2],       */
/* W3[o][h2], b3[o], o = sum of head sizes.                                  */
/* ------------------------------------------------------------------------ */

static void mlp_layer(const double *W, const double *bias, int out, int in,
                      const double *a, double *z)
{
    for (int o = 0; o < out; o++) {
        double s = bias[o];
        for (int i = 0; i < in; i++)
            s += W[(size_t)o * in + i] * a[i];
        z[o] = s;
    }
}

void orc_mlp_forward(const double *P, int d_in, int h1, int h2, int o,
                     const double *X, int B, double *logits)
{
    const double *W1 = P, *b1 = W1 + (size_t)h1 * d_in, *W2 = b1 + h1,
                 *b2 = W2 + (size_t)h2 * h1, *W3 = b2 + h2, *b3 = W3 + (size_t)o * h2;
    double *a1 = (double *)malloc(sizeof(double) * (size_t)h1);
    double *a2 = (double *)malloc(sizeof(double) * (size_t)h2);
    for (int s = 0; s < B; s++) {
        mlp_layer(W1, b1, h1, d_in, X + (size_t)s * d_in, a1);
        for (int i = 0; i < h1; i++) a1[i] = a1[i] > 0.0 ? a1[i] : 0.0;
        mlp_layer(W2, b2, h2, h1, a1, a2);
        for (int i = 0; i < h2; i++) a2[i] = a2[i] > 0.0 ? a2[i] : 0.0;
        mlp_layer(W3, b3, o, h2, a2, logits + (size_t)s * o);
    }
    free(a1); free(a2);
}

/* Loss = (1/B) sum_s sum_heads -log softmax(logits_head)[label], and its
 * gradient with respect to every parameter (grad has the blob's layout).
 * heads[h] is the size of head h; labels is B x nh.  Returns the loss. */
double orc_mlp_loss_grad(const double *P, int d_in, int h1, int h2, int nh,
                         const int *heads, const double *X, const int *labels,
                         int B, double *grad)
{
    int o = 0;
    for (int h = 0; h < nh; h++) o += heads[h];
    size_t np = (size_t)h1 * d_in + h1 + (size_t)h2 * h1 + h2 + (size_t)o * h2 + o;
    memset(grad, 0, sizeof(double) * np);
    const double *W1 = P, *b1 = W1 + (size_t)h1 * d_in, *W2 = b1 + h1,
                 *b2 = W2 + (size_t)h2 * h1, *W3 = b2 + h2, *b3 = W3 + (size_t)o * h2;
    double *gW1 = grad, *gb1 = gW1 + (size_t)h1 * d_in, *gW2 = gb1 + h1,
           *gb2 = gW2 + (size_t)h2 * h1, *gW3 = gb2 + h2, *gb3 = gW3 + (size_t)o * h2;
    (void)b3;
    double *z1 = (double *)malloc(sizeof(double) * (size_t)h1);
    double *a1 = (double *)malloc(sizeof(double) * (size_t)h1);
    double *z2 = (double *)malloc(sizeof(double) * (size_t)h2);
    double *a2 = (double *)malloc(sizeof(double) * (size_t)h2);
    double *z3 = (double *)malloc(sizeof(double) * (size_t)o);
    double *d3 = (double *)malloc(sizeof(double) * (size_t)o);
    double *d2 = (double *)malloc(sizeof(double) * (size_t)h2);
    double *d1 = (double *)malloc(sizeof(double) * (size_t)h1);
    double loss = 0.0;
    for (int s = 0; s < B; s++) {
        const double *x = X + (size_t)s * d_in;
        mlp_layer(W1, b1, h1, d_in, x, z1);
        for (int i = 0; i < h1; i++) a1[i] = z1[i] > 0.0 ? z1[i] : 0.0;
        mlp_layer(W2, b2, h2, h1, a1, z2);
        for (int i = 0; i < h2; i++) a2[i] = z2[i] > 0.0 ? z2[i] : 0.0;
        mlp_layer(W3, P + ((size_t)h1 * d_in + h1 + (size_t)h2 * h1 + h2 + (size_t)o * h2),
                  o, h2, a2, z3);
        /* softmax cross-entropy per head: dL/dz = (softmax - onehot) / B */
        int off = 0;
        for (int h = 0; h < nh; h++) {
            int K = heads[h];
            double mx = z3[off];
            for (int c = 1; c < K; c++) if (z3[off + c] > mx) mx = z3[off + c];
            double se = 0.0;
            for (int c = 0; c < K; c++) se += exp(z3[off + c] - mx);
            int lab = labels[(size_t)s * nh + h];
            loss += -(z3[off + lab] - mx - log(se)) / B;
            for (int c = 0; c < K; c++)
                d3[off + c] = (exp(z3[off + c] - mx) / se - (c == lab ? 1.0 : 0.0)) / B;
            off += K;
        }
        for (int q = 0; q < o; q++) {
            gb3[q] += d3[q];
            for (int i = 0; i < h2; i++) gW3[(size_t)q * h2 + i] += d3[q] * a2[i];
        }
        for (int i = 0; i < h2; i++) {
            double s2 = 0.0;
            for (int q = 0; q < o; q++) s2 += W3[(size_t)q * h2 + i] * d3[q];
            d2[i] = z2[i] > 0.0 ? s2 : 0.0;
        }
        for (int q = 0; q < h2; q++) {
            gb2[q] += d2[q];
            for (int i = 0; i < h1; i++) gW2[(size_t)q * h1 + i] += d2[q] * a1[i];
        }
        for (int i = 0; i < h1; i++) {
            double s1 = 0.0;
            for (int q = 0; q < h2; q++) s1 += W2[(size_t)q * h1 + i] * d2[q];
            d1[i] = z1[i] > 0.0 ? s1 : 0.0;
        }
        for (int q = 0; q < h1; q++) {
            gb1[q] += d1[q];
            for (int i = 0; i < d_in; i++) gW1[(size_t)q * d_in + i] += d1[q] * x[i];
        }
    }
    free(z1); free(a1); free(z2); free(a2); free(z3); free(d3); free(d2); free(d1);
    return loss;
}

/* Adam (Kingma & Ba), step t >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
void orc_adam(double *P, const double *G, double *M, double *Vv, int np, int t,
              double lr, double b1, double b2, double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int i = 0; i < np; i++) {
        M[i] = b1 * M[i] + (1.0 - b1) * G[i];
        Vv[i] = b2 * Vv[i] + (1.0 - b2) * G[i] * G[i];
        P[i] -= lr * (M[i] / c1) / (sqrt(Vv[i] / c2) + eps);
    }
}
