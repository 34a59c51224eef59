/*
 * cpcp_oracle.c -- plain, slow, fp64 CPU oracle for the multilevel CPCP
 * proximal step.  TEST INFRASTRUCTURE ONLY: nothing on the product path may
 * link, import or call this file; only the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * What it computes (each function cites the passage it follows):
 *   - shrink (soft thresholding) S_theta[x] = sign(x) max(|x| - theta, 0)
 *     (Sec. 2.1, Alg. 1 step S; Alg. 3 thresholding step).
 *   - singular value thresholding U S_theta[Sigma] V^T (Sec. 2.1, Alg. 1;
 *     Sec. 3.2, minimiser of the coarse augmented Lagrangian).
 *   - the SVD itself by one-sided (Hestenes) Jacobi rotations, hand written.
 *   - the interpolation operator R_n of eq. (Rx) following its worked example
 *     (Sec. 3.1), and the composite multilevel R = R_n R_{n/2} ... R_{n_H}
 *     (Sec. 3.1), formed as an explicit product of per-level matrices.
 *   - the CPCP objective of eq. (cpcp) and its gradient eq. (cpcp-grad-LS).
 *   - an accelerated proximal-gradient solver for eq. (cpcp) whose L-prox is
 *     the coarse SVT + prolongation step of Alg. 4 (restrict -> SVD -> SVT ->
 *     prolong) and whose S-prox is the shrink of Alg. 3, with the joint step
 *     1/2 fixed by the 2-Lipschitz gradient (Sec. 2.3).
 *   - Frank-Wolfe Thresholding (Alg. 3) and ML-FWT (Alg. 6) for eq. (cpcp),
 *     with the exact two-segment line search.
 *   - the paper-literal IALM (Alg. 1) and ML-IALM (Alg. 4), the latter also
 *     with two other transfer operators for comparison: the printed R
 *     unscaled, and R_o = R (R^T R)^{-1/2}, the operator with orthonormal
 *     columns and the same range, for which Theorem LH-eps gives epsilon = 0.
 *
 * Readings taken where the paper is silent:
 *   * momentum: FISTA extrapolation on both L and S, restarted at level switches;
 *   * continuation: mu_k = max(mu_0 eta^k, mu_bar), eta = 0.9, mu_0 = ||P_Q D||_2;
 *   * residual: relative gradient-mapping norm at mu_bar on the fine level;
 *   * level switching: start coarsest; every c iterations on a coarse level
 *     move one level finer when the restricted gradient keeps less than
 *     kappa(level) of the gradient's norm (see or_restriction_kappa); once
 *     mu_k = mu_bar, every c iterations evaluate the fine residual: stop if
 *     rel-KKT <= tol, and on a coarse level also move finer if the residual
 *     fell by less than the switch ratio since the last check on this level;
 *   * R is scaled to unit spectral norm (Assumption 4);
 *   * odd n: coarse node j sits at fine index 2j-1;
 *   * n > m: the transposed problem is solved.
 *
 * All matrices are row-major double arrays unless stated otherwise.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_NOTCONV 3

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static double *dalloc(size_t n) { return (double *)calloc(n ? n : 1, sizeof(double)); }

/* C (m x n) = A (m x k) * B (k x n), all row-major. */
static void matmul(int m, int k, int n, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(static) if ((long)m * k * n > 200000)
    for (int i = 0; i < m; i++) {
        double *c = C + (size_t)i * n;
        for (int j = 0; j < n; j++) c[j] = 0.0;
        for (int p = 0; p < k; p++) {
            double a = A[(size_t)i * k + p];
            if (a == 0.0) continue;
            const double *b = B + (size_t)p * n;
            for (int j = 0; j < n; j++) c[j] += a * b[j];
        }
    }
}

/* C (m x n) = A (m x k) * B^T where B is n x k, row-major. */
static void matmul_nt(int m, int k, int n, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(static) if ((long)m * k * n > 200000)
    for (int i = 0; i < m; i++) {
        const double *a = A + (size_t)i * k;
        for (int j = 0; j < n; j++) {
            const double *b = B + (size_t)j * k;
            double s = 0.0;
            for (int p = 0; p < k; p++) s += a[p] * b[p];
            C[(size_t)i * n + j] = s;
        }
    }
}

static void transpose(int m, int n, const double *A, double *T)
{
    for (int i = 0; i < m; i++)
        for (int j = 0; j < n; j++) T[(size_t)j * m + i] = A[(size_t)i * n + j];
}

static double frob2(size_t len, const double *A)
{
    double s = 0.0;
    for (size_t i = 0; i < len; i++) s += A[i] * A[i];
    return s;
}

/* ------------------------------------------------------------------ */
/* shrink (soft thresholding), Sec. 2.1 and Alg. 3                     */
/* ------------------------------------------------------------------ */

/* S_theta[x] = sign(x) * max(|x| - theta, 0), elementwise. */
void or_shrink(size_t len, const double *X, double theta, double *Y)
{
    for (size_t i = 0; i < len; i++) {
        double a = fabs(X[i]) - theta;
        Y[i] = a > 0.0 ? copysign(a, X[i]) : copysign(0.0, X[i]);
    }
}

/* ------------------------------------------------------------------ */
/* one-sided Jacobi SVD                                                */
/* ------------------------------------------------------------------ */

/*
 * Orthogonalise the n columns of W (column-major, m x n) by plane rotations
 * and apply the same rotations to the columns of V (column-major, n x n).
 * Pairs are visited in round-robin order, so the pairs of one round are
 * disjoint and independent.  Returns the number of sweeps used.
 */
static int jacobi_cols(int m, int n, double *W, double *V, int max_sweeps)
{
    const double tol = (double)(m > 1 ? m : 1) * 2.220446049250313e-16;
    int N = n + (n & 1);
    int *perm = (int *)malloc(sizeof(int) * (N > 0 ? N : 1));
    for (int i = 0; i < N; i++) perm[i] = i;
    int sweep;
    for (sweep = 0; sweep < max_sweeps; sweep++) {
        long rot = 0;
        for (int round = 0; round < N - 1; round++) {
#pragma omp parallel for schedule(static) reduction(+ : rot) if ((long)m * n > 2000)
            for (int t = 0; t < N / 2; t++) {
                int p = perm[t], q = perm[N - 1 - t];
                if (p >= n || q >= n) continue;
                double *wp = W + (size_t)p * m, *wq = W + (size_t)q * m;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int i = 0; i < m; i++) {
                    a += wp[i] * wp[i];
                    b += wq[i] * wq[i];
                    g += wp[i] * wq[i];
                }
                if (a == 0.0 || b == 0.0) continue;
                if (fabs(g) <= tol * sqrt(a) * sqrt(b)) continue;
                double zeta = (b - a) / (2.0 * g);
                double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + tt * tt), s = c * tt;
                for (int i = 0; i < m; i++) {
                    double x = wp[i], y = wq[i];
                    wp[i] = c * x - s * y;
                    wq[i] = s * x + c * y;
                }
                double *vp = V + (size_t)p * n, *vq = V + (size_t)q * n;
                for (int i = 0; i < n; i++) {
                    double x = vp[i], y = vq[i];
                    vp[i] = c * x - s * y;
                    vq[i] = s * x + c * y;
                }
                rot++;
            }
            /* circle method: keep slot 0, rotate the others by one */
            if (N > 2) {
                int last = perm[N - 1];
                for (int i = N - 1; i > 1; i--) perm[i] = perm[i - 1];
                perm[1] = last;
            }
        }
        if (rot == 0) break;
    }
    free(perm);
    return sweep;
}

typedef struct {
    double s;
    int idx;
} sv_pair;

static int sv_cmp(const void *x, const void *y)
{
    const sv_pair *a = (const sv_pair *)x, *b = (const sv_pair *)y;
    if (a->s > b->s) return -1;
    if (a->s < b->s) return 1;
    return a->idx - b->idx;
}

/*
 * Thin SVD of the m x n row-major matrix A = U diag(s) V^T with p = min(m, n),
 * singular values in descending order.  U is m x p, V is n x p (row-major).
 * V0 (optional, only used when m >= n) is an n x n orthogonal matrix
 * (row-major) used as the starting rotation: Jacobi is applied to A V0, which
 * has the same singular values; the accumulated rotation still gives V.
 * Returns the number of sweeps, or -1 on allocation failure.
 */
int or_svd(int m, int n, const double *A, double *U, double *s, double *V, const double *V0)
{
    int trans = m < n;
    int mm = trans ? n : m, nn = trans ? m : n; /* work on an mm x nn matrix, mm >= nn */
    double *W = dalloc((size_t)mm * nn), *VV = dalloc((size_t)nn * nn);
    if (!W || !VV) {
        free(W);
        free(VV);
        return -1;
    }
    /* W column j = column j of (trans ? A^T : A), column-major */
    if (!trans) {
        if (V0) {
            /* W = A V0, VV = V0 (column-major: VV[j*nn + i] = V0[i][j]) */
            for (int j = 0; j < nn; j++)
                for (int i = 0; i < nn; i++) VV[(size_t)j * nn + i] = V0[(size_t)i * nn + j];
#pragma omp parallel for schedule(static) if ((long)mm * nn * nn > 200000)
            for (int j = 0; j < nn; j++)
                for (int i = 0; i < mm; i++) {
                    double acc = 0.0;
                    for (int p = 0; p < nn; p++) acc += A[(size_t)i * n + p] * VV[(size_t)j * nn + p];
                    W[(size_t)j * mm + i] = acc;
                }
        } else {
            for (int j = 0; j < nn; j++)
                for (int i = 0; i < mm; i++) W[(size_t)j * mm + i] = A[(size_t)i * n + j];
            for (int j = 0; j < nn; j++) VV[(size_t)j * nn + j] = 1.0;
        }
    } else {
        /* A^T is n x m = mm x nn; its column j is row j of A */
        for (int j = 0; j < nn; j++)
            for (int i = 0; i < mm; i++) W[(size_t)j * mm + i] = A[(size_t)j * n + i];
        for (int j = 0; j < nn; j++) VV[(size_t)j * nn + j] = 1.0;
    }
    int sweeps = jacobi_cols(mm, nn, W, VV, 60);
    sv_pair *ord = (sv_pair *)malloc(sizeof(sv_pair) * (nn > 0 ? nn : 1));
    for (int j = 0; j < nn; j++) {
        ord[j].s = sqrt(frob2((size_t)mm, W + (size_t)j * mm));
        ord[j].idx = j;
    }
    qsort(ord, (size_t)nn, sizeof(sv_pair), sv_cmp);
    /* left vectors of the worked matrix: W_j / s_j; right vectors: VV_j */
    double *Ul = trans ? V : U; /* left factor of A^T is V of A */
    double *Vr = trans ? U : V;
    int ldl = nn, ldr = nn;     /* both outputs have p = nn columns */
    for (int c = 0; c < nn; c++) {
        int j = ord[c].idx;
        double sj = ord[c].s;
        s[c] = sj;
        for (int i = 0; i < mm; i++) Ul[(size_t)i * ldl + c] = sj > 0.0 ? W[(size_t)j * mm + i] / sj : 0.0;
        for (int i = 0; i < nn; i++) Vr[(size_t)i * ldr + c] = VV[(size_t)j * nn + i];
    }
    free(ord);
    free(W);
    free(VV);
    return sweeps;
}

/* ------------------------------------------------------------------ */
/* singular value thresholding, Sec. 2.1 (Alg. 1) and Sec. 3.2         */
/* ------------------------------------------------------------------ */

/*
 * L = U S_theta[Sigma] V^T of the m x n matrix M; returns the rank kept
 * (singular values strictly above theta).  If nuc is non-NULL it receives the
 * nuclear norm of L.  Vwarm (optional, n x n row-major, m >= n only) is used
 * as the Jacobi starting rotation and overwritten with the new right vectors.
 */
int or_svt(int m, int n, const double *M, double theta, double *L, double *nuc, double *Vwarm)
{
    int p = m < n ? m : n;
    double *U = dalloc((size_t)m * p), *s = dalloc((size_t)p), *V = dalloc((size_t)n * p);
    int use_warm = (Vwarm != NULL) && (m >= n);
    or_svd(m, n, M, U, s, V, use_warm ? Vwarm : NULL);
    int r = 0;
    double nn = 0.0;
    while (r < p && s[r] > theta) {
        nn += s[r] - theta;
        r++;
    }
    /* L = (U_r diag(s - theta)) V_r^T */
    double *A = dalloc((size_t)m * (r ? r : 1)), *B = dalloc((size_t)n * (r ? r : 1));
    for (int i = 0; i < m; i++)
        for (int c = 0; c < r; c++) A[(size_t)i * r + c] = U[(size_t)i * p + c] * (s[c] - theta);
    for (int i = 0; i < n; i++)
        for (int c = 0; c < r; c++) B[(size_t)i * r + c] = V[(size_t)i * p + c];
    if (r > 0)
        matmul_nt(m, r, n, A, B, L);
    else
        memset(L, 0, sizeof(double) * (size_t)m * n);
    if (use_warm) memcpy(Vwarm, V, sizeof(double) * (size_t)n * n);
    if (nuc) *nuc = nn;
    free(A);
    free(B);
    free(U);
    free(s);
    free(V);
    return r;
}

/* ------------------------------------------------------------------ */
/* interpolation operator R_n, eq. (Rx) and its worked example         */
/* ------------------------------------------------------------------ */

/* coarse size of one level: n/2 for even n, (n+1)/2 for odd n */
int or_coarse_size(int n) { return (n + 1) / 2; }

/*
 * One level, n x nh (row-major), nh = or_coarse_size(n).  Rows are indexed
 * 1-based as in the worked example of Sec. 3.1:
 *   even n: row 1 = e_1; row 2j = e_j; row 2j+1 = (e_j + e_{j+1}) / 2
 *   odd n : row 2j-1 = e_j; row 2j = (e_j + e_{j+1}) / 2
 */
void or_interp_level(int n, double *R)
{
    int nh = or_coarse_size(n);
    memset(R, 0, sizeof(double) * (size_t)n * nh);
    for (int I = 1; I <= n; I++) {
        double *row = R + (size_t)(I - 1) * nh;
        if (n % 2 == 0) {
            if (I == 1) {
                row[0] = 1.0;
            } else if (I % 2 == 0) {
                row[I / 2 - 1] = 1.0;
            } else {
                int j = (I - 1) / 2;
                row[j - 1] = 0.5;
                row[j] = 0.5;
            }
        } else {
            if (I % 2 == 1) {
                row[(I + 1) / 2 - 1] = 1.0;
            } else {
                int j = I / 2;
                row[j - 1] = 0.5;
                row[j] = 0.5;
            }
        }
    }
}

/* coarse size after `halvings` levels */
int or_coarse_dim(int n, int halvings)
{
    for (int h = 0; h < halvings; h++) n = or_coarse_size(n);
    return n;
}

/*
 * Composite R = R_n R_{n_1} ... R_{n_H} (Sec. 3.1), n x nH row-major, as the
 * explicit product of the per-level matrices.  halvings = levels - 1.
 */
int or_restriction(int n, int halvings, double *R)
{
    int cur = n;
    double *P = dalloc((size_t)n * n); /* current product, n x cur */
    for (int i = 0; i < n; i++) P[(size_t)i * n + i] = 1.0;
    for (int h = 0; h < halvings; h++) {
        int nh = or_coarse_size(cur);
        double *Rl = dalloc((size_t)cur * nh), *Q = dalloc((size_t)n * nh);
        or_interp_level(cur, Rl);
        matmul(n, cur, nh, P, Rl, Q);
        free(P);
        free(Rl);
        P = Q;
        cur = nh;
    }
    memcpy(R, P, sizeof(double) * (size_t)n * cur);
    free(P);
    return cur;
}

/* Largest singular value of a row-major m x n matrix (Jacobi SVD). */
double or_spectral_norm(int m, int n, const double *A)
{
    int p = m < n ? m : n;
    double *U = dalloc((size_t)m * p), *s = dalloc((size_t)p), *V = dalloc((size_t)n * p);
    or_svd(m, n, A, U, s, V, NULL);
    double r = p > 0 ? s[0] : 0.0;
    free(U);
    free(s);
    free(V);
    return r;
}

/* R scaled to unit spectral norm (Assumption 4 read as ||R||_2 = 1). */
int or_restriction_scaled(int n, int halvings, double *R, double *scale_out)
{
    int nh = or_restriction(n, halvings, R);
    double nr = or_spectral_norm(n, nh, R);
    for (size_t i = 0; i < (size_t)n * nh; i++) R[i] /= nr;
    if (scale_out) *scale_out = 1.0 / nr;
    return nh;
}

/*
 * R_o = R_p (R_p^T R_p)^{-1/2} with R_p the composite interpolation of
 * Sec. 3.1 (unscaled): orthonormal columns spanning the range of R_p, so
 * R_o R_o^T is the orthogonal projector onto that range.  Theorem LH-eps
 * gives epsilon = 0 for such an R (its singular values are all 1); the paper
 * sets it aside as dense.  (R_p^T R_p)^{-1/2} comes from the SVD of the
 * symmetric positive definite R_p^T R_p, which is its eigendecomposition:
 * V diag(s^{-1/2}) V^T.  Returns n_H, or -1 on allocation failure.
 */
int or_restriction_orth(int n, int halvings, double *R)
{
    int nh = or_restriction(n, halvings, R);
    double *G = dalloc((size_t)nh * nh), *U = dalloc((size_t)nh * nh), *sv = dalloc((size_t)nh),
           *V = dalloc((size_t)nh * nh), *W = dalloc((size_t)nh * nh), *Ro = dalloc((size_t)n * nh);
    if (!G || !U || !sv || !V || !W || !Ro) {
        free(G), free(U), free(sv), free(V), free(W), free(Ro);
        return -1;
    }
    for (int a = 0; a < nh; a++)
        for (int b = 0; b < nh; b++) {
            double t = 0.0;
            for (int j = 0; j < n; j++) t += R[(size_t)j * nh + a] * R[(size_t)j * nh + b];
            G[(size_t)a * nh + b] = t;
        }
    or_svd(nh, nh, G, U, sv, V, NULL);
    for (int a = 0; a < nh; a++)
        for (int b = 0; b < nh; b++) {
            double t = 0.0;
            for (int c = 0; c < nh; c++) t += V[(size_t)a * nh + c] * V[(size_t)b * nh + c] / sqrt(sv[c]);
            W[(size_t)a * nh + b] = t;
        }
    matmul(n, nh, nh, R, W, Ro);
    memcpy(R, Ro, sizeof(double) * (size_t)n * nh);
    free(G), free(U), free(sv), free(V), free(W), free(Ro);
    return nh;
}

/* ------------------------------------------------------------------ */
/* objective and gradient, eq. (cpcp) and eq. (cpcp-grad-LS)           */
/* ------------------------------------------------------------------ */

/* G = P_Q[L + S - D]  (mask NULL = all observed) */
void or_grad(int m, int n, const double *D, const unsigned char *mask, const double *L, const double *S,
             double *G)
{
    size_t len = (size_t)m * n;
    for (size_t i = 0; i < len; i++) G[i] = (!mask || mask[i]) ? (L[i] + S[i] - D[i]) : 0.0;
}

double or_nuclear_norm(int m, int n, const double *A)
{
    int p = m < n ? m : n;
    double *U = dalloc((size_t)m * p), *s = dalloc((size_t)p), *V = dalloc((size_t)n * p);
    or_svd(m, n, A, U, s, V, NULL);
    double r = 0.0;
    for (int i = 0; i < p; i++) r += s[i];
    free(U);
    free(s);
    free(V);
    return r;
}

/* 1/2 ||P_Q[L+S-D]||_F^2 + mu ||L||_* + lam mu ||S||_1 */
double or_objective(int m, int n, const double *D, const unsigned char *mask, double lam, double mu,
                    const double *L, const double *S)
{
    size_t len = (size_t)m * n;
    double *G = dalloc(len);
    or_grad(m, n, D, mask, L, S, G);
    double f = 0.5 * frob2(len, G);
    double l1 = 0.0;
    for (size_t i = 0; i < len; i++) l1 += fabs(S[i]);
    f += mu * or_nuclear_norm(m, n, L) + lam * mu * l1;
    free(G);
    return f;
}

/*
 * Relative gradient-mapping residual at (L, S) for weights (mu, lam mu) and
 * step tau: || (L - SVT_{tau mu}(L - tau G), S - shrink_{tau lam mu}(S - tau G)) ||_F
 * / tau / ||P_Q D||_F with G = P_Q[L + S - D].  Zero iff (L, S) minimises
 * eq. (cpcp).  Full SVD on the fine level.
 */
static double relkkt_warm(int m, int n, const double *D, const unsigned char *mask, double lam, double mu,
                          double tau, const double *L, const double *S, double *Vwarm)
{
    size_t len = (size_t)m * n;
    double *G = dalloc(len), *X = dalloc(len), *Y = dalloc(len);
    or_grad(m, n, D, mask, L, S, G);
    for (size_t i = 0; i < len; i++) X[i] = L[i] - tau * G[i];
    or_svt(m, n, X, tau * mu, Y, NULL, Vwarm);
    double r2 = 0.0;
    for (size_t i = 0; i < len; i++) r2 += (L[i] - Y[i]) * (L[i] - Y[i]);
    for (size_t i = 0; i < len; i++) X[i] = S[i] - tau * G[i];
    or_shrink(len, X, tau * lam * mu, Y);
    for (size_t i = 0; i < len; i++) r2 += (S[i] - Y[i]) * (S[i] - Y[i]);
    double pqd = 0.0;
    for (size_t i = 0; i < len; i++)
        if (!mask || mask[i]) pqd += D[i] * D[i];
    free(G);
    free(X);
    free(Y);
    return sqrt(r2) / tau / sqrt(pqd);
}

double or_relkkt(int m, int n, const double *D, const unsigned char *mask, double lam, double mu, double tau,
                 const double *L, const double *S)
{
    return relkkt_warm(m, n, D, mask, lam, mu, tau, L, S, NULL);
}

/* ------------------------------------------------------------------ */
/* accelerated proximal gradient with the multilevel L-prox            */
/* ------------------------------------------------------------------ */

typedef struct {
    double tau;          /* step size, 1/2 (gradient is 2-Lipschitz, Sec. 2.3) */
    double eta;          /* continuation factor */
    double mu0;          /* first weight; <= 0 means ||P_Q D||_2 */
    int check_every;     /* c: iterations between fine-level residual checks */
    int max_iter;        /* iteration cap */
    double switch_ratio; /* move finer when rel-KKT > ratio * previous check */
    int start_level;     /* halvings to start at; < 0 means levels - 1 */
    int fixed_iters;     /* > 0: run exactly this many iterations at start_level, no checks */
    int transfer;        /* 0: R scaled to unit norm (Assumption 4); 1: R (R^T R)^{-1/2} (orthonormal
                            columns, the same range; or_restriction_orth) */
    int early_test;      /* nonzero: the coarse-gradient test also runs after the first iteration on
                            each coarse level (a study of an alternative to the level rule) */
} or_opts;

typedef struct {
    int iters;
    int final_level;
    int rank;
    int checks;
    int status;
    double relkkt;
    double objective;
    int level_iters[16];
} or_info;

/*
 * Prox of mu_k ||.||_* composed with the transfer operators: with M (m x n),
 * M_H = M R, L_H = SVT_theta(M_H), L = L_H R^T.  R = NULL means level 0
 * (L = SVT_theta(M)).  Returns the rank.  Vw: warm rotation (nh x nh).
 */
static int ml_prox_L(int m, int n, int nh, const double *R, const double *M, double theta, double *L, double *Vw)
{
    if (!R) return or_svt(m, n, M, theta, L, NULL, Vw);
    double *MH = dalloc((size_t)m * nh), *LH = dalloc((size_t)m * nh);
    matmul(m, n, nh, M, R, MH);           /* restriction M R       */
    int r = or_svt(m, nh, MH, theta, LH, NULL, Vw); /* coarse SVT   */
    matmul_nt(m, nh, n, LH, R, L);       /* prolongation L_H R^T  */
    free(MH);
    free(LH);
    return r;
}

/*
 * Threshold of the coarse-gradient test for one level: the geometric mean of
 * the ratio ||g R|| / ||g|| that a row of white noise gets on average
 * (||R||_F / sqrt(n)) and the ratio that a row constant along the columns gets
 * (||1^T R|| / sqrt(n)).  A gradient whose restriction keeps less than this
 * share of its norm is dominated by fine-scale components that the coarse
 * model cannot represent.
 */
double or_restriction_kappa(int n, int nh, const double *R)
{
    double fro2 = 0.0, cs2 = 0.0;
    for (int c = 0; c < nh; c++) {
        double cs = 0.0;
        for (int j = 0; j < n; j++) {
            double r = R[(size_t)j * nh + c];
            fro2 += r * r;
            cs += r;
        }
        cs2 += cs * cs;
    }
    return sqrt(sqrt(fro2 / n) * sqrt(cs2 / n));
}

static int fista_core(int m, int n, const double *D, const unsigned char *mask, double lam, double mu_bar,
                      int levels, double tol, const or_opts *o, double *L, double *S, or_info *info,
                      double *trace, int trace_cap)
{
    size_t len = (size_t)m * n;
    int H = levels - 1;
    double tau = o->tau > 0 ? o->tau : 0.5;
    double eta = o->eta > 0 ? o->eta : 0.9;
    int c = o->check_every > 0 ? o->check_every : 10;
    int max_iter = o->max_iter > 0 ? o->max_iter : 5000;
    double ratio = o->switch_ratio > 0 ? o->switch_ratio : 0.9;
    int level = o->start_level >= 0 ? o->start_level : H;
    if (level > H) level = H;
    int level_start = 0; /* iteration at which the current level began */

    /* restriction operators for every level (level 0 = identity) */
    double **R = (double **)calloc((size_t)H + 1, sizeof(double *));
    int *nhs = (int *)calloc((size_t)H + 1, sizeof(int));
    nhs[0] = n;
    for (int h = 1; h <= H; h++) {
        nhs[h] = or_coarse_dim(n, h);
        R[h] = dalloc((size_t)n * nhs[h]);
        if (o->transfer == 1)
            or_restriction_orth(n, h, R[h]);
        else
            or_restriction_scaled(n, h, R[h], NULL);
    }
    double *kappa = dalloc((size_t)H + 1);
    for (int h = 1; h <= H; h++) kappa[h] = or_restriction_kappa(n, nhs[h], R[h]);
    double *GR = H > 0 ? dalloc((size_t)m * nhs[1]) : NULL;
    double **Vw = (double **)calloc((size_t)H + 1, sizeof(double *));
    for (int h = 0; h <= H; h++) {
        if (m >= nhs[h]) {
            Vw[h] = dalloc((size_t)nhs[h] * nhs[h]);
            for (int i = 0; i < nhs[h]; i++) Vw[h][(size_t)i * nhs[h] + i] = 1.0;
        }
    }

    double *Vchk = dalloc((size_t)n * n); /* warm rotation of the fine residual SVD */
    for (int i = 0; i < n; i++) Vchk[(size_t)i * n + i] = 1.0;
    double *PQD = dalloc(len);
    for (size_t i = 0; i < len; i++) PQD[i] = (!mask || mask[i]) ? D[i] : 0.0;
    double mu0 = o->mu0 > 0 ? o->mu0 : or_spectral_norm(m, n, PQD);

    double *Lp = dalloc(len), *Sp = dalloc(len), *Lh = dalloc(len), *Sh = dalloc(len), *G = dalloc(len),
           *X = dalloc(len), *Ln = dalloc(len), *Sn = dalloc(len);
    memset(L, 0, sizeof(double) * len);
    memset(S, 0, sizeof(double) * len);
    double t = 1.0, mu_k = mu0, prev = INFINITY, rel = INFINITY;
    int k, rank = 0, status = OR_NOTCONV, checks = 0;
    if (info) memset(info->level_iters, 0, sizeof(info->level_iters));
    for (k = 0; k < max_iter; k++) {
        mu_k = mu0 * pow(eta, (double)k);
        if (mu_k < mu_bar) mu_k = mu_bar;
        double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        double beta = (t - 1.0) / t1;
        /* extrapolation */
        for (size_t i = 0; i < len; i++) {
            Lh[i] = L[i] + beta * (L[i] - Lp[i]);
            Sh[i] = S[i] + beta * (S[i] - Sp[i]);
        }
        or_grad(m, n, D, mask, Lh, Sh, G);
        /* S-prox: shrink with threshold tau lam mu_k */
        for (size_t i = 0; i < len; i++) X[i] = Sh[i] - tau * G[i];
        or_shrink(len, X, tau * lam * mu_k, Sn);
        /* L-prox on the current level */
        for (size_t i = 0; i < len; i++) X[i] = Lh[i] - tau * G[i];
        rank = ml_prox_L(m, n, nhs[level], level ? R[level] : NULL, X, tau * mu_k, Ln, Vw[level]);
        memcpy(Lp, L, sizeof(double) * len);
        memcpy(Sp, S, sizeof(double) * len);
        memcpy(L, Ln, sizeof(double) * len);
        memcpy(S, Sn, sizeof(double) * len);
        t = t1;
        if (info && level < 16) info->level_iters[level]++;
        if (o->fixed_iters > 0) {
            if (k + 1 >= o->fixed_iters) {
                k++;
                status = OR_OK;
                break;
            }
            continue;
        }
        /* decisions: every c iterations, and with early_test also at a coarse
           level's first iteration (the coarse-gradient test only) */
        const int periodic = (k + 1) % c == 0;
        const int early = o->early_test && level > 0 && k == level_start;
        if (!periodic && !early) continue;
        int finer = 0;
        if (level > 0) {
            /* coarse-gradient test: keep the coarse model while the
               restricted gradient G R carries at least kappa of ||G|| */
            matmul(m, n, nhs[level], G, R[level], GR);
            double gn = sqrt(frob2(len, G)), grn = sqrt(frob2((size_t)m * nhs[level], GR));
            if (gn > 0.0 && grn < kappa[level] * gn) finer = 1;
        }
        if (periodic && !finer && mu_k == mu_bar) {
            /* fine residual at the final weight: stop test, and on a coarse
               level a stall test */
            rel = relkkt_warm(m, n, D, mask, lam, mu_bar, tau, L, S, Vchk);
            if (trace && checks < trace_cap) trace[checks] = rel;
            checks++;
            if (rel <= tol) {
                k++;
                status = OR_OK;
                break;
            }
            if (level > 0 && rel > ratio * prev) finer = 1;
            prev = rel;
        }
        if (finer) {
            level--;
            level_start = k + 1;
            prev = INFINITY;
            t = 1.0; /* momentum restart */
            memcpy(Lp, L, sizeof(double) * len);
            memcpy(Sp, S, sizeof(double) * len);
        }
    }
    if (info) {
        info->iters = k;
        info->final_level = level;
        info->rank = rank;
        info->checks = checks;
        info->status = status;
        info->relkkt = rel;
        info->objective = or_objective(m, n, D, mask, lam, mu_bar, L, S);
    }
    for (int h = 0; h <= H; h++) {
        free(R[h]);
        free(Vw[h]);
    }
    free(R);
    free(Vw);
    free(nhs);
    free(kappa);
    free(GR);
    free(Vchk);
    free(PQD);
    free(Lp);
    free(Sp);
    free(Lh);
    free(Sh);
    free(G);
    free(X);
    free(Ln);
    free(Sn);
    return status;
}

/*
 * One step of the iteration above from an explicit state, with dense L:
 *   Lhat = L_k + beta (L_k - L_p), Shat = S_k + beta (S_k - S_p)
 *   G = P_Q[Lhat + Shat - D]                         eq. (cpcp-grad-LS)
 *   S_out = shrink_{tau lam mu_k}(Shat - tau G)       Alg. 3 threshold
 *   L_out = SVT_{tau mu_k}((Lhat - tau G) R) R^T       Alg. 4 (R = I if halvings = 0)
 * Returns the rank of the coarse SVT.  Requires n <= m.
 */
int or_step(int m, int n, const double *D, const unsigned char *mask, double lam, double mu_k, double beta,
            int halvings, const double *Sk, const double *Sp, const double *Lk, const double *Lp, double *S_out,
            double *L_out)
{
    const double tau = 0.5;
    size_t len = (size_t)m * n;
    int nh = or_coarse_dim(n, halvings);
    double *R = NULL;
    if (halvings > 0) {
        R = dalloc((size_t)n * nh);
        or_restriction_scaled(n, halvings, R, NULL);
    }
    double *Lh = dalloc(len), *Sh = dalloc(len), *G = dalloc(len), *X = dalloc(len);
    for (size_t i = 0; i < len; i++) {
        Lh[i] = Lk[i] + beta * (Lk[i] - Lp[i]);
        Sh[i] = Sk[i] + beta * (Sk[i] - Sp[i]);
    }
    or_grad(m, n, D, mask, Lh, Sh, G);
    for (size_t i = 0; i < len; i++) X[i] = Sh[i] - tau * G[i];
    or_shrink(len, X, tau * lam * mu_k, S_out);
    for (size_t i = 0; i < len; i++) X[i] = Lh[i] - tau * G[i];
    int r = ml_prox_L(m, n, nh, R, X, tau * mu_k, L_out, NULL);
    free(R);
    free(Lh);
    free(Sh);
    free(G);
    free(X);
    return r;
}

/*
 * Solve eq. (cpcp) with lambda_L = mu_bar and lambda_S = lam * mu_bar.
 * D (m x n) row-major; mask (m x n bytes, nonzero = observed) or NULL.
 * levels >= 1 (1 = single level).  If n > m the transposed problem is solved
 * and the results transposed back (the restriction then acts on the rows).
 */
int or_fista(int m, int n, const double *D, const unsigned char *mask, double lam, double mu_bar, int levels,
             double tol, const or_opts *o, double *L, double *S, or_info *info, double *trace, int trace_cap)
{
    if (m < 1 || n < 1 || levels < 1 || !(lam > 0) || !(mu_bar > 0) || !D || !L || !S) return OR_EINVAL;
    if (n <= m) return fista_core(m, n, D, mask, lam, mu_bar, levels, tol, o, L, S, info, trace, trace_cap);
    size_t len = (size_t)m * n;
    double *Dt = dalloc(len), *Lt = dalloc(len), *St = dalloc(len);
    unsigned char *Mt = NULL;
    transpose(m, n, D, Dt);
    if (mask) {
        Mt = (unsigned char *)malloc(len);
        for (int i = 0; i < m; i++)
            for (int j = 0; j < n; j++) Mt[(size_t)j * m + i] = mask[(size_t)i * n + j];
    }
    int st = fista_core(n, m, Dt, Mt, lam, mu_bar, levels, tol, o, Lt, St, info, trace, trace_cap);
    transpose(n, m, Lt, L);
    transpose(n, m, St, S);
    free(Dt);
    free(Lt);
    free(St);
    free(Mt);
    return st;
}

/* ------------------------------------------------------------------ */
/* paper-literal IALM (Alg. 1) and ML-IALM (Alg. 4) for eq. (rpca)     */
/* ------------------------------------------------------------------ */

/*
 * Alg. 1 (levels == 1) or Alg. 4 (levels > 1) with the transfer operator
 * `transfer`: 0 = R scaled to unit spectral norm (the reading of Assumption
 * 4), 1 = R_o of or_restriction_orth, 2 = the printed R unscaled:
 *   M   = D - S + Y / mu_k              (ML: M_H = M R)
 *   L   = U S_{1/mu_k}[Sigma] V^T        (ML: L = L_H R^T)
 *   S   = S_{lam/mu_k}[D - L + Y / mu_k]
 *   Y  += mu_k (D - L - S)
 * with S_0 = Y_0 = 0.  Penalty schedule: rho > 1 gives mu_{k+1} = rho mu_k,
 * otherwise mu_k = mu0 (1 + k) (non-decreasing, sum 1/mu_k = inf,
 * sum 1/mu_k^2 < inf, as Theorems 1 and 3 require).  mu0 <= 0 means
 * 1.25 / ||D||_2.  Stops when the feasibility gap ||D-L-S||_F/||D||_F <= tol.
 * fg (optional) receives the gap after each iteration.  Returns iterations.
 */
int or_ialm_ex(int m, int n, const double *D, double lam, int levels, double mu0, double rho, int max_iter,
               double tol, double *L, double *S, double *fg, double *final_fg, int transfer)
{
    if (n > m) return -1; /* the column restriction needs n <= m */
    size_t len = (size_t)m * n;
    int H = levels - 1;
    int nh = or_coarse_dim(n, H);
    double *R = NULL;
    if (H > 0) {
        R = dalloc((size_t)n * nh);
        if (transfer == 1)
            or_restriction_orth(n, H, R);
        else if (transfer == 2)
            or_restriction(n, H, R);
        else
            or_restriction_scaled(n, H, R, NULL);
    }
    double *Y = dalloc(len), *M = dalloc(len), *Vw = dalloc((size_t)nh * nh);
    for (int i = 0; i < nh; i++) Vw[(size_t)i * nh + i] = 1.0;
    if (!(mu0 > 0)) mu0 = 1.25 / or_spectral_norm(m, n, D);
    double nD = sqrt(frob2(len, D));
    memset(L, 0, sizeof(double) * len);
    memset(S, 0, sizeof(double) * len);
    double mu = mu0, gap = INFINITY;
    int k;
    for (k = 0; k < max_iter; k++) {
        for (size_t i = 0; i < len; i++) M[i] = D[i] - S[i] + Y[i] / mu;
        ml_prox_L(m, n, nh, R, M, 1.0 / mu, L, Vw);
        for (size_t i = 0; i < len; i++) M[i] = D[i] - L[i] + Y[i] / mu;
        or_shrink(len, M, lam / mu, S);
        double g2 = 0.0;
        for (size_t i = 0; i < len; i++) {
            double e = D[i] - L[i] - S[i];
            Y[i] += mu * e;
            g2 += e * e;
        }
        gap = sqrt(g2) / nD;
        if (fg) fg[k] = gap;
        mu = rho > 1.0 ? mu * rho : mu0 * (double)(k + 2);
        if (gap <= tol) {
            k++;
            break;
        }
    }
    if (final_fg) *final_fg = gap;
    free(R);
    free(Y);
    free(M);
    free(Vw);
    return k;
}

int or_ialm(int m, int n, const double *D, double lam, int levels, double mu0, double rho, int max_iter,
            double tol, double *L, double *S, double *fg, double *final_fg)
{
    return or_ialm_ex(m, n, D, lam, levels, mu0, rho, max_iter, tol, L, S, fg, final_fg, 0);
}

/* ------------------------------------------------------------------ */
/* Frank-Wolfe Thresholding (Alg. 3) and its multilevel form (Alg. 6)  */
/* ------------------------------------------------------------------ */

static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/*
 * Exact minimiser over [0,1]^2 of the convex quadratic
 *     q(a, b) = 1/2 (A a^2 + 2 C a b + B b^2) + ga a + gb b,
 * the line search of Alg. 3 over the two segments [(L, t_L), (V_L, V_tL)]
 * and [(S, t_S), (V_S, V_tS)]: A = ||P_Q[V_L - L]||^2, B = ||P_Q[V_S - S]||^2,
 * C their inner product, ga and gb the derivatives of the objective along the
 * segments at a = b = 0.  Candidates: the stationary point when it lies in
 * the box, and the exact minimiser on each of the four edges; the smallest
 * value wins (the minimiser of a convex function on a box is one of them).
 */
void or_fw_line_search(double A, double B, double C, double ga, double gb, double *a_out, double *b_out)
{
    double best = INFINITY, ba = 0.0, bb = 0.0;
    double ca[6], cb[6];
    int nc = 0;
    const double det = A * B - C * C;
    if (det > 0.0) {
        const double a = (-ga * B + gb * C) / det, b = (-gb * A + ga * C) / det;
        if (a >= 0.0 && a <= 1.0 && b >= 0.0 && b <= 1.0) {
            ca[nc] = a;
            cb[nc++] = b;
        }
    }
    for (int e = 0; e < 2; e++) {
        /* edge a = e: minimise 1/2 B b^2 + (gb + C e) b */
        const double lin = gb + C * e;
        ca[nc] = e;
        cb[nc++] = B > 0.0 ? clamp01(-lin / B) : (lin < 0.0 ? 1.0 : 0.0);
        /* edge b = e */
        const double lin2 = ga + C * e;
        ca[nc] = A > 0.0 ? clamp01(-lin2 / A) : (lin2 < 0.0 ? 1.0 : 0.0);
        cb[nc++] = e;
    }
    for (int i = 0; i < nc; i++) {
        const double a = ca[i], b = cb[i];
        const double q = 0.5 * (A * a * a + 2.0 * C * a * b + B * b * b) + ga * a + gb * b;
        if (q < best) {
            best = q;
            ba = a;
            bb = b;
        }
    }
    *a_out = ba;
    *b_out = bb;
}

/*
 * FW-T (Alg. 3; levels == 1) and ML-FWT (Alg. 6; levels > 1) for eq. (cpcp)
 * with lambda_L = mu and lambda_S = lam mu, in the epigraph form of
 * eq. (cpcp-fw): f = 1/2 ||P_Q[L + S - D]||_F^2 + lambda_L t_L + lambda_S t_S,
 * ||L||_* <= t_L <= U_L, ||S||_1 <= t_S <= U_S.  Per iteration, with
 * G = P_Q[L + S - D]:
 *   - nuclear-ball LMO: M_L = -u v^T for the top singular pair (u, v) of G;
 *     multilevel: the top pair (u, v_H) of G R and M_L = -u (R v_H)^T, the
 *     coarse ball of radius 1 / ||R|| = 1 (R scaled to unit norm) lifted by
 *     R^T (Sec. 3.4); <G, M_L> = -sigma_1 either way.  transfer = 1 (or_fwt_ex)
 *     takes R (R^T R)^{-1/2} instead, whose lifted vertices have nuclear norm 1;
 *   - l1-ball LMO: M_S = -sign(G_ij) e_i e_j^T at the largest |G_ij|;
 *   - V_L = U_L M_L, V_tL = U_L unless lambda_L >= sigma_1 (then 0), and
 *     likewise V_S, V_tS against max |G_ij| (with a relative margin, below);
 *   - exact line search over the two segments (or_fw_line_search);
 *   - thresholding: S = shrink_{lambda_S}(S - P_Q[L + S - D]) with the new L
 *     (the step of unit length of the S-block, whose gradient is 1-Lipschitz),
 *     t_S = ||S||_1;
 *   - bounds U_L = f / lambda_L, U_S = f / lambda_S at the new point.
 * Starts from L = S = 0, t_L = t_S = 0, U = f_0 / lambda.  Stops when the
 * relative objective decrease |f_{k-1} - f_k| <= tol f_{k-1} (the paper's
 * 10^-3 criterion, taken from the FW-T reference it cites) or after
 * max_iter iterations.  ftrace (optional) receives f after each iteration;
 * tl_ts (optional) the final t_L, t_S.  Returns the iterations taken.
 */
int or_fwt_ex(int m, int n, const double *D, const unsigned char *mask, double lam, double mu, int levels,
              int max_iter, double tol, double *L, double *S, double *ftrace, double *tl_ts, int transfer)
{
    const size_t len = (size_t)m * n;
    const double lamL = mu, lamS = lam * mu;
    const int H = levels - 1;
    const int nh = or_coarse_dim(n, H);
    double *R = NULL, *GR = NULL;
    if (H > 0) {
        R = dalloc((size_t)n * nh);
        GR = dalloc((size_t)m * nh);
        if (transfer == 1)
            or_restriction_orth(n, H, R); /* lifted vertices on the unit nuclear sphere */
        else
            or_restriction_scaled(n, H, R, NULL);
    }
    const int nc = H > 0 ? nh : n;
    const int p = m < nc ? m : nc;
    double *G = dalloc(len), *PA = dalloc(len), *PB = dalloc(len), *U = dalloc((size_t)m * p),
           *sv = dalloc((size_t)p), *V = dalloc((size_t)nc * p), *v = dalloc((size_t)n), *u = dalloc((size_t)m);
    memset(L, 0, sizeof(double) * len);
    memset(S, 0, sizeof(double) * len);
    double tL = 0.0, tS = 0.0;
    or_grad(m, n, D, mask, L, S, G);
    double f = 0.5 * frob2(len, G);
    double UL = f / lamL, US = f / lamS;
    int k;
    for (k = 0; k < max_iter; k++) {
        const double fprev = f;
        or_grad(m, n, D, mask, L, S, G);
        /* nuclear-ball LMO (fine, or coarse and lifted) */
        if (H > 0) {
            matmul(m, n, nh, G, R, GR);
            or_svd(m, nh, GR, U, sv, V, NULL);
        } else {
            or_svd(m, n, G, U, sv, V, NULL);
        }
        const double sig = sv[0];
        for (int i = 0; i < m; i++) u[i] = U[(size_t)i * p];
        if (H > 0) {
            for (int j = 0; j < n; j++) {
                double t = 0.0;
                for (int c = 0; c < nh; c++) t += R[(size_t)j * nh + c] * V[(size_t)c * p];
                v[j] = t;
            }
        } else {
            for (int j = 0; j < n; j++) v[j] = V[(size_t)j * p];
        }
        const int useL = lamL < sig;
        const double VtL = useL ? UL : 0.0;
        /* l1-ball LMO: the first entry of largest magnitude */
        size_t imax = 0;
        double gmax = -1.0;
        for (size_t i = 0; i < len; i++)
            if (fabs(G[i]) > gmax) {
                gmax = fabs(G[i]);
                imax = i;
            }
        /* after a thresholding step every entry of the support of S has
         * |G_ij| = lambda_S exactly (and the others |G_ij| <= lambda_S), so the
         * test lambda_S >= max |G_ij| is taken with a relative margin of 1e-12:
         * without it rounding would decide it */
        const int useS = lamS * (1.0 + 1e-12) < gmax;
        const double VtS = useS ? US : 0.0;
        const double vs = useS ? -US * (G[imax] > 0.0 ? 1.0 : -1.0) : 0.0;
        /* directions P_Q[V_L - L], P_Q[V_S - S] and the quadratic's coefficients */
        double A = 0.0, B = 0.0, Cq = 0.0, ga = 0.0, gb = 0.0;
        for (int i = 0; i < m; i++)
            for (int j = 0; j < n; j++) {
                const size_t q = (size_t)i * n + j;
                const int obs = !mask || mask[q];
                const double vl = useL ? -UL * u[i] * v[j] : 0.0;
                const double vsq = q == imax ? vs : 0.0;
                PA[q] = vl - L[q];
                PB[q] = vsq - S[q];
                if (obs) {
                    A += PA[q] * PA[q];
                    B += PB[q] * PB[q];
                    Cq += PA[q] * PB[q];
                    ga += G[q] * PA[q];
                    gb += G[q] * PB[q];
                }
            }
        ga += lamL * (VtL - tL);
        gb += lamS * (VtS - tS);
        double a, b;
        or_fw_line_search(A, B, Cq, ga, gb, &a, &b);
        for (size_t q = 0; q < len; q++) {
            L[q] += a * PA[q];
            S[q] += b * PB[q];
        }
        tL += a * (VtL - tL);
        tS += b * (VtS - tS);
        /* thresholding step of the S-block, then t_S = ||S||_1 */
        or_grad(m, n, D, mask, L, S, G);
        for (size_t q = 0; q < len; q++) PB[q] = S[q] - G[q];
        or_shrink(len, PB, lamS, S);
        tS = 0.0;
        for (size_t q = 0; q < len; q++) tS += fabs(S[q]);
        or_grad(m, n, D, mask, L, S, G);
        f = 0.5 * frob2(len, G) + lamL * tL + lamS * tS;
        UL = f / lamL;
        US = f / lamS;
        if (ftrace) ftrace[k] = f;
        if (fabs(fprev - f) <= tol * fprev) {
            k++;
            break;
        }
    }
    if (tl_ts) {
        tl_ts[0] = tL;
        tl_ts[1] = tS;
    }
    free(R), free(GR), free(G), free(PA), free(PB), free(U), free(sv), free(V), free(v), free(u);
    return k;
}

int or_fwt(int m, int n, const double *D, const unsigned char *mask, double lam, double mu, int levels,
           int max_iter, double tol, double *L, double *S, double *ftrace, double *tl_ts)
{
    return or_fwt_ex(m, n, D, mask, lam, mu, levels, max_iter, tol, L, S, ftrace, tl_ts, 0);
}

/* Thread count the oracle uses (for reporting the CPU baseline). */
int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Sets the thread count of the oracle's parallel loops (for the single-thread
 * CPU baseline); n < 1 restores the default. */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    static int dflt = 0;
    if (dflt == 0) dflt = omp_get_max_threads();
    omp_set_num_threads(n >= 1 ? n : dflt);
#else
    (void)n;
#endif
}
