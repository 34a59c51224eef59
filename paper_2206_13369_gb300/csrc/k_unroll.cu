// k_unroll.cu -- kernels of the unrolled (differentiable) multilevel iteration
// and of its reverse sweep.
//
// The differentiated program is K steps of the accelerated proximal step at a
// fixed level (Alg. 4 coarse step with an exact SVT, Alg. 3 shrink, FISTA
// momentum, continuation mu_k = mu max(rho eta^k, 1)); it keeps L_k, S_k
// dense.  Its reverse sweep needs, per step,
//
//   the elementwise step and its adjoint (momentum, P_Q gradient, shrink),
//   the exact thin SVD of M_H (one-sided Jacobi over every column pair: a
//     cooperative launch whose CTAs meet at a bounded grid barrier after each
//     round of the round-robin ordering),
//   the SVT adjoint core B = Gs o sym(A) + Ga o skew(A) + diag(f' o diag A)
//     with Gs_ij = (f_i - f_j)/(s_i - s_j), Ga_ij = (f_i + f_j)/(s_i + s_j),
//     f(s) = max(s - theta, 0), and the threshold gradient -sum_{s_i>theta} A_ii,
//   row-wise prolongation X R^T of a coarse matrix.
// The contractions between them use the library's fp32 GEMM kernels.
#include <cfloat>

#include "common.cuh"

namespace cpcp {

namespace {

constexpr int EW_NT = 256;
constexpr float TAU = 0.5f;

__device__ __forceinline__ uint64_t gtimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// elementwise forward step
//   Lh = L_k + b (L_k - L_p), Sh = S_k + b (S_k - S_p), G = P_Q[Lh + Sh - D]
//   S_out = shrink(Sh - tau G, thS), XL = Lh - tau G
// ---------------------------------------------------------------------------
__global__ void unroll_step_kernel(int m, int n, const float *__restrict__ D, int64_t ldd,
                                   const uint32_t *__restrict__ Q, int64_t ldq, const float *__restrict__ Lk,
                                   const float *__restrict__ Lp, const float *__restrict__ Sk,
                                   const float *__restrict__ Sp, int64_t ld, float beta, float thS,
                                   float *__restrict__ Sout, float *__restrict__ XL)
{
    const int64_t total = (int64_t)m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int64_t o = (int64_t)i * ld + j;
        const bool obs = Q == nullptr || ((Q[(int64_t)i * ldq + (j >> 5)] >> (j & 31)) & 1u);
        const float lk = Lk[o], lp = Lp[o], sk = Sk[o], sp = Sp[o];
        const float lh = lk + beta * (lk - lp), sh = sk + beta * (sk - sp);
        const float g = obs ? lh + sh - D[(int64_t)i * ldd + j] : 0.f;
        Sout[o] = obs ? shrink(sh - TAU * g, thS) : 0.f;
        XL[o] = lh - TAU * g;
    }
}

// ---------------------------------------------------------------------------
// elementwise adjoint of one step.  Inputs: the step's states (L_k, L_p, S_k,
// S_p), gXL (adjoint of XL), gSn (adjoint of S_{k+1}); in/out: gLp, gSp
// (partial adjoints of L_k, S_k from the next step), dD.  Outputs: gLn, gSn
// overwritten with the adjoints of L_k and S_k (and gL32, an fp32 copy of
// gLn for the next step's contractions); gLp, gSp with the partial adjoints
// of L_{k-1}, S_{k-1}; per-block sums of -gS sign(XS) [|XS| > thS] (the
// threshold gradient of the shrink).  The adjoint recursion and dD are kept
// in fp64: summed over the steps in fp32 they lose about four digits on a
// 50-step sweep, while the contractions of the SVT adjoint may stay fp32.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(EW_NT)
    unroll_adjoint_kernel(int m, int n, const float *__restrict__ D, int64_t ldd, const uint32_t *__restrict__ Q,
                          int64_t ldq, const float *__restrict__ Lk, const float *__restrict__ Lp,
                          const float *__restrict__ Sk, const float *__restrict__ Sp, int64_t ld, double beta,
                          float thS, const float *__restrict__ gXL, double *__restrict__ gLn,
                          double *__restrict__ gSn, double *__restrict__ gLp, double *__restrict__ gSp,
                          double *__restrict__ dD, float *__restrict__ gL32, double *__restrict__ part)
{
    __shared__ double red[EW_NT / 32];
    double gth = 0.0;
    const int64_t total = (int64_t)m * n;
    const float bf = (float)beta;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int64_t o = (int64_t)i * ld + j;
        const bool obs = Q == nullptr || ((Q[(int64_t)i * ldq + (j >> 5)] >> (j & 31)) & 1u);
        // the forward's own fp32 arithmetic, to recover its active set
        const float lk = Lk[o], lp = Lp[o], sk = Sk[o], sp = Sp[o];
        const float lh = lk + bf * (lk - lp), sh = sk + bf * (sk - sp);
        const float g = obs ? lh + sh - D[(int64_t)i * ldd + j] : 0.f;
        const float xs = sh - TAU * g;
        const double gs = gSn[o];
        const bool act = fabsf(xs) > thS;
        const double gxs = act ? gs : 0.0;
        if (act) gth -= gs * (xs > 0.f ? 1.0 : -1.0);
        const double gxl = gXL[o];
        const double gpq = obs ? -0.5 * (gxl + gxs) : 0.0;
        const double glh = gxl + gpq, gsh = gxs + gpq;
        dD[o] -= gpq;
        const double gln = gLp[o] + (1.0 + beta) * glh;
        gLn[o] = gln;
        gL32[o] = (float)gln;
        gLp[o] = -beta * glh;
        gSn[o] = gSp[o] + (1.0 + beta) * gsh;
        gSp[o] = -beta * gsh;
    }
    gth = warp_sum(gth);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = gth;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < EW_NT / 32; w++) s += red[w];
        part[blockIdx.x] = s;
    }
}

// y (double, ld ly) = x (float, ld lx) or 0 when x is null; and the reverse
__global__ void widen_kernel(int m, int n, const float *__restrict__ x, int64_t lx, double *__restrict__ y, int64_t ly)
{
    const int64_t total = (int64_t)m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        y[(int64_t)i * ly + j] = x ? (double)x[(int64_t)i * lx + j] : 0.0;
    }
}

__global__ void narrow_kernel(int m, int n, const double *__restrict__ x, int64_t lx, float *__restrict__ y, int64_t ly)
{
    const int64_t total = (int64_t)m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        y[(int64_t)i * ly + j] = (float)x[(int64_t)i * lx + j];
    }
}

// out[i][j] = w0[j] Y[i][j0[j]] + w1[j] Y[i][j0[j] + 1]  (X R^T, row-wise prolongation)
__global__ void row_prolong_kernel(int m, int n, int nh, const float *__restrict__ Y, int64_t ldy,
                                   TransferDev<float> tr, float *__restrict__ out, int64_t ldo)
{
    const int64_t total = (int64_t)m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int a = tr.j0[j];
        float v = tr.w0[j] * Y[(int64_t)i * ldy + a];
        if (a + 1 < nh) v = fmaf(tr.w1[j], Y[(int64_t)i * ldy + a + 1], v);
        out[(int64_t)i * ldo + j] = v;
    }
}

// ---------------------------------------------------------------------------
// exact thin SVD by one-sided Jacobi over all column pairs
// ---------------------------------------------------------------------------

// X (q columns of length m, column c at X + c * m) = M^T; V = I (q x q, column-major)
__global__ void jfull_init_kernel(int m, int q, const float *__restrict__ M, int64_t ldm, float *__restrict__ X,
                                  float *__restrict__ V)
{
    const int64_t total = (int64_t)m * q;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / m), i = (int)(e % m);
        X[e] = M[(int64_t)i * ldm + c];
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)q * q;
         e += (int64_t)gridDim.x * blockDim.x)
        V[e] = (e / q == e % q) ? 1.f : 0.f;
}

struct GridSync {
    unsigned int count;
    unsigned int gen;
    unsigned long long maxrel[2];  // largest rotated |g|/sqrt(ab) of the sweep (double bits), by sweep parity
    int abort;
    int sweeps;
};

// Bounded grid barrier of a cooperative launch: false (and the abort flag set)
// if the other CTAs did not arrive within about one second.
__device__ bool grid_barrier(GridSync *gs, int *err)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *genp = &gs->gen;
        const unsigned int my = *genp;
        __threadfence();
        const unsigned int arrived = atomicAdd(&gs->count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&gs->count, 0u);
            __threadfence();
            atomicAdd(&gs->gen, 1u);
        } else {
            const uint64_t t0 = gtimer_ns();
            while (*genp == my) {
                if (*(volatile int *)&gs->abort) break;
                if (gtimer_ns() - t0 > 1000000000ull) {
                    atomicExch(&gs->abort, 1);
                    atomicExch(err, 1);
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile int *)&gs->abort) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

constexpr int JF_NT = 256;

// Sweeps of the round-robin ordering; CTA b handles pairs b, b + grid, ... of
// each round.  Dot products in fp64, rotations applied in fp32.  A pair of
// nonzero columns is rotated when |g| > tol sqrt(a b); the sweep loop ends
// when no pair needed a rotation.
__global__ void __launch_bounds__(JF_NT)
    jfull_sweeps_kernel(int m, int q, float *__restrict__ X, float *__restrict__ V, GridSync *gs, int *err,
                        int max_sweeps, float tol)
{
    __shared__ double red[3][JF_NT / 32];
    __shared__ double s_abg[3];
    const int N = q + (q & 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int sweep = 0;
    for (; sweep < max_sweeps; sweep++) {
        for (int round = 0; round < N - 1; round++) {
            for (int pr = blockIdx.x; pr < N / 2; pr += gridDim.x) {
                const int p = pr == 0 ? 0 : 1 + (pr - 1 + round) % (N - 1);
                const int r = 1 + (N - 2 - pr + round) % (N - 1);
                if (p >= q || r >= q) continue;
                float *xp = X + (int64_t)p * m, *xr = X + (int64_t)r * m;
                double a = 0.0, b = 0.0, g = 0.0;
                for (int i = tid; i < m; i += JF_NT) {
                    const double u = xp[i], v = xr[i];
                    a += u * u;
                    b += v * v;
                    g += u * v;
                }
                a = warp_sum(a);
                b = warp_sum(b);
                g = warp_sum(g);
                if (lane == 0) {
                    red[0][warp] = a;
                    red[1][warp] = b;
                    red[2][warp] = g;
                }
                __syncthreads();
                if (tid == 0) {
                    double ta = 0.0, tb = 0.0, tg = 0.0;
                    for (int w = 0; w < JF_NT / 32; w++) {
                        ta += red[0][w];
                        tb += red[1][w];
                        tg += red[2][w];
                    }
                    s_abg[0] = ta;
                    s_abg[1] = tb;
                    s_abg[2] = tg;
                }
                __syncthreads();
                a = s_abg[0];
                b = s_abg[1];
                g = s_abg[2];
                __syncthreads();
                // every pair of nonzero columns is made orthogonal, the small ones
                // too: the SVT adjoint uses the whole basis U, not only the
                // singular vectors above the threshold
                if (!(a > 0.0) || !(b > 0.0)) continue;
                const double rel = fabs(g) / (sqrt(a) * sqrt(b));
                if (!(rel > (double)tol)) continue;
                const double zeta = (b - a) / (2.0 * g);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                const float c32 = (float)cs, s32 = (float)sn;
                for (int i = tid; i < m; i += JF_NT) {
                    const float u = xp[i], v = xr[i];
                    xp[i] = c32 * u - s32 * v;
                    xr[i] = s32 * u + c32 * v;
                }
                float *vp = V + (int64_t)p * q, *vr = V + (int64_t)r * q;
                for (int i = tid; i < q; i += JF_NT) {
                    const float u = vp[i], v = vr[i];
                    vp[i] = c32 * u - s32 * v;
                    vr[i] = s32 * u + c32 * v;
                }
                if (tid == 0) atomicMax(&gs->maxrel[sweep & 1], (unsigned long long)__double_as_longlong(rel));
            }
            if (!grid_barrier(gs, err)) return;
            // the slot of the next sweep was last read before this round began
            if (round == 0 && blockIdx.x == 0 && tid == 0) gs->maxrel[(sweep + 1) & 1] = 0ull;
        }
        const double mr = __longlong_as_double((long long)*(volatile unsigned long long *)&gs->maxrel[sweep & 1]);
        if (!(mr > 0.0)) break;  // no rotation in this sweep: orthogonal to tol
        if (!grid_barrier(gs, err)) return;
    }
    if (blockIdx.x == 0 && tid == 0) gs->sweeps = sweep;
}

// s_c = ||x_c||, sorted descending; U (m x q row-major) = x_c / s_c, V row-major
__global__ void jfull_finish_kernel(int m, int q, const float *__restrict__ X, const float *__restrict__ Vc,
                                    float *__restrict__ U, int64_t ldu, float *__restrict__ Vout, int64_t ldv,
                                    double *__restrict__ sig, int *__restrict__ pos, double *__restrict__ nrm)
{
    // one CTA: norms, ranks; then the copies (grid-stride over the CTA only)
    const int tid = threadIdx.x;
    for (int c = tid; c < q; c += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < m; i++) s += (double)X[(int64_t)c * m + i] * X[(int64_t)c * m + i];
        nrm[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = tid; c < q; c += blockDim.x) {
        int p = 0;
        for (int c2 = 0; c2 < q; c2++) p += (nrm[c2] > nrm[c]) || (nrm[c2] == nrm[c] && c2 < c);
        pos[c] = p;
        sig[p] = nrm[c];
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)m * q; e += blockDim.x) {
        const int c = (int)(e / m), i = (int)(e % m);
        const double s = nrm[c];
        U[(int64_t)i * ldu + pos[c]] = s > 0.0 ? (float)((double)X[e] / s) : 0.f;
    }
    for (int64_t e = tid; e < (int64_t)q * q; e += blockDim.x) {
        const int c = (int)(e / q), i = (int)(e % q);
        Vout[(int64_t)i * ldv + pos[c]] = Vc[e];
    }
}

// ---------------------------------------------------------------------------
// SVT pieces on the singular triplets
// ---------------------------------------------------------------------------

// Bf = diag(f(sig)) V^T (q x q): the right factor of Y = U Bf.  Singular values
// and the threshold are fp64: f = sig - theta cancels when sig is just above
// theta, and the fp32 roundings of both would dominate its error.
__global__ void svt_right_kernel(int q, const double *__restrict__ sig, const float *__restrict__ V, int64_t ldv,
                                 double theta, float *__restrict__ Bf, int64_t ldb)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < q * q; e += gridDim.x * blockDim.x) {
        const int c = e / q, j = e % q;  // Bf[c][j] = f_c V[j][c]
        Bf[(int64_t)c * ldb + j] = (float)(fmax(sig[c] - theta, 0.0) * (double)V[(int64_t)j * ldv + c]);
    }
}

// B = Gs o sym(A) + Ga o skew(A) + diag(f' o diag A); gth = -sum_{s_i > theta} A_ii
__global__ void svt_adjoint_core_kernel(int q, const float *__restrict__ A, int64_t lda, const double *__restrict__ sig,
                                        double theta, float *__restrict__ B, int64_t ldb, double *__restrict__ gth)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < q * q; e += gridDim.x * blockDim.x) {
        const int i = e / q, j = e % q;
        const double si = sig[i], sj = sig[j];
        const double fi = fmax(si - theta, 0.0), fj = fmax(sj - theta, 0.0);
        const double aij = A[(int64_t)i * lda + j];
        double b;
        if (i == j) {
            b = si > theta ? aij : 0.0;
            if (si > theta) acc -= aij;
        } else {
            const double aji = A[(int64_t)j * lda + i];
            const double sym = 0.5 * (aij + aji), skew = 0.5 * (aij - aji);
            // both above theta: f is the shift s - theta on both, Gs = 1 exactly
            // (the quotient would cancel for close pairs and tie the result to
            // the individual vectors of a cluster); both below: 0
            const bool ai = si > theta, aj = sj > theta;
            const double d = si - sj;
            const double gs = (ai && aj) ? 1.0 : ((!ai && !aj) ? 0.0 : (d != 0.0 ? (fi - fj) / d : 0.5));
            const double ssum = si + sj;
            const double ga = ssum > 0.0 ? (fi + fj) / ssum : 0.0;
            b = gs * sym + ga * skew;
        }
        B[(int64_t)i * ldb + j] = (float)b;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        gth[blockIdx.x] = s;
    }
}

// Z = T + (P - W) diag(f / s)
__global__ void svt_adjoint_combine_kernel(int m, int q, const float *__restrict__ T, const float *__restrict__ P,
                                           const float *__restrict__ W, int64_t ld, const double *__restrict__ sig,
                                           double theta, float *__restrict__ Z)
{
    const int64_t total = (int64_t)m * q;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / q), c = (int)(e % q);
        const double s = sig[c], f = fmax(s - theta, 0.0);
        const float fs = s > 0.0 ? (float)(f / s) : 0.f;
        const int64_t o = (int64_t)i * ld + c;
        Z[o] = T[o] + (P[o] - W[o]) * fs;
    }
}

// dmu += (tau gthL + tau lam gthS) dmu_k, dlam += tau mu_k gthS (block partials summed in order)
__global__ void unroll_scalars_kernel(const double *__restrict__ gthL_part, int nL, const double *__restrict__ gthS_part,
                                      int nS, double lam, double mu_k, double dmu_k, double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double gL = 0.0, gS = 0.0;
    for (int i = 0; i < nL; i++) gL += gthL_part[i];
    for (int i = 0; i < nS; i++) gS += gthS_part[i];
    out[1] += (0.5 * gL + 0.5 * lam * gS) * dmu_k;  // d/dmu
    out[0] += 0.5 * mu_k * gS;                       // d/dlambda
}

int ew_grid(int64_t total)
{
    int64_t g = (total + EW_NT - 1) / EW_NT;
    return (int)std::min<int64_t>(g, 152 * 8);
}

}  // namespace

void launch_unroll_step(int m, int n, const float *D, int64_t ldd, const uint32_t *Q, int64_t ldq, const float *Lk,
                        const float *Lp, const float *Sk, const float *Sp, int64_t ld, float beta, float thS,
                        float *Sout, float *XL, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    unroll_step_kernel<<<ew_grid((int64_t)m * n), EW_NT, 0, st>>>(m, n, D, ldd, Q, ldq, Lk, Lp, Sk, Sp, ld, beta, thS,
                                                                 Sout, XL);
}

int launch_unroll_adjoint(int m, int n, const float *D, int64_t ldd, const uint32_t *Q, int64_t ldq, const float *Lk,
                          const float *Lp, const float *Sk, const float *Sp, int64_t ld, double beta, float thS,
                          const float *gXL, double *gLn, double *gSn, double *gLp, double *gSp, double *dD,
                          float *gL32, double *part, cudaStream_t st)
{
    const int g = ew_grid((int64_t)m * n);
    CPCP_COUNT_LAUNCH();
    unroll_adjoint_kernel<<<g, EW_NT, 0, st>>>(m, n, D, ldd, Q, ldq, Lk, Lp, Sk, Sp, ld, beta, thS, gXL, gLn, gSn, gLp,
                                               gSp, dD, gL32, part);
    return g;
}

void launch_widen(int m, int n, const float *x, int64_t lx, double *y, int64_t ly, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    widen_kernel<<<ew_grid((int64_t)m * n), EW_NT, 0, st>>>(m, n, x, lx, y, ly);
}

void launch_narrow(int m, int n, const double *x, int64_t lx, float *y, int64_t ly, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    narrow_kernel<<<ew_grid((int64_t)m * n), EW_NT, 0, st>>>(m, n, x, lx, y, ly);
}

void launch_row_prolong(int m, int n, int nh, const float *Y, int64_t ldy, const TransferDev<float> &tr, float *out,
                        int64_t ldo, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    row_prolong_kernel<<<ew_grid((int64_t)m * n), EW_NT, 0, st>>>(m, n, nh, Y, ldy, tr, out, ldo);
}

// Exact thin SVD of M (m x q, m >= q): U (m x q), V (q x q) row-major, sig
// descending.  work: X (q m floats), Vc (q q), nrm (q), pos (q ints),
// gs (a GridSync).  Returns the sweeps done, -1 on a launch error, -2 when a
// grid barrier timed out.
int launch_full_svd(int m, int q, const float *M, int64_t ldm, float *U, int64_t ldu, float *V, int64_t ldv,
                    double *sig, float *X, float *Vc, double *nrm, int *pos, void *gs_v, int *err, cudaStream_t st)
{
    GridSync *gs = static_cast<GridSync *>(gs_v);
    if (cudaMemsetAsync(gs, 0, sizeof(GridSync), st) != cudaSuccess) return -1;
    CPCP_COUNT_LAUNCH();
    jfull_init_kernel<<<ew_grid((int64_t)m * q), EW_NT, 0, st>>>(m, q, M, ldm, X, Vc);
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jfull_sweeps_kernel, JF_NT, 0);
    const int pairs = (q + (q & 1)) / 2;
    int grid = std::min(pairs, std::max(1, sms * std::max(1, occ)));
    grid = std::max(grid, 1);
    int max_sweeps = 40;
    // fp64 dot products; fp32 storage leaves |g|/sqrt(ab) near eps after a rotation
    float tol = 1e-7f;
    void *args[] = {&m, &q, &X, &Vc, &gs, &err, &max_sweeps, &tol};
    CPCP_COUNT_LAUNCH();
    if (cudaLaunchCooperativeKernel((const void *)jfull_sweeps_kernel, dim3(grid), dim3(JF_NT), args, 0, st) !=
        cudaSuccess)
        return -1;
    CPCP_COUNT_LAUNCH();
    jfull_finish_kernel<<<1, 1024, 0, st>>>(m, q, X, Vc, U, ldu, V, ldv, sig, pos, nrm);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_svt_right(int q, const double *sig, const float *V, int64_t ldv, double theta, float *Bf, int64_t ldb,
                      cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    svt_right_kernel<<<std::max(1, std::min(152, (q * q + 255) / 256)), 256, 0, st>>>(q, sig, V, ldv, theta, Bf, ldb);
}

int launch_svt_adjoint_core(int q, const float *A, int64_t lda, const double *sig, double theta, float *B, int64_t ldb,
                            double *gth_part, cudaStream_t st)
{
    const int g = std::max(1, std::min(152, (q * q + 255) / 256));
    CPCP_COUNT_LAUNCH();
    svt_adjoint_core_kernel<<<g, 256, 0, st>>>(q, A, lda, sig, theta, B, ldb, gth_part);
    return g;
}

void launch_svt_adjoint_combine(int m, int q, const float *T, const float *P, const float *W, int64_t ld,
                                const double *sig, double theta, float *Z, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    svt_adjoint_combine_kernel<<<ew_grid((int64_t)m * q), EW_NT, 0, st>>>(m, q, T, P, W, ld, sig, theta, Z);
}

void launch_unroll_scalars(const double *gthL_part, int nL, const double *gthS_part, int nS, double lam, double mu_k,
                           double dmu_k, double *out, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    unroll_scalars_kernel<<<1, 32, 0, st>>>(gthL_part, nL, gthS_part, nS, lam, mu_k, dmu_k, out);
}

size_t full_svd_sync_bytes() { return sizeof(GridSync); }

}  // namespace cpcp
