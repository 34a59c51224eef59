// k_ialm.cu -- the elementwise passes of the inexact augmented Lagrangian
// method for PCP, eq. (rpca): Alg. 1 (IALM) and its multilevel form Alg. 4
// (ML-IALM), whose low-rank step reuses the restriction, subspace SVD, SVT
// and prolongation of the CPCP path (solver.cu, ialm_core).
//
//   ialm_m       M = D - S + Y / mu_k                       (Alg. 1, the SVT argument)
//   ialm_update  S = shrink(D - L + Y / mu_k, lambda / mu_k) (Alg. 1, the S step)
//                E = D - L - S,  Y += mu_k E                 (the multiplier step)
//                per-block fp64 partial sums of ||E||_F^2    (the feasibility gap)
//   ialm_ctrl    the SVT threshold 1 / mu_k into the control block, and the
//                width bookkeeping after an iteration
//   bidiag_*     ML-IALM with an orthonormal basis of the range of R (option):
//                R C^{-1} with R^T R = C^T C; R^T R is tridiagonal (each row of
//                the composite R has two adjacent nonzeros at most), so C is
//                upper bidiagonal and M_H C^{-1}, C^{-1} V are two recurrences
#include "common.cuh"

namespace cpcp {

namespace {

constexpr int IALM_NT = 256;

template <typename T>
__global__ void __launch_bounds__(IALM_NT) ialm_m_kernel(int m, int n, const T *__restrict__ D, int64_t ldd,
                                                         const T *__restrict__ S, const T *__restrict__ Y,
                                                         int64_t lds, T inv_mu, T *__restrict__ M, int64_t ldm)
{
    const int64_t total = (int64_t)m * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - (idx / n) * n;
        M[i * ldm + j] = (D[i * ldd + j] - S[i * lds + j]) + Y[i * lds + j] * inv_mu;
    }
}

template <typename T>
__global__ void __launch_bounds__(IALM_NT) ialm_update_kernel(int m, int n, const T *__restrict__ D, int64_t ldd,
                                                              const T *__restrict__ L, int64_t ldl, T *__restrict__ S,
                                                              T *__restrict__ Y, int64_t lds, T mu, T inv_mu,
                                                              T theta, double *__restrict__ partial)
{
    __shared__ double red[IALM_NT / 32];
    double e2 = 0.0;
    const int64_t total = (int64_t)m * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - (idx / n) * n;
        const T d = D[i * ldd + j], l = L[i * ldl + j], y = Y[i * lds + j];
        const T s = shrink((d - l) + y * inv_mu, theta);
        const T e = (d - l) - s;
        S[i * lds + j] = s;
        Y[i * lds + j] = y + mu * e;
        e2 += (double)e * (double)e;
    }
    e2 = warp_sum(e2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < IALM_NT / 32; w++) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// begin (end == 0): SVT threshold 1 / mu for the fused SVT; end: the factors
// of this iteration become the current ones and the width moves on
__global__ void ialm_ctrl_kernel(Ctrl *c, double mu, int end)
{
    if (!end) {
        c->mu_k = mu;
        c->theta_L = 1.0 / mu;
    } else {
        c->rp = c->rk;
        c->rk = c->r_new;
        c->k = c->k_next;
        c->iter += 1;
    }
}

// X C = Y in place, one thread per row: x_0 = y_0 / c_0,
// x_a = (y_a - x_{a-1} e_{a-1}) / c_a (the rows are independent; n_H is short)
template <typename T>
__global__ void bidiag_right_solve_kernel(int rows, int nh, T *X, int64_t ld, const T *__restrict__ cd,
                                          const T *__restrict__ ce)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        T *x = X + r * ld;
        T prev = x[0] / cd[0];
        x[0] = prev;
        for (int a = 1; a < nh; a++) {
            prev = (x[a] - prev * ce[a - 1]) / cd[a];
            x[a] = prev;
        }
    }
}

// Out = C^{-1} V, one thread per column: v'_{nh-1} = v_{nh-1} / c_{nh-1},
// v'_a = (v_a - e_a v'_{a+1}) / c_a
template <typename T>
__global__ void bidiag_left_solve_kernel(int nh, const T *__restrict__ V, int64_t ldv, const int *kdyn,
                                         const T *__restrict__ cd, const T *__restrict__ ce, T *__restrict__ Out,
                                         int64_t ldo)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= *kdyn) return;
    T next = V[(int64_t)(nh - 1) * ldv + c] / cd[nh - 1];
    Out[(int64_t)(nh - 1) * ldo + c] = next;
    for (int a = nh - 2; a >= 0; a--) {
        next = (V[(int64_t)a * ldv + c] - ce[a] * next) / cd[a];
        Out[(int64_t)a * ldo + c] = next;
    }
}

}  // namespace

constexpr int IALM_BLOCKS = 608;  // four per SM, a fixed count so the fp64 partial sums reduce in a fixed order

int ialm_blocks() { return IALM_BLOCKS; }

template <typename T>
void launch_ialm_m(int m, int n, const T *D, int64_t ldd, const T *S, const T *Y, int64_t lds, double mu, T *M,
                   int64_t ldm, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    ialm_m_kernel<T><<<IALM_BLOCKS, IALM_NT, 0, st>>>(m, n, D, ldd, S, Y, lds, T(1.0 / mu), M, ldm);
}

template <typename T>
void launch_ialm_update(int m, int n, const T *D, int64_t ldd, const T *L, int64_t ldl, T *S, T *Y, int64_t lds,
                        double lam, double mu, double *partial, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    ialm_update_kernel<T><<<IALM_BLOCKS, IALM_NT, 0, st>>>(m, n, D, ldd, L, ldl, S, Y, lds, T(mu), T(1.0 / mu),
                                                           T(lam / mu), partial);
}

void launch_ialm_ctrl(Ctrl *c, double mu, int end, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    ialm_ctrl_kernel<<<1, 1, 0, st>>>(c, mu, end);
}

template <typename T>
void launch_bidiag_right_solve(int rows, int nh, T *X, int64_t ld, const T *cd, const T *ce, cudaStream_t st)
{
    const int blocks = (int)std::min<int64_t>(((int64_t)rows + 127) / 128, 1216);
    CPCP_COUNT_LAUNCH();
    bidiag_right_solve_kernel<T><<<blocks, 128, 0, st>>>(rows, nh, X, ld, cd, ce);
}

template <typename T>
void launch_bidiag_left_solve(int nh, const T *V, int64_t ldv, const int *kdyn, int kmax, const T *cd, const T *ce,
                              T *Out, int64_t ldo, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    bidiag_left_solve_kernel<T><<<(kmax + 63) / 64, 64, 0, st>>>(nh, V, ldv, kdyn, cd, ce, Out, ldo);
}

#define INST(T)                                                                                                    \
    template void launch_ialm_m<T>(int, int, const T *, int64_t, const T *, const T *, int64_t, double, T *,        \
                                   int64_t, cudaStream_t);                                                         \
    template void launch_ialm_update<T>(int, int, const T *, int64_t, const T *, int64_t, T *, T *, int64_t, double, \
                                        double, double *, cudaStream_t);                                            \
    template void launch_bidiag_right_solve<T>(int, int, T *, int64_t, const T *, const T *, cudaStream_t);         \
    template void launch_bidiag_left_solve<T>(int, const T *, int64_t, const int *, int, const T *, const T *, T *,  \
                                              int64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cpcp
