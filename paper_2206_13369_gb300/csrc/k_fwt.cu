// k_fwt.cu -- the m x n passes of Frank-Wolfe Thresholding (Alg. 3) and
// ML-FWT (Alg. 6) for eq. (cpcp) in the epigraph form of eq. (cpcp-fw).
// The LMO of the nuclear ball (the top singular pair of the gradient, or of
// its restriction) comes from the subspace SVD of the CPCP path; what is
// here streams L, S, D and the mask:
//
//   fwt_grad     G = P_Q[L + S - D] at the start, with per-block argmax |G|
//   fwt_coef     the two-segment line search's coefficients, as fp64
//                per-block partial sums:  A = ||P_Q[V_L - L]||^2,
//                B = ||P_Q[V_S - S]||^2, C = <P_Q[V_L - L], P_Q[V_S - S]>,
//                <G, P_Q[V_L - L]>, <G, P_Q[V_S - S]>,  with V_L = cL u v^T
//                (rank one; cL = -U_L or 0) and V_S = vs e_{i*} (one entry)
//   fwt_update   L += a (V_L - L); S' = S + b (V_S - S); the thresholding
//                step S = shrink_{lambda_S}(S' - P_Q[L + S' - D]); the new
//                gradient G = P_Q[L + S - D] written for the next LMO, with
//                per-block ||S||_1, ||G||_F^2 and argmax |G|
//
// Argmax ties go to the smallest row-major index, so the LMO of the l1 ball
// is the first entry of largest magnitude.
#include "common.cuh"

namespace cpcp {

namespace {

constexpr int FWT_NT = 256;
constexpr int FWT_BLOCKS = 608;  // fixed, so the fp64 partial sums reduce in a fixed order

__device__ __forceinline__ bool observed(const uint32_t *Q, int64_t ldq, int64_t i, int64_t j)
{
    return Q == nullptr || ((Q[i * ldq + (j >> 5)] >> (j & 31)) & 1u);
}

// block argmax of (value, index): larger value wins, ties to the smaller index
__device__ __forceinline__ void amax_merge(double &v, int64_t &ix, double v2, int64_t ix2)
{
    if (v2 > v || (v2 == v && ix2 < ix)) {
        v = v2;
        ix = ix2;
    }
}

template <int NS>
__device__ __forceinline__ void block_sums(double (&s)[NS], double amv, int64_t amix, double *partial, double *amax_v,
                                           int64_t *amax_i)
{
    __shared__ double red[FWT_NT / 32][NS + 1];
    __shared__ int64_t redi[FWT_NT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NS; q++) s[q] = warp_sum(s[q]);
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, amv, o);
        const int64_t i2 = __shfl_xor_sync(0xffffffffu, amix, o);
        amax_merge(amv, amix, v2, i2);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NS; q++) red[w][q] = s[q];
        red[w][NS] = amv;
        redi[w] = amix;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[NS];
#pragma unroll
        for (int q = 0; q < NS; q++) t[q] = 0.0;
        double bv = -1.0;
        int64_t bi = INT64_MAX;
        for (int ww = 0; ww < FWT_NT / 32; ww++) {
#pragma unroll
            for (int q = 0; q < NS; q++) t[q] += red[ww][q];
            amax_merge(bv, bi, red[ww][NS], redi[ww]);
        }
#pragma unroll
        for (int q = 0; q < NS; q++) partial[(int64_t)blockIdx.x * NS + q] = t[q];
        if (amax_v) {
            amax_v[blockIdx.x] = bv;
            amax_i[blockIdx.x] = bi;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(FWT_NT) fwt_grad_kernel(int m, int n, const T *__restrict__ D, int64_t ldd,
                                                          const uint32_t *__restrict__ Q, int64_t ldq,
                                                          const T *__restrict__ L, const T *__restrict__ S,
                                                          int64_t ld, T *__restrict__ G, double *partial,
                                                          double *amax_v, int64_t *amax_i)
{
    double s[1] = {0.0}, amv = -1.0;
    int64_t amix = INT64_MAX;
    const int64_t total = (int64_t)m * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - i * n;
        const T g = observed(Q, ldq, i, j) ? (L[i * ld + j] + S[i * ld + j]) - D[i * ldd + j] : T(0);
        G[i * ld + j] = g;
        s[0] += (double)g * (double)g;
        amax_merge(amv, amix, fabs((double)g), idx);
    }
    block_sums<1>(s, amv, amix, partial, amax_v, amax_i);
}

template <typename T>
__global__ void __launch_bounds__(FWT_NT) fwt_coef_kernel(int m, int n, const uint32_t *__restrict__ Q, int64_t ldq,
                                                          const T *__restrict__ L, const T *__restrict__ S,
                                                          const T *__restrict__ G, int64_t ld,
                                                          const T *__restrict__ u, int64_t ldu,
                                                          const T *__restrict__ v, int64_t ldv, T cL, int64_t istar,
                                                          T vs, double *partial)
{
    double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t total = (int64_t)m * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - i * n;
        if (!observed(Q, ldq, i, j)) continue;
        const double pa = (double)(cL * u[i * ldu] * v[j * ldv]) - (double)L[i * ld + j];
        const double pb = (idx == istar ? (double)vs : 0.0) - (double)S[i * ld + j];
        const double g = (double)G[i * ld + j];
        s[0] += pa * pa;
        s[1] += pb * pb;
        s[2] += pa * pb;
        s[3] += g * pa;
        s[4] += g * pb;
    }
    block_sums<5>(s, -1.0, INT64_MAX, partial, nullptr, nullptr);
}

template <typename T>
__global__ void __launch_bounds__(FWT_NT) fwt_update_kernel(int m, int n, const T *__restrict__ D, int64_t ldd,
                                                            const uint32_t *__restrict__ Q, int64_t ldq,
                                                            T *__restrict__ L, T *__restrict__ S, T *__restrict__ G,
                                                            int64_t ld, const T *__restrict__ u, int64_t ldu,
                                                            const T *__restrict__ v, int64_t ldv, T cL,
                                                            int64_t istar, T vs, T a, T b, T lamS, double *partial,
                                                            double *amax_v, int64_t *amax_i)
{
    double s[2] = {0.0, 0.0}, amv = -1.0;
    int64_t amix = INT64_MAX;
    const int64_t total = (int64_t)m * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx - i * n;
        const bool obs = observed(Q, ldq, i, j);
        const T d = D[i * ldd + j];
        const T l0 = L[i * ld + j], s0 = S[i * ld + j];
        const T l = l0 + a * (cL * u[i * ldu] * v[j * ldv] - l0);
        const T sh = s0 + b * ((idx == istar ? vs : T(0)) - s0);
        const T r = obs ? (l + sh) - d : T(0);
        const T sn = shrink(sh - r, lamS);
        const T g = obs ? (l + sn) - d : T(0);
        L[i * ld + j] = l;
        S[i * ld + j] = sn;
        G[i * ld + j] = g;
        s[0] += fabs((double)sn);
        s[1] += (double)g * (double)g;
        amax_merge(amv, amix, fabs((double)g), idx);
    }
    block_sums<2>(s, amv, amix, partial, amax_v, amax_i);
}

}  // namespace

int fwt_blocks() { return FWT_BLOCKS; }

template <typename T>
void launch_fwt_grad(int m, int n, const T *D, int64_t ldd, const uint32_t *Q, int64_t ldq, const T *L, const T *S,
                     int64_t ld, T *G, double *partial, double *amax_v, int64_t *amax_i, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_grad_kernel<T><<<FWT_BLOCKS, FWT_NT, 0, st>>>(m, n, D, ldd, Q, ldq, L, S, ld, G, partial, amax_v, amax_i);
}

template <typename T>
void launch_fwt_coef(int m, int n, const uint32_t *Q, int64_t ldq, const T *L, const T *S, const T *G, int64_t ld,
                     const T *u, int64_t ldu, const T *v, int64_t ldv, double cL, int64_t istar, double vs,
                     double *partial, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_coef_kernel<T><<<FWT_BLOCKS, FWT_NT, 0, st>>>(m, n, Q, ldq, L, S, G, ld, u, ldu, v, ldv, T(cL), istar, T(vs),
                                                      partial);
}

template <typename T>
void launch_fwt_update(int m, int n, const T *D, int64_t ldd, const uint32_t *Q, int64_t ldq, T *L, T *S, T *G,
                       int64_t ld, const T *u, int64_t ldu, const T *v, int64_t ldv, double cL, int64_t istar,
                       double vs, double a, double b, double lamS, double *partial, double *amax_v, int64_t *amax_i,
                       cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_update_kernel<T><<<FWT_BLOCKS, FWT_NT, 0, st>>>(m, n, D, ldd, Q, ldq, L, S, G, ld, u, ldu, v, ldv, T(cL),
                                                        istar, T(vs), T(a), T(b), T(lamS), partial, amax_v, amax_i);
}

#define INST(T)                                                                                                      \
    template void launch_fwt_grad<T>(int, int, const T *, int64_t, const uint32_t *, int64_t, const T *, const T *,  \
                                     int64_t, T *, double *, double *, int64_t *, cudaStream_t);                     \
    template void launch_fwt_coef<T>(int, int, const uint32_t *, int64_t, const T *, const T *, const T *, int64_t,  \
                                     const T *, int64_t, const T *, int64_t, double, int64_t, double, double *,      \
                                     cudaStream_t);                                                                  \
    template void launch_fwt_update<T>(int, int, const T *, int64_t, const uint32_t *, int64_t, T *, T *, T *,       \
                                       int64_t, const T *, int64_t, const T *, int64_t, double, int64_t, double,     \
                                       double, double, double, double *, double *, int64_t *, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cpcp
