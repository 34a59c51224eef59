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
                                                          const T *__restrict__ v, int64_t ldv,
                                                          const FwScal *__restrict__ sc, double *partial)
{
    if (sc->done) return;
    const T cL = T(sc->cL), vs = T(sc->vs);
    const int64_t istar = sc->istar;
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
                                                            const T *__restrict__ v, int64_t ldv,
                                                            const FwScal *__restrict__ sc, double *partial,
                                                            double *amax_v, int64_t *amax_i)
{
    if (sc->done) return;
    const T cL = T(sc->cL), vs = T(sc->vs), a = T(sc->a), b = T(sc->b), lamS = T(sc->lamS);
    const int64_t istar = sc->istar;
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

// sum over the FWT_BLOCKS blocks of slot q (of ns per block) by one warp, in a
// fixed order (lane-strided partial sums, then a fixed shuffle tree)
__device__ __forceinline__ double warp_block_sum(const double *partial, int ns, int q)
{
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    for (int b = lane; b < FWT_BLOCKS; b += 32) t += partial[(int64_t)b * ns + q];
    return warp_sum(t);
}

// argmax over the blocks' (value, index) by one warp, ties to the smaller index
__device__ __forceinline__ void warp_block_amax(const double *amax_v, const int64_t *amax_i, double &v, int64_t &ix)
{
    const int lane = threadIdx.x & 31;
    v = -1.0;
    ix = INT64_MAX;
    for (int b = lane; b < FWT_BLOCKS; b += 32) amax_merge(v, ix, amax_v[b], amax_i[b]);
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t i2 = __shfl_xor_sync(0xffffffffu, ix, o);
        amax_merge(v, ix, v2, i2);
    }
}

// Exact minimiser over [0,1]^2 of 1/2 (A a^2 + 2 C a b + B b^2) + ga a + gb b
// (convex: A, B >= 0, A B >= C^2): the stationary point if it lies in the box,
// else the best of the four edge minimisers.  The two-segment line search of
// Alg. 3.
__device__ void fw_box_qp(double A, double B, double C, double ga, double gb, double *a_out, double *b_out)
{
    double best_a = 0.0, best_b = 0.0, best = 0.0;  // q(0, 0) = 0
    auto q = [&](double a, double b) { return 0.5 * (A * a * a + 2.0 * C * a * b + B * b * b) + ga * a + gb * b; };
    auto c01 = [](double x) { return fmin(1.0, fmax(0.0, x)); };
    auto consider = [&](double a, double b) {
        const double v = q(a, b);
        if (v < best) {
            best = v;
            best_a = a;
            best_b = b;
        }
    };
    const double det = A * B - C * C;
    if (det > 0.0) {
        const double a = (C * gb - B * ga) / det, b = (C * ga - A * gb) / det;
        if (a >= 0.0 && a <= 1.0 && b >= 0.0 && b <= 1.0) consider(a, b);
    }
    for (int ei = 0; ei < 2; ei++) {
        const double e = (double)ei;
        const double lb = gb + C * e, la = ga + C * e;
        consider(e, B > 0.0 ? c01(-lb / B) : (lb < 0.0 ? 1.0 : 0.0));
        consider(A > 0.0 ? c01(-la / A) : (la < 0.0 ? 1.0 : 0.0), e);
    }
    *a_out = best_a;
    *b_out = best_b;
}

__global__ void fwt_first_kernel(FwScal *sc, const double *__restrict__ partial, const double *__restrict__ amax_v,
                                 const int64_t *__restrict__ amax_i)
{
    // one warp
    const double g2 = warp_block_sum(partial, 1, 0);
    double v;
    int64_t ix;
    warp_block_amax(amax_v, amax_i, v, ix);
    if (threadIdx.x == 0) {
        sc->f = 0.5 * g2;
        sc->gmax = v;
        sc->istar = ix;
        sc->UL = sc->f / sc->lamL;
        sc->US = sc->f / sc->lamS;
        sc->tL = 0.0;
        sc->tS = 0.0;
        sc->rel = INFINITY;
        sc->done = 0;
        sc->iters = 0;
    }
}

template <typename T>
__global__ void fwt_lmo_kernel(FwScal *sc, const T *__restrict__ sig, const T *__restrict__ G, int64_t ld, int m,
                               int n)
{
    if (sc->done) return;
    const int64_t istar = sc->istar;
    // no finite entry of G (non-finite input): no argmax, nothing to step on
    if (istar < 0 || istar >= (int64_t)m * n || !isfinite(sc->f)) {
        sc->done = 2;
        return;
    }
    const double s0 = (double)sig[0];
    const double gval = (double)G[(istar / n) * ld + (istar % n)];
    // after a thresholding step every entry of the support of S has
    // |G_ij| = lambda_S exactly, the others |G_ij| <= lambda_S: the l1 test takes
    // a relative margin of a few hundred units of rounding of T
    const bool useL = sc->lamL < s0, useS = sc->lamS * (1.0 + sc->margin) < sc->gmax;
    sc->cL = useL ? -sc->UL : 0.0;
    sc->VtL = useL ? sc->UL : 0.0;
    sc->vs = useS ? -sc->US * (gval > 0.0 ? 1.0 : -1.0) : 0.0;
    sc->VtS = useS ? sc->US : 0.0;
}

__global__ void fwt_ls_kernel(FwScal *sc, const double *__restrict__ partial)
{
    // five warps, one per coefficient
    __shared__ double c[5];
    if (sc->done) return;
    const int w = threadIdx.x >> 5;
    const double t = warp_block_sum(partial, 5, w);
    if ((threadIdx.x & 31) == 0) c[w] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double ga = c[3] + sc->lamL * (sc->VtL - sc->tL), gb = c[4] + sc->lamS * (sc->VtS - sc->tS);
        double a, b;
        fw_box_qp(c[0], c[1], c[2], ga, gb, &a, &b);
        sc->a = a;
        sc->b = b;
    }
}

__global__ void fwt_post_kernel(FwScal *sc, const double *__restrict__ partial, const double *__restrict__ amax_v,
                                const int64_t *__restrict__ amax_i, double *trace)
{
    // three warps: ||S||_1, ||G||_F^2, argmax |G|
    __shared__ double c[2];
    __shared__ double sv;
    __shared__ int64_t si;
    if (sc->done) return;
    const int w = threadIdx.x >> 5;
    if (w < 2) {
        const double t = warp_block_sum(partial, 2, w);
        if ((threadIdx.x & 31) == 0) c[w] = t;
    } else {
        double v;
        int64_t ix;
        warp_block_amax(amax_v, amax_i, v, ix);
        if ((threadIdx.x & 31) == 0) {
            sv = v;
            si = ix;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double fprev = sc->f;
        sc->tL += sc->a * (sc->VtL - sc->tL);
        sc->tS = c[0];
        const double f = 0.5 * c[1] + sc->lamL * sc->tL + sc->lamS * sc->tS;
        sc->f = f;
        sc->gmax = sv;
        sc->istar = si;
        sc->UL = f / sc->lamL;
        sc->US = f / sc->lamS;
        if (trace != nullptr) trace[sc->iters] = f;
        sc->iters += 1;
        if (!isfinite(f)) {
            sc->done = 2;
        } else {
            sc->rel = fabs(fprev - f) / fprev;
            if (sc->rel <= sc->tol) sc->done = 1;
        }
    }
}

}  // namespace

void launch_fwt_first(FwScal *sc, const double *partial, const double *amax_v, const int64_t *amax_i,
                      cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_first_kernel<<<1, 32, 0, st>>>(sc, partial, amax_v, amax_i);
}

template <typename T>
void launch_fwt_lmo(FwScal *sc, const T *sig, const T *G, int64_t ld, int m, int n, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_lmo_kernel<T><<<1, 1, 0, st>>>(sc, sig, G, ld, m, n);
}

void launch_fwt_ls(FwScal *sc, const double *partial, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_ls_kernel<<<1, 160, 0, st>>>(sc, partial);
}

void launch_fwt_post(FwScal *sc, const double *partial, const double *amax_v, const int64_t *amax_i, double *trace,
                     cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_post_kernel<<<1, 96, 0, st>>>(sc, partial, amax_v, amax_i, trace);
}

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
                     const T *u, int64_t ldu, const T *v, int64_t ldv, const FwScal *sc, double *partial,
                     cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_coef_kernel<T><<<FWT_BLOCKS, FWT_NT, 0, st>>>(m, n, Q, ldq, L, S, G, ld, u, ldu, v, ldv, sc, partial);
}

template <typename T>
void launch_fwt_update(int m, int n, const T *D, int64_t ldd, const uint32_t *Q, int64_t ldq, T *L, T *S, T *G,
                       int64_t ld, const T *u, int64_t ldu, const T *v, int64_t ldv, const FwScal *sc,
                       double *partial, double *amax_v, int64_t *amax_i, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    fwt_update_kernel<T><<<FWT_BLOCKS, FWT_NT, 0, st>>>(m, n, D, ldd, Q, ldq, L, S, G, ld, u, ldu, v, ldv, sc, partial,
                                                        amax_v, amax_i);
}

#define INST(T)                                                                                                      \
    template void launch_fwt_grad<T>(int, int, const T *, int64_t, const uint32_t *, int64_t, const T *, const T *,  \
                                     int64_t, T *, double *, double *, int64_t *, cudaStream_t);                     \
    template void launch_fwt_coef<T>(int, int, const uint32_t *, int64_t, const T *, const T *, const T *, int64_t,  \
                                     const T *, int64_t, const T *, int64_t, const FwScal *, double *, cudaStream_t); \
    template void launch_fwt_update<T>(int, int, const T *, int64_t, const uint32_t *, int64_t, T *, T *, T *,       \
                                       int64_t, const T *, int64_t, const T *, int64_t, const FwScal *, double *,    \
                                       double *, int64_t *, cudaStream_t);                                           \
    template void launch_fwt_lmo<T>(FwScal *, const T *, const T *, int64_t, int, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cpcp
