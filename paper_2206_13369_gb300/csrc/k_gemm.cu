// k_gemm.cu -- tall-skinny contractions of the subspace-iteration SVD and the
// transfer operators.
//
//   gemm_nn          C = A B        (Y = M_H Omega, Q = X R^{-1}, U = Q Ut, ...)
//   gemm_tn_partial  C_s = A_s^T B_s over row splits s, then a fixed-order
//                    reduction (Z = M_H^T Q, Gram matrices X^T X), so the
//                    result is bit-reproducible run to run
//   restrict         M_H = M R  (Sec. 3.1, Alg. 4 restriction)
//   prolong          B = R V    (Sec. 3.2: L = L_H R^T = U (R V)^T)
//
// Operands are row-major.  Widths that change during a solve (the subspace
// width k, the rank r) are read from device memory so that launches do not
// depend on host-side values; grids are sized for the maximum width and
// blocks beyond the live width return immediately.
#include <algorithm>

#include "common.cuh"

namespace cpcp {

namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

// C = A B; with gridDim.z > 1 block z sums the K range [z ks, (z+1) ks) into
// the slice z of C (a partial buffer of gridDim.z slices of rows x ldc).
template <typename T>
__global__ void __launch_bounds__(NT)
    gemm_nn_kernel(int rows, int Kstat, const T *__restrict__ A, int64_t lda, const T *__restrict__ B, int64_t ldb,
                   T *__restrict__ C, int64_t ldc, const int *kdynK, const int *kdynN, int Nstat, int ks)
{
    __shared__ T As[TK][TM + 4];
    __shared__ T Bs[TK][TN + 4];
    const int Kall = kdynK ? *kdynK : Kstat;
    const int N = kdynN ? *kdynN : Nstat;
    const int rb = blockIdx.x * TM, cb = blockIdx.y * TN;
    if (cb >= N) return;
    const int kbeg = blockIdx.z * ks;
    const int K = min(Kall, kbeg + ks);
    C += (int64_t)blockIdx.z * rows * ldc;
    A += kbeg;
    B += (int64_t)kbeg * ldb;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = T(0);
    const int Kloc = K - kbeg;
    for (int k0 = 0; k0 < Kloc; k0 += TK) {
        {
            int row = t >> 2, kk = (t & 3) * 4, gr = rb + row;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                int kx = k0 + kk + u;
                As[kk + u][row] = (gr < rows && kx < Kloc) ? A[(int64_t)gr * lda + kx] : T(0);
            }
            int kr = t >> 4, c4 = (t & 15) * 4, gk = k0 + kr;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                int c = cb + c4 + u;
                Bs[kr][c4 + u] = (gk < Kloc && c < N) ? B[(int64_t)gk * ldb + c] : T(0);
            }
        }
        __syncthreads();
        // the TK terms of a chunk are summed apart and then added to the total
        // (rounding ~ (sqrt(TK) + sqrt(K / TK)) eps rather than sqrt(K) eps)
        T part[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) part[i][j] = T(0);
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][4 * tx + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) part[i][j] = fma(a[i], b[j], part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] += part[i][j];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int row = rb + ty + 16 * i;
        if (row >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int c = cb + 4 * tx + j;
            if (c < N) C[(int64_t)row * ldc + c] = acc[i][j];
        }
    }
}

// partial[s][p][c] = sum_{i in split s} A[i][p] B[i][c]
template <typename T>
__global__ void __launch_bounds__(NT)
    gemm_tn_partial_kernel(int rows, int Kstat, int rows_per_split, const T *__restrict__ A, int64_t lda,
                           const T *__restrict__ B, int64_t ldb, T *__restrict__ partial, const int *kdynK,
                           const int *kdynN, int Nstat, int Kmax, int Nmax, const int *skip)
{
    if (skip != nullptr && *skip) return;
    __shared__ T As[TK][TM + 4];
    __shared__ T Bs[TK][TN + 4];
    const int K = kdynK ? *kdynK : Kstat;
    const int N = kdynN ? *kdynN : Nstat;
    const int pb = blockIdx.x * TM, cb = blockIdx.y * TN, s = blockIdx.z;
    if (pb >= K || cb >= N) return;
    const int i0 = s * rows_per_split, i1 = min(rows, i0 + rows_per_split);
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = T(0);
    for (int r0 = i0; r0 < i1; r0 += TK) {
        {
            int rr = t >> 4, c4 = (t & 15) * 4, gi = r0 + rr;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                int p = pb + c4 + u, c = cb + c4 + u;
                As[rr][c4 + u] = (gi < i1 && p < K) ? A[(int64_t)gi * lda + p] : T(0);
                Bs[rr][c4 + u] = (gi < i1 && c < N) ? B[(int64_t)gi * ldb + c] : T(0);
            }
        }
        __syncthreads();
        T part[4][4];  // chunk sum, then added to the total (as in gemm_nn_kernel)
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) part[i][j] = T(0);
#pragma unroll
        for (int kk = 0; kk < TK; kk++) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][4 * tx + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) part[i][j] = fma(a[i], b[j], part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] += part[i][j];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int p = pb + ty + 16 * i;
        if (p >= K) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int c = cb + 4 * tx + j;
            if (c < N) partial[((int64_t)s * Kmax + p) * Nmax + c] = acc[i][j];
        }
    }
}

template <typename T>
__global__ void reduce_partial_kernel(const T *__restrict__ partial, int splits, int Kstat, int Nstat, int Kmax,
                                      int Nmax, T *__restrict__ C, int64_t ldc, const int *kdynK, const int *kdynN)
{
    const int K = kdynK ? *kdynK : Kstat;
    const int N = kdynN ? *kdynN : Nstat;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)K * N) return;
    int p = (int)(idx / N), c = (int)(idx % N);
    T s = T(0);
    for (int q = 0; q < splits; q++) s += partial[((int64_t)q * Kmax + p) * Nmax + c];
    C[(int64_t)p * ldc + c] = s;
}

template <typename T>
__global__ void restrict_kernel(int m, int n, const T *__restrict__ M, int64_t ldm, T *__restrict__ MH, int64_t ldh,
                                TransferDev<T> tr)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= tr.nh) return;
    for (int i = blockIdx.y; i < m; i += gridDim.y) {  // rows beyond the 65535 grid rows loop
        T s = T(0);
        for (int j = tr.clo[c]; j <= tr.chi[c]; j++) {
            T w = (tr.j0[j] == c) ? tr.w0[j] : ((tr.j0[j] + 1 == c) ? tr.w1[j] : T(0));
            s = fma(M[(int64_t)i * ldm + j], w, s);
        }
        MH[(int64_t)i * ldh + c] = s;
    }
}

// B[j][c] = w0[j] V[j0[j]][c] + w1[j] V[j0[j]+1][c] for c < r; zero for r <= c < kmax
template <typename T>
__global__ void prolong_kernel(int n, const T *__restrict__ V, int64_t ldv, T *__restrict__ B, int64_t ldb,
                               TransferDev<T> tr, const int *kdyn, int kmax)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= kmax) return;
    int r = kdyn ? *kdyn : kmax;
    for (int j = blockIdx.y; j < n; j += gridDim.y) {
        T v = T(0);
        if (c < r) {
            int a = tr.j0[j];
            v = tr.w0[j] * V[(int64_t)a * ldv + c];
            if (a + 1 < tr.nh && tr.w1[j] != T(0)) v = fma(tr.w1[j], V[(int64_t)(a + 1) * ldv + c], v);
        }
        B[(int64_t)j * ldb + c] = v;
    }
}

// Omega[c][:] = sum_j R[j][c] B[j][:] for the coarse rows c < nh, columns < r;
// random columns are filled later.  (Restriction of a right factor.)
template <typename T>
__global__ void restrict_rows_kernel(const T *__restrict__ B, int64_t ldb, T *__restrict__ Om, int64_t ldo,
                                     TransferDev<T> tr, const int *kdyn, int kmax)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= kmax) return;
    int r = kdyn ? *kdyn : kmax;
    if (c >= r) return;
    for (int row = blockIdx.y; row < tr.nh; row += gridDim.y) {
        T s = T(0);
        for (int j = tr.clo[row]; j <= tr.chi[row]; j++) {
            T w = (tr.j0[j] == row) ? tr.w0[j] : ((tr.j0[j] + 1 == row) ? tr.w1[j] : T(0));
            s = fma(w, B[(int64_t)j * ldb + c], s);
        }
        Om[(int64_t)row * ldo + c] = s;
    }
}

template <typename T>
__global__ void transpose_kernel(int rows, int cols, const T *__restrict__ A, int64_t lda, T *__restrict__ B,
                                 int64_t ldb)
{
    __shared__ T tile[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int r = by + y, c = bx + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = A[(int64_t)r * lda + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int r = bx + y, c = by + threadIdx.x;  // output row = input column
        if (r < cols && c < rows) B[(int64_t)r * ldb + c] = tile[threadIdx.x][y];
    }
}

// transposed bit mask: out (cols x rows) from in (rows x cols), one word per thread
__global__ void transpose_mask_kernel(int rows, int cols, const uint32_t *__restrict__ in, int64_t ldi,
                                      uint32_t *__restrict__ out, int64_t ldo)
{
    int w = blockIdx.x * blockDim.x + threadIdx.x;  // word index along the output row
    if ((int64_t)w >= ldo) return;
    for (int r = blockIdx.y; r < cols; r += gridDim.y) {  // output row = input column
        uint32_t word = 0;
        for (int b = 0; b < 32; b++) {
            int c = w * 32 + b;  // output column = input row
            if (c >= rows) break;
            uint32_t bit = (in[(int64_t)c * ldi + (r >> 5)] >> (r & 31)) & 1u;
            word |= bit << b;
        }
        out[(int64_t)r * ldo + w] = word;
    }
}

}  // namespace

template <typename T>
void launch_restrict_rows(const T *B, int64_t ldb, T *Om, int64_t ldo, const TransferDev<T> &tr, const int *kdyn,
                          int kmax, cudaStream_t st)
{
    dim3 grid((kmax + 63) / 64, std::min(tr.nh, 65535));
    CPCP_COUNT_LAUNCH();
    restrict_rows_kernel<T><<<grid, 64, 0, st>>>(B, ldb, Om, ldo, tr, kdyn, kmax);
}

template <typename T>
void launch_transpose(int rows, int cols, const T *A, int64_t lda, T *B, int64_t ldb, cudaStream_t st)
{
    dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    CPCP_COUNT_LAUNCH();
    transpose_kernel<T><<<grid, dim3(32, 8), 0, st>>>(rows, cols, A, lda, B, ldb);
}

void launch_transpose_mask(int rows, int cols, const uint32_t *in, int64_t ldi, uint32_t *out, int64_t ldo,
                           cudaStream_t st)
{
    dim3 grid((unsigned)((ldo + 63) / 64), (unsigned)std::min(cols, 65535));
    CPCP_COUNT_LAUNCH();
    transpose_mask_kernel<<<grid, 64, 0, st>>>(rows, cols, in, ldi, out, ldo);
}

template <typename T>
void launch_gemm_nn(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc,
                    const int *kdyn_K, const int *kdyn_N, int kmaxN, cudaStream_t st)
{
    if (rows <= 0 || kmaxN <= 0) return;
    dim3 grid((rows + TM - 1) / TM, (kmaxN + TN - 1) / TN);
    CPCP_COUNT_LAUNCH();
    gemm_nn_kernel<T><<<grid, NT, 0, st>>>(rows, K, A, lda, B, ldb, C, ldc, kdyn_K, kdyn_N, kmaxN, 1 << 30);
}

// C (rows x N) = A (rows x K) B (K x N) with a static, long K split over
// blocks when there are few row tiles; partial holds 16 slices of rows x ldc.
template <typename T>
void launch_gemm_nn_splitk(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc,
                           T *partial, const int *kdyn_N, int kmaxN, cudaStream_t st)
{
    if (rows <= 0 || kmaxN <= 0) return;
    const int rblocks = (rows + TM - 1) / TM;
    int splits = 304 / rblocks;
    splits = std::min(splits, std::min(16, (K + 63) / 64));
    if (splits <= 1) {
        launch_gemm_nn<T>(rows, K, A, lda, B, ldb, C, ldc, nullptr, kdyn_N, kmaxN, st);
        return;
    }
    int ks = (K + splits - 1) / splits;
    ks = (ks + TK - 1) / TK * TK;
    splits = (K + ks - 1) / ks;
    dim3 grid(rblocks, (kmaxN + TN - 1) / TN, splits);
    CPCP_COUNT_LAUNCH();
    gemm_nn_kernel<T><<<grid, NT, 0, st>>>(rows, K, A, lda, B, ldb, partial, ldc, nullptr, kdyn_N, kmaxN, ks);
    launch_reduce_partial<T>(partial, splits, rows, (int)ldc, C, ldc, nullptr, kdyn_N, st);
}

// returns the number of splits used (partial holds splits x kmaxK x kmaxN)
template <typename T>
int launch_gemm_tn_partial(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *partial,
                           const int *kdyn_N, int kmaxN, int kmaxK, cudaStream_t st, const int *skip)
{
    // Gram matrices (K < 0) are small and reduced by one CTA: fewer, taller splits
    const int per = K < 0 ? 256 : 128;
    int splits = (rows + per - 1) / per;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
    int rps = (rows + splits - 1) / splits;
    rps = (rps + TK - 1) / TK * TK;
    splits = (rows + rps - 1) / rps;
    if (splits < 1) splits = 1;
    dim3 grid((kmaxK + TM - 1) / TM, (kmaxN + TN - 1) / TN, splits);
    // K dynamic when K < 0 (then the K dimension follows kdyn_N: Gram matrices)
    const int *kdynK = K < 0 ? kdyn_N : nullptr;
    CPCP_COUNT_LAUNCH();
    gemm_tn_partial_kernel<T><<<grid, NT, 0, st>>>(rows, K < 0 ? kmaxK : K, rps, A, lda, B, ldb, partial, kdynK,
                                                   kdyn_N, kmaxN, kmaxK, kmaxN, skip);
    return splits;
}

template <typename T>
void launch_reduce_partial(const T *partial, int splits, int K, int N, T *C, int64_t ldc, const int *kdyn_K,
                           const int *kdyn_N, cudaStream_t st)
{
    int64_t tot = (int64_t)K * N;
    int blocks = (int)((tot + 255) / 256);
    if (blocks < 1) return;
    CPCP_COUNT_LAUNCH();
    reduce_partial_kernel<T><<<blocks, 256, 0, st>>>(partial, splits, K, N, K, N, C, ldc, kdyn_K, kdyn_N);
}

template <typename T>
void launch_restrict(int m, int n, const T *M, int64_t ldm, T *MH, int64_t ldh, const TransferDev<T> &tr,
                     cudaStream_t st)
{
    dim3 grid((tr.nh + 127) / 128, std::min(m, 65535));
    CPCP_COUNT_LAUNCH();
    restrict_kernel<T><<<grid, 128, 0, st>>>(m, n, M, ldm, MH, ldh, tr);
}

template <typename T>
void launch_prolong(int n, const T *V, int64_t ldv, T *B, int64_t ldb, const TransferDev<T> &tr, const int *kdyn,
                    int kmax, cudaStream_t st)
{
    dim3 grid((kmax + 63) / 64, std::min(n, 65535));
    CPCP_COUNT_LAUNCH();
    prolong_kernel<T><<<grid, 64, 0, st>>>(n, V, ldv, B, ldb, tr, kdyn, kmax);
}

#define INST(T)                                                                                                    \
    template void launch_gemm_nn<T>(int, int, const T *, int64_t, const T *, int64_t, T *, int64_t, const int *,     \
                                    const int *, int, cudaStream_t);                                               \
    template void launch_gemm_nn_splitk<T>(int, int, const T *, int64_t, const T *, int64_t, T *, int64_t, T *,      \
                                           const int *, int, cudaStream_t);                                        \
    template int launch_gemm_tn_partial<T>(int, int, const T *, int64_t, const T *, int64_t, T *, const int *, int, \
                                           int, cudaStream_t, const int *);                                        \
    template void launch_reduce_partial<T>(const T *, int, int, int, T *, int64_t, const int *, const int *,        \
                                           cudaStream_t);                                                          \
    template void launch_restrict<T>(int, int, const T *, int64_t, T *, int64_t, const TransferDev<T> &,            \
                                     cudaStream_t);                                                                \
    template void launch_prolong<T>(int, const T *, int64_t, T *, int64_t, const TransferDev<T> &, const int *, int, \
                                    cudaStream_t);                                                                \
    template void launch_restrict_rows<T>(const T *, int64_t, T *, int64_t, const TransferDev<T> &, const int *, int, \
                                          cudaStream_t);                                                          \
    template void launch_transpose<T>(int, int, const T *, int64_t, T *, int64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cpcp
