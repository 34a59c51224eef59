// k_tsgemm.cu -- the tall-skinny contractions of the subspace-iteration SVD
// (Sec. 2.2 randomized/subspace SVD; Alg. 4 coarse step) on the SIMT cores:
//
//   ts_nn   C = A B     Y = M_H Omega (K = n_H long), Q = X R^{-1}, U = Q Ut, ...
//   ts_tn   C = A^T B   Z = M_H^T Q (K = m long), Gram matrices X^T X
//
// Tiles of 64 x 64 outputs, 256 threads with 4 x 4 register tiles, and a
// three-stage cp.async pipeline over K chunks.  A long K is split over the
// CTAs of one thread-block cluster (up to 8): each CTA leaves its partial tile
// in shared memory and, after a cluster barrier, every CTA sums a slice of
// rows over the cluster's tiles through distributed shared memory in rank
// order.  The reduction order is fixed, so results are bit-reproducible run to
// run, and no partial buffer or second launch is needed.  Gram matrices can
// use several clusters over disjoint row ranges, each writing one partial
// slice that the Cholesky kernel sums in a fixed order.
//
// Widths that change during a solve (the subspace width k) are read from
// device memory; grids are sized for the maximum width and tiles beyond the
// live width return at once (a whole cluster shares its column tile).
#include <algorithm>

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace cpcp {

namespace {

constexpr int TS_BM = 64, TS_BN = 64, TS_NT = 256, TS_ST = 3;

template <typename T>
struct TsCfg {
    static constexpr int TK = sizeof(T) == 4 ? 32 : 16;  // K chunk
    static constexpr int V = 16 / sizeof(T);             // elements per 16-byte copy
    static constexpr int LDA_NN = TK + 4;                // A stage, NN: [BM][TK + 4]
    static constexpr int LDA_TN = TS_BM + 4;             // A stage, TN: [TK][BM + 4]
    static constexpr int LDB = TS_BN + 4;                // B stage: [TK][BN + 4]
    static constexpr int A_ELEMS = TS_BM * (TK + 4) > TK * (TS_BM + 4) ? TS_BM * (TK + 4) : TK * (TS_BM + 4);
    static constexpr int B_ELEMS = TK * (TS_BN + 4);
    static constexpr int STAGE = A_ELEMS + B_ELEMS;
    static constexpr int LDC = TS_BN + 4;  // partial tile for the cluster reduction
};

template <typename T>
size_t ts_smem()
{
    const size_t pipe = (size_t)TS_ST * TsCfg<T>::STAGE * sizeof(T);
    const size_t red = (size_t)TS_BM * TsCfg<T>::LDC * sizeof(T);
    return std::max(pipe, red);
}

// 16-byte asynchronous copy global -> shared; bytes < 16 zero-fills the rest
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ld4(const float *p, float (&v)[4])
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4])
{
    const double2 q0 = *reinterpret_cast<const double2 *>(p);
    const double2 q1 = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = q0.x;
    v[1] = q0.y;
    v[2] = q1.x;
    v[3] = q1.y;
}

// one 16-byte piece of a row of `len` valid elements starting at element x
// (x a multiple of V): the bytes that lie inside the row, the rest zero
template <typename T>
__device__ __forceinline__ void load_piece(T *dst, const T *row, int x, int len, bool ok)
{
    constexpr int V = TsCfg<T>::V;
    int valid = ok ? len - x : 0;
    valid = valid < 0 ? 0 : (valid > V ? V : valid);
    cp_async16(dst, valid > 0 ? (const void *)(row + x) : (const void *)row, valid * (int)sizeof(T));
}

// C (rows x N, ld ldc) = A B (NN: A rows x K) or A^T B (TN: A K x rows), B K x N.
// Grid: x = cluster rank + cl * group, y = row tile, z = column tile.  Group g
// sums the K range [g, g + 1) / groups and writes to C + g * slice.  kdynR:
// live number of rows (Gram matrices: the width k).  skip: when *skip is set,
// NN (no cluster) writes C = A (the factor is the identity) and TN does nothing.
template <typename T, bool TN>
__global__ void __launch_bounds__(TS_NT)
    ts_gemm_kernel(int Rstat, int Kstat, const T *__restrict__ A, int64_t lda, const T *__restrict__ B, int64_t ldb,
                   T *__restrict__ C, int64_t ldc, int64_t slice, const int *kdynR, const int *kdynK,
                   const int *kdynN, int Nstat, int ks, const int *skip)
{
    pdl_enter();
    using Cfg = TsCfg<T>;
    constexpr int TK = Cfg::TK, V = Cfg::V;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    const int cl = (int)(cg::this_cluster().num_blocks());
    const int rank = (int)blockIdx.x % cl, group = (int)blockIdx.x / cl;
    const int rows = kdynR ? *kdynR : Rstat;
    const int K = kdynK ? *kdynK : Kstat;
    const int N = kdynN ? *kdynN : Nstat;
    const int rb = blockIdx.y * TS_BM, cb = blockIdx.z * TS_BN;
    if (cb >= N || rb >= rows) return;  // the whole cluster shares this tile
    if (TN && skip != nullptr && *skip) return;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;

    if (!TN && skip != nullptr && *skip) {
        // C = A on this tile: every load issued before the first store
        constexpr int PER = TS_BM * TS_BN / TS_NT;
        T v[PER];
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int idx = t + TS_NT * u, r = rb + idx / TS_BN, c = cb + idx % TS_BN;
            v[u] = (r < rows && c < N) ? A[(int64_t)r * lda + c] : T(0);
        }
#pragma unroll
        for (int u = 0; u < PER; u++) {
            const int idx = t + TS_NT * u, r = rb + idx / TS_BN, c = cb + idx % TS_BN;
            if (r < rows && c < N) C[(int64_t)r * ldc + c] = v[u];
        }
        return;
    }

    const int split = (int)blockIdx.x;  // position of this CTA's K range
    const int kbeg = min(K, split * ks), kend = min(K, kbeg + ks);
    const int nch = (kend - kbeg + TK - 1) / TK;
    C += (int64_t)group * slice;

    // stage s: A at sm + s * STAGE, B after it
    auto issue = [&](int ch, int s) {
        T *As = sm + s * Cfg::STAGE;
        T *Bs = As + Cfg::A_ELEMS;
        const int k0 = kbeg + ch * TK;
        if (!TN) {
            // A rows rb.. (BM rows), K columns k0.. (TK): TK / V pieces per row
            constexpr int PR = TK / V;
            for (int idx = t; idx < TS_BM * PR; idx += TS_NT) {
                const int r = idx / PR, x = (idx % PR) * V;
                const int gr = rb + r;
                const T *row = A + (int64_t)(gr < rows ? gr : 0) * lda + k0;
                load_piece(As + r * Cfg::LDA_NN + x, row, x, kend - k0, gr < rows);
            }
        } else {
            // A rows k0.. (TK rows of K), columns rb.. (BM): BM / V pieces per row
            constexpr int PR = TS_BM / V;
            for (int idx = t; idx < TK * PR; idx += TS_NT) {
                const int r = idx / PR, x = (idx % PR) * V;
                const int gk = k0 + r;
                const T *row = A + (int64_t)(gk < kend ? gk : kbeg) * lda + rb;
                load_piece(As + r * Cfg::LDA_TN + x, row, x, rows - rb, gk < kend);
            }
        }
        constexpr int PB = TS_BN / V;
        for (int idx = t; idx < TK * PB; idx += TS_NT) {
            const int r = idx / PB, x = (idx % PB) * V;
            const int gk = k0 + r;
            const T *row = B + (int64_t)(gk < kend ? gk : kbeg) * ldb + cb;
            load_piece(Bs + r * Cfg::LDB + x, row, x, N - cb, gk < kend);
        }
    };

    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = T(0);

#pragma unroll
    for (int s = 0; s < TS_ST - 1; s++) {
        if (s < nch) issue(s, s);
        cp_async_commit();
    }
    for (int ch = 0; ch < nch; ch++) {
        if (ch + TS_ST - 1 < nch) issue(ch + TS_ST - 1, (ch + TS_ST - 1) % TS_ST);
        cp_async_commit();
        cp_async_wait<TS_ST - 1>();
        __syncthreads();
        const T *As = sm + (ch % TS_ST) * Cfg::STAGE;
        const T *Bs = As + Cfg::A_ELEMS;
        // the TK terms of a chunk are summed apart and then added to the total
        // (rounding ~ (sqrt(TK) + sqrt(K / TK)) eps rather than sqrt(K) eps)
        T part[4][4];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) part[i][j] = T(0);
        if (!TN) {
#pragma unroll
            for (int kq = 0; kq < TK / 4; kq++) {
                T a[4][4];
#pragma unroll
                for (int i = 0; i < 4; i++) ld4(As + (4 * ty + i) * Cfg::LDA_NN + 4 * kq, a[i]);
#pragma unroll
                for (int kk = 0; kk < 4; kk++) {
                    T b[4];
                    ld4(Bs + (4 * kq + kk) * Cfg::LDB + 4 * tx, b);
#pragma unroll
                    for (int i = 0; i < 4; i++)
#pragma unroll
                        for (int j = 0; j < 4; j++) part[i][j] = fma(a[i][kk], b[j], part[i][j]);
                }
            }
        } else {
#pragma unroll
            for (int kk = 0; kk < TK; kk++) {
                T a[4], b[4];
                ld4(As + kk * Cfg::LDA_TN + 4 * ty, a);
                ld4(Bs + kk * Cfg::LDB + 4 * tx, b);
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) part[i][j] = fma(a[i], b[j], part[i][j]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[i][j] += part[i][j];
        __syncthreads();
    }
    cp_async_wait<0>();

    if (cl == 1) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int r = rb + 4 * ty + i;
            if (r >= rows) continue;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int c = cb + 4 * tx + j;
                if (c < N) C[(int64_t)r * ldc + c] = acc[i][j];
            }
        }
        return;
    }

    // cluster reduction: partial tiles in shared memory, then rank q sums
    // rows [q BM / cl, (q + 1) BM / cl) over ranks 0, 1, ... in order
    cg::cluster_group cluster = cg::this_cluster();
    T *Ct = sm;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) Ct[(4 * ty + i) * Cfg::LDC + 4 * tx + j] = acc[i][j];
    cluster.sync();
    const int per = TS_BM / cl;
    for (int idx = t; idx < per * TS_BN; idx += TS_NT) {
        const int lr = rank * per + idx / TS_BN, c = idx % TS_BN;
        T s = T(0);
        for (int q = 0; q < cl; q++) {
            const T *rem = cluster.map_shared_rank(Ct, q);
            s += rem[lr * Cfg::LDC + c];
        }
        const int r = rb + lr, gc = cb + c;
        if (r < rows && gc < N) C[(int64_t)r * ldc + gc] = s;
    }
    cluster.sync();  // keep this CTA's tile alive until every rank has read it
}

template <typename T, bool TN>
void ts_launch(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc, int64_t slice,
               const int *kdynR, const int *kdynK, const int *kdynN, int kmaxN, int cl, int groups, int Kmax,
               const int *skip, cudaStream_t st)
{
    // (a cluster of 16 that the device refuses is launched as 8, each CTA
    // then covering twice the K range; only single-slice launches ask for 16)
    static bool attr = false;
    static bool wide_ok = false;  // clusters of 16 (beyond the portable 8) accepted
    if (!attr) {
        cudaFuncSetAttribute(ts_gemm_kernel<T, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts_smem<T>());
        wide_ok = cudaFuncSetAttribute(ts_gemm_kernel<T, TN>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                  cudaSuccess;
        cudaGetLastError();
        attr = true;
    }
    if (cl > 8 && !wide_ok) cl = 8;
    // K range per CTA: a multiple of the chunk, covering Kmax over cl * groups CTAs
    const int parts = cl * groups;
    int ks = (Kmax + parts - 1) / parts;
    ks = (ks + TsCfg<T>::TK - 1) / TsCfg<T>::TK * TsCfg<T>::TK;
    if (ks < TsCfg<T>::TK) ks = TsCfg<T>::TK;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)parts, (unsigned)((rows + TS_BM - 1) / TS_BM), (unsigned)((kmaxN + TS_BN - 1) / TS_BN));
    cfg.blockDim = dim3(TS_NT);
    cfg.dynamicSmemBytes = ts_smem<T>();
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = g_pdl ? 2 : 1;
    CPCP_COUNT_LAUNCH();
    cudaError_t e = cudaLaunchKernelEx(&cfg, ts_gemm_kernel<T, TN>, rows, K, A, lda, B, ldb, C, ldc, slice, kdynR,
                                       kdynK, kdynN, kmaxN, ks, skip);
    if (e != cudaSuccess && cl > 8) {
        // the device would not co-schedule 16 CTAs of this size: use 8 from now on
        cudaGetLastError();
        wide_ok = false;
        at[0].val.clusterDim.x = 8;
        ks = (Kmax + 8 * groups - 1) / (8 * groups);
        ks = (ks + TsCfg<T>::TK - 1) / TsCfg<T>::TK * TsCfg<T>::TK;
        cfg.gridDim.x = (unsigned)(8 * groups);
        cudaLaunchKernelEx(&cfg, ts_gemm_kernel<T, TN>, rows, K, A, lda, B, ldb, C, ldc, slice, kdynR, kdynK, kdynN,
                           kmaxN, ks, skip);
    }
}

int ts_cluster_for(int tiles, int K)
{
    // split a long K over a cluster (up to 8 CTAs) until about two CTAs per
    // SM are busy, keeping at least 128 terms per CTA (clusters of 16, 64
    // terms per CTA, measured slower at 2000 x 2000)
    int cl = 1;
    while (cl < 8 && tiles * cl < 304 && K >= 128 * cl * 2) cl *= 2;
    return cl;
}

template <typename T>
bool aligned16(const T *p, int64_t ld)
{
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld * (int64_t)sizeof(T)) % 16 == 0;
}

}  // namespace

template <typename T>
bool launch_ts_nn(int rows, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc,
                  const int *kdyn_K, const int *kdyn_N, int kmaxK, int kmaxN, const int *skip, cudaStream_t st)
{
    if (!aligned16(A, lda) || !aligned16(B, ldb)) return false;
    if (rows <= 0 || kmaxN <= 0) return true;
    const int Kmax = kdyn_K ? kmaxK : K;
    const int tiles = (rows + TS_BM - 1) / TS_BM;
    const int cl = (kdyn_K || skip) ? 1 : ts_cluster_for(tiles, K);
    ts_launch<T, false>(rows, K, A, lda, B, ldb, C, ldc, 0, nullptr, kdyn_K, kdyn_N, kmaxN, cl, 1, Kmax, skip, st);
    return true;
}

template <typename T>
bool launch_ts_tn(int P, int K, const T *A, int64_t lda, const T *B, int64_t ldb, T *C, int64_t ldc,
                  const int *kdyn_N, int kmaxN, cudaStream_t st)
{
    if (!aligned16(A, lda) || !aligned16(B, ldb)) return false;
    if (P <= 0 || kmaxN <= 0) return true;
    const int tiles = (P + TS_BM - 1) / TS_BM;
    ts_launch<T, true>(P, K, A, lda, B, ldb, C, ldc, 0, nullptr, nullptr, kdyn_N, kmaxN, ts_cluster_for(tiles, K),
                       1, K, nullptr, st);
    return true;
}

template <typename T>
int launch_ts_gram(int rows, const T *X, int64_t ldx, T *partial, const int *kdyn, int kmax, const int *skip,
                   cudaStream_t st)
{
    // X^T X (k x k, k = *kdyn): clusters of up to 8 CTAs over disjoint row
    // ranges, one partial slice (kmax x kmax) per cluster; -1 when X is not
    // 16-byte aligned (the caller then uses the plain kernels)
    if (!aligned16(X, ldx)) return -1;
    const int cl = rows >= 1024 ? 8 : (rows >= 256 ? 4 : 1);
    int groups = (rows + 64 * cl - 1) / (64 * cl);
    groups = std::max(1, std::min(groups, 4));
    ts_launch<T, true>(kmax, rows, X, ldx, X, ldx, partial, kmax, (int64_t)kmax * kmax, kdyn, nullptr, kdyn, kmax, cl,
                       groups, rows, skip, st);
    return groups;
}

#define INST(T)                                                                                                     \
    template bool launch_ts_nn<T>(int, int, const T *, int64_t, const T *, int64_t, T *, int64_t, const int *,       \
                                  const int *, int, int, const int *, cudaStream_t);                                \
    template bool launch_ts_tn<T>(int, int, const T *, int64_t, const T *, int64_t, T *, int64_t, const int *, int,  \
                                  cudaStream_t);                                                                    \
    template int launch_ts_gram<T>(int, const T *, int64_t, T *, const int *, int, const int *, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cpcp
