// k_umma.cu -- the subspace-iteration contractions of the mixed-precision
// path on the 5th-generation tensor cores (tcgen05), BF16 operands with fp32
// accumulation in tensor memory.
//
// Both products of the range finder, Y = M_H Omega and Z = M_H^T Q (the two
// passes over the restricted iterate in each subspace step of the SVT,
// Sec. 4 and Alg. 4), are computed in the form
//
//     C[row][c] = sum_K A[row][K] * B[c][K]        (A: rows x K, B: N x K)
//
// with both operands K-major in global memory: the solver keeps M_H in BF16
// twice, as M_H (for Y) and as M_H^T (for Z), and the thin operand (Omega^T
// or Q^T) in BF16 as N x K.  One CTA owns a 128-row panel of A and a slice of
// K (split-K), streams 128 x 64 tiles of A and N x 64 tiles of B through a
// four-stage TMA / mbarrier pipeline into 128-byte-swizzled shared memory, and
// one elected thread issues tcgen05.mma (M = 128, N = round16(k), K = 16) into
// a TMEM accumulator.  The epilogue reads the accumulator with tcgen05.ld and
// writes fp32 split-K partials, which a fixed-order reduction sums (so the
// result is deterministic).
//
// Every wait on an mbarrier is bounded (about one second of %globaltimer);
// on expiry the kernel raises an error flag that the host turns into
// CPCP_ERR_TIMEOUT, drains its own copies in flight and frees its TMEM.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"

namespace cpcp {

namespace {

constexpr int BM = 128;       // rows of one UMMA tile (TMEM lanes)
constexpr int BK = 64;        // K elements per stage: 128 bytes of BF16 = one swizzle row
constexpr int STAGES = 4;
constexpr int NT = 128;       // four warps: producer, MMA issuer, TMEM owner; all four read TMEM out
constexpr uint32_t A_STAGE_BYTES = BM * BK * 2;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of parity `parity` to complete; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 64; i++)
            if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > 1000000000ull) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row swizzle atoms 1024 bytes apart (stride byte offset); the
// leading byte offset is unused for this layout and set to 16 bytes.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *p)
{
    const uint64_t addr = smem_u32(p);
    uint64_t d = (addr >> 4) & 0x3FFFull;
    d |= (uint64_t)(16 >> 4) << 16;    // leading dimension byte offset
    d |= (uint64_t)(1024 >> 4) << 32;  // stride dimension byte offset
    d |= 1ull << 46;                   // descriptor version of tcgen05
    d |= 2ull << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: fp32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n (multiple of 16).
__device__ __forceinline__ uint32_t idesc_bf16(int n)
{
    return (1u << 4)                        // accumulator format fp32
           | (1u << 7)                      // A format BF16
           | (1u << 10)                     // B format BF16
           | ((uint32_t)(n >> 3) << 17)     // N / 8
           | ((uint32_t)(BM >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// partial[(split * rows_max + row) * ldp + c] = sum over this split's K range
// of A[row][K] B[c][K], for c < N = round16(*kdyn) (at most nbox).
__global__ void __launch_bounds__(NT, 1)
    umma_tn_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, int rows,
                   int kblocks, int kb_per_split, int nbox, uint32_t tmem_cols, const int *__restrict__ kdyn,
                   float *__restrict__ partial, int rows_max, int ldp, int *__restrict__ err)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t b_stage_bytes = (uint32_t)nbox * BK * 2;
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_STAGE_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + STAGES * b_stage_bytes);
    uint64_t *empty = full + STAGES;
    uint64_t *done = empty + STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    int *flags = reinterpret_cast<int *>(tmem_slot + 1);  // [0] failure, [1] stages consumed

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int split = blockIdx.y;
    const int kb0 = split * kb_per_split;
    const int nkb = min(kblocks, kb0 + kb_per_split) - kb0;
    int n = kdyn ? *kdyn : nbox;
    n = (n + 15) / 16 * 16;
    n = max(16, min(n, nbox));

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        flags[0] = 0;
        flags[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (threadIdx.x == 0) {
        // producer: one TMA load of A and of B per stage
        for (int i = 0; i < nkb; i++) {
            const int s = i % STAGES;
            if (i >= STAGES && !mbar_wait(&empty[s], ((i / STAGES) & 1) ^ 1)) {
                flags[0] = 1;
                break;
            }
            mbar_expect_tx(&full[s], A_STAGE_BYTES + b_stage_bytes);
            const int kx = (kb0 + i) * BK;
            tma_load_2d(sA + s * A_STAGE_BYTES, &mapA, &full[s], kx, blockIdx.x * BM);
            tma_load_2d(sB + s * b_stage_bytes, &mapB, &full[s], kx, 0);
            issued = i + 1;
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        const uint32_t idesc = idesc_bf16(n);
        int consumed = 0;
        for (int i = 0; i < nkb; i++) {
            const int s = i % STAGES;
            if (!mbar_wait(&full[s], (i / STAGES) & 1)) {
                flags[0] = 1;
                break;
            }
            tc_fence_after();
            const uint64_t ad = smem_desc_sw128(sA + s * A_STAGE_BYTES);
            const uint64_t bd = smem_desc_sw128(sB + s * b_stage_bytes);
#pragma unroll
            for (int kk = 0; kk < BK / 16; kk++)  // 16 BF16 = 32 bytes = 2 descriptor units per step
                umma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&empty[s]);
            consumed = i + 1;
        }
        flags[1] = consumed;
        umma_commit(done);  // arrives when every MMA issued above has completed
    }

    // epilogue: each warp reads its 32 TMEM lanes (rows), 16 columns at a
    // time, and stores the columns c < min(k, ldp) of its rows
    const bool ok = mbar_wait(done, 0);
    tc_fence_after();
    __syncwarp();
    const int row = blockIdx.x * BM + warp * 32 + lane;
    const int kv = min(kdyn ? *kdyn : nbox, ldp);
    float *out = partial + ((int64_t)split * rows_max + row) * ldp;
    for (int c0 = 0; c0 < n; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (row < rows) {
#pragma unroll
            for (int j = 0; j < 16; j++)
                if (c0 + j < kv) out[c0 + j] = (ok && nkb > 0) ? v[j] : 0.f;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        // drain loads that were issued but never consumed (only after a failure)
        for (int i = flags[1]; i < issued; i++) mbar_wait(&full[i % STAGES], (i / STAGES) & 1);
        if (!ok || flags[0]) atomicExch(err, 1);
    }
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

// fp32 X (rows x cols, ldx) -> BF16 copies: Xb (same orientation, rows_b x
// ldb, zero outside rows x cols) and/or Xt (transposed, rows_t x ldt, zero
// outside cols x rows).  32 x 32 tiles through shared memory.
__global__ void bf16_pair_kernel(int rows, int cols, const float *__restrict__ X, int64_t ldx,
                                 __nv_bfloat16 *__restrict__ Xb, int rows_b, int64_t ldb,
                                 __nv_bfloat16 *__restrict__ Xt, int rows_t, int64_t ldt)
{
    __shared__ float tile[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + tx;
        const float v = (r < rows && c < cols) ? X[(int64_t)r * ldx + c] : 0.f;
        tile[i][tx] = v;
        if (Xb != nullptr && r < rows_b && c < ldb) Xb[(int64_t)r * ldb + c] = __float2bfloat16_rn(v);
    }
    if (Xt == nullptr) return;
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + tx;  // Xt[c][r] = X[r][c]
        if (c < rows_t && r < ldt) Xt[(int64_t)c * ldt + r] = __float2bfloat16_rn(tile[tx][i]);
    }
}

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point
// (the library links only the CUDA runtime)
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// 2-D BF16 tensor map over a row-major (outer x inner) array with leading
// dimension ld elements; boxes of box_outer rows x 64 columns, 128-byte swizzle.
bool make_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t outer, uint64_t ld, uint32_t box_outer)
{
    EncodeTiledFn fn = encode_fn();
    if (fn == nullptr) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int umma_pad_rows(int rows) { return (rows + BM - 1) / BM * BM; }
int umma_pad_k(int k) { return (k + BK - 1) / BK * BK; }

void launch_bf16_pair(int rows, int cols, const float *X, int64_t ldx, __nv_bfloat16 *Xb, int rows_b, int64_t ldb,
                      __nv_bfloat16 *Xt, int rows_t, int64_t ldt, cudaStream_t st)
{
    // cover the padded extents so that the padding is written with zeros
    int R = rows, C = cols;
    if (Xb) {
        R = max(R, rows_b);
        C = max(C, (int)ldb);
    }
    if (Xt) {
        R = max(R, (int)ldt);
        C = max(C, rows_t);
    }
    dim3 grid((C + 31) / 32, (R + 31) / 32);
    CPCP_COUNT_LAUNCH();
    bf16_pair_kernel<<<grid, 256, 0, st>>>(rows, cols, X, ldx, Xb, rows_b, ldb, Xt, rows_t, ldt);
}

// C partials of A (rows_pad x kpad BF16, ld lda, zero padded) times B^T
// (nrows_b x kpad BF16, ld ldb, zero padded); N is round16(*kdyn) <= nbox <=
// nrows_b.  Returns the number of K splits written to `partial`
// (splits x rows x ldp fp32), or -1 when the tensor maps cannot be made.
int launch_umma_tn(int rows, int rows_pad, int kpad, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *B,
                   int nrows_b, int64_t ldb, int nbox, const int *kdyn, float *partial, int ldp, int max_splits,
                   int *err, cudaStream_t st)
{
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, (uint64_t)kpad, (uint64_t)rows_pad, (uint64_t)lda, BM)) return -1;
    if (!make_map(&mb, B, (uint64_t)kpad, (uint64_t)nrows_b, (uint64_t)ldb, (uint32_t)nbox)) return -1;
    const int kblocks = kpad / BK;
    const int tiles = rows_pad / BM;
    // enough CTAs to cover the 152 SMs about twice, at least two K blocks per split
    int splits = (2 * 152 + tiles - 1) / tiles;
    splits = min(splits, max(1, kblocks / 2));
    splits = max(1, min(splits, max_splits));
    const int per = (kblocks + splits - 1) / splits;
    splits = (kblocks + per - 1) / per;
    uint32_t cols = 32;
    while ((int)cols < nbox) cols <<= 1;
    const size_t smem = 1024 + STAGES * ((size_t)A_STAGE_BYTES + (size_t)nbox * BK * 2) + 128;
    static size_t smem_set = 0;
    if (smem > smem_set) {
        if (cudaFuncSetAttribute(umma_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return -1;
        smem_set = smem;
    }
    dim3 grid(tiles, splits);
    CPCP_COUNT_LAUNCH();
    umma_tn_kernel<<<grid, NT, smem, st>>>(ma, mb, rows, kblocks, per, nbox, cols, kdyn, partial, rows, ldp, err);
    return splits;
}

}  // namespace cpcp
