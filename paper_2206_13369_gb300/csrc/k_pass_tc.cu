// k_pass_tc.cu -- the fused fine-level iteration pass (momentum, masked
// gradient eq. (cpcp-grad-LS), l1 shrink, M = L-hat - tau G; Alg. 4 on the
// finest level) with the rank-K contraction
//
//     L-hat = (1 + beta) A_k B_k^T - beta A_{k-1} B_{k-1}^T = A^ B^^T,
//     A^ = [(1 + beta) A_k, -beta A_{k-1}],  B^ = [B_k, B_{k-1}],
//
// on the 5th-generation tensor cores.  fp32 accuracy from TF32 operands: each
// factor entry is split as x = x_h + x_m + x_l, three TF32 numbers taken by
// successive round-to-nearest (11 significant bits each, so the split is exact
// to 2^-33), and
//     a b ~ a_m b_m + a_l b_h + a_h b_l + a_m b_h + a_h b_m + a_h b_h
// (the dropped terms are below 2^-32 relative).  The five small products
// accumulate in one fp32 TMEM accumulator and a_h b_h in another; the
// epilogue adds the two in fp32.  Each operand stage holds the three parts of
// a 16-wide K slice of A^ and of B^ (64-byte swizzle), and the MMA issuer
// pairs them: six MMAs per K step of 8.
//
// Measured alternatives, each worse on the 2000 x 2000 rank-50 workload:
// two-term splitting (a_h b_h + a_h b_l + a_l b_h) represents a factor only
// to 2^-22, and one accumulator shared by all six products loses the small
// terms' low bits to the large running sum; both left a rel-KKT floor near
// 1.7e-6, because the momentum step cancels most of L-hat.  Laying the six
// products out as one contraction over an extended K = 6 K re-read the
// operands six times from L2.
//
// One persistent CTA per SM walks 128 x 128 output tiles.  Warp roles:
//   warp 0   TMA producer of the operand stages (A^ and B^, three parts each)
//   warp 1   MMA issuer: tcgen05.mma kind::tf32, M = 128, N = 128, K = 8
//   warp 2   TMEM allocator (per buffer a 128-column accumulator for a_h b_h and
//            one for the small products; two buffers: all 512 columns)
//   warp 3   TMA producer of the epilogue tiles: D, S_k, S_{k-1} in 32-column
//            quarters (128-byte swizzle), double buffered
//   warps 4-7 epilogue: tcgen05.ld of the accumulator (one TMEM lane quarter
//            per warp, one row per thread), the elementwise step, stores.
// So the HBM stream of the epilogue inputs runs while the tensor cores work
// on the next tile, and the operands (L2-resident factors) never touch the
// SIMT pipes.
//
// Every mbarrier wait is bounded (about one second of %globaltimer) and also
// ends when another role has given up (a shared abort flag); the kernel then
// raises the error flag that the host turns into CPCP_ERR_TIMEOUT, drains the
// copies it issued and frees its TMEM.
#include <cuda.h>

#include <mutex>

#include "common.cuh"

namespace cpcp {

namespace {

constexpr int TBM = 128;   // tile rows = TMEM lanes
constexpr int TBN = 128;   // tile columns = accumulator columns
constexpr int TBK = 16;    // K per operand stage: 64 bytes of fp32
constexpr int HALF = 32;   // epilogue sub-tile columns (128 bytes of fp32)
constexpr int OPS = 2;     // operand stages
constexpr int EPS = 2;     // epilogue sub-tile buffers
constexpr int NT = 256;
constexpr uint32_t A_BYTES = TBM * TBK * 4;             // 8 KB per part
constexpr uint32_t B_BYTES = TBN * TBK * 4;             // 8 KB per part
constexpr uint32_t OP_BYTES = 3 * A_BYTES + 3 * B_BYTES;  // three parts of each
constexpr uint32_t EP_TILE = TBM * HALF * 4;            // 16 KB per array
constexpr uint32_t EP_BYTES = 3 * EP_TILE;              // D, S_k, S_{k-1}
constexpr uint32_t TMEM_COLS = 4 * TBN;  // two buffers x (large, small)
constexpr size_t SMEM_BYTES = 1024 + OPS * (size_t)OP_BYTES + EPS * (size_t)EP_BYTES + 256;

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

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Wait for the phase of parity `parity`; false after ~1 s or once *abort is
// set (abort == nullptr: the time bound only).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        for (int i = 0; i < 64; i++)
            if (mbar_try_wait(bar, parity)) return true;
        if (abort != nullptr && *abort) return false;
        if (globaltimer_ns() - t0 > 1000000000ull) {
            if (abort != nullptr) *abort = 1;
            return false;
        }
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

// K-major operand, 64-byte swizzle, 64-byte rows, 8-row atoms 512 bytes apart
__device__ __forceinline__ uint64_t smem_desc_sw64(const void *p)
{
    const uint64_t addr = smem_u32(p);
    uint64_t d = (addr >> 4) & 0x3FFFull;
    d |= (uint64_t)(16 >> 4) << 16;   // leading dimension byte offset (unused here)
    d |= (uint64_t)(512 >> 4) << 32;  // stride dimension byte offset
    d |= 1ull << 46;                  // descriptor version of tcgen05
    d |= 4ull << 61;                  // 64-byte swizzle
    return d;
}

// kind::tf32: fp32 accumulator, TF32 A and B (both K-major), M = 128, N = 128
__device__ __forceinline__ uint32_t idesc_tf32()
{
    return (1u << 4)                        // accumulator format fp32
           | (2u << 7)                      // A format TF32
           | (2u << 10)                     // B format TF32
           | ((uint32_t)(TBN >> 3) << 17)   // N / 8
           | ((uint32_t)(TBM >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
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

__device__ __forceinline__ float tf32_rn(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// live K of the contraction (the same on every role); the extended K is 6 K
__device__ __forceinline__ int live_k(const int *rk, const int *rp, const Ctrl *ctrl)
{
    const int a = rk ? *rk : 0;
    const int b = (rp && ctrl->beta != 0.0) ? *rp : 0;
    return a + b;
}

struct TcMaps {
    CUtensorMap a[3], b[3];  // split factors: high, middle, low parts (K-major, 64-byte swizzle)
    CUtensorMap d, sk, sp;   // epilogue inputs (32-column boxes, 128-byte swizzle)
};

struct TcArgs {
    int m, n;
    const uint32_t *Q;
    int64_t ldq;
    float *Sout;
    int64_t ldso;
    float *M;
    int64_t ldm;
    const int *rk, *rp;
    const Ctrl *ctrl;
    int has_sp;
    int *err;
};

// element (r, c) of a 128-row x 32-column fp32 TMA box with 128-byte swizzle
__device__ __forceinline__ const float4 *swz4(const uint8_t *tile, int r, int c4)
{
    return reinterpret_cast<const float4 *>(tile + r * 128 + ((c4 ^ (r & 7)) << 4));
}

__global__ void __launch_bounds__(NT, 1) pass_tc_kernel(const __grid_constant__ TcMaps maps, TcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sOp = smem;                        // OPS x [A hi | A lo | B hi | B lo]
    uint8_t *sEp = smem + OPS * OP_BYTES;       // EPS x [D | S_k | S_{k-1}]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sEp + EPS * EP_BYTES);
    uint64_t *op_full = bars, *op_empty = bars + OPS;
    uint64_t *ep_full = bars + 2 * OPS, *ep_empty = ep_full + EPS;
    uint64_t *acc_full = ep_empty + EPS, *acc_empty = acc_full + 2;
    uint64_t *mma_done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_n = (a.n + TBN - 1) / TBN;
    const int ntiles = ((a.m + TBM - 1) / TBM) * tiles_n;
    const int K = live_k(a.rk, a.rp, a.ctrl);
    const int nkb = (K + TBK - 1) / TBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OPS; s++) {
            mbar_init(&op_full[s], 1);
            mbar_init(&op_empty[s], 1);
        }
        for (int s = 0; s < EPS; s++) {
            mbar_init(&ep_full[s], 1);
            mbar_init(&ep_empty[s], 4);  // one arrival per epilogue warp
        }
        for (int s = 0; s < 2; s++) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 4);
        }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // operand producer
        if (lane == 0) {
            int i = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const int rb = (t / tiles_n) * TBM, cb = (t % tiles_n) * TBN;
                for (int kb = 0; kb < nkb; kb++, i++) {
                    const int s = i % OPS;
                    if (i >= OPS && !mbar_wait(&op_empty[s], ((i / OPS) & 1) ^ 1, abort_flag)) break;
                    uint8_t *st = sOp + s * OP_BYTES;
                    mbar_expect_tx(&op_full[s], OP_BYTES);
#pragma unroll
                    for (int q = 0; q < 3; q++) {
                        tma_load_2d(st + q * A_BYTES, &maps.a[q], &op_full[s], kb * TBK, rb);
                        tma_load_2d(st + 3 * A_BYTES + q * B_BYTES, &maps.b[q], &op_full[s], kb * TBK, cb);
                    }
                }
            }
            // drain: the last phase issued on each stage has landed (time bound
            // only: no copy may still be in flight when the CTA exits)
            for (int s = 0; s < OPS && s < i; s++) {
                const int last = i - 1 - ((i - 1 - s) % OPS);
                if (!mbar_wait(&op_full[s], (last / OPS) & 1, nullptr)) *abort_flag = 1;
            }
        }
    } else if (warp == 3) {
        // epilogue-input producer
        if (lane == 0) {
            int i = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const int rb = (t / tiles_n) * TBM, cb = (t % tiles_n) * TBN;
                for (int h = 0; h < TBN / HALF; h++, i++) {
                    const int s = i % EPS;
                    if (i >= EPS && !mbar_wait(&ep_empty[s], ((i / EPS) & 1) ^ 1, abort_flag)) break;
                    uint8_t *st = sEp + s * EP_BYTES;
                    mbar_expect_tx(&ep_full[s], a.has_sp ? EP_BYTES : 2 * EP_TILE);
                    tma_load_2d(st, &maps.d, &ep_full[s], cb + h * HALF, rb);
                    tma_load_2d(st + EP_TILE, &maps.sk, &ep_full[s], cb + h * HALF, rb);
                    if (a.has_sp) tma_load_2d(st + 2 * EP_TILE, &maps.sp, &ep_full[s], cb + h * HALF, rb);
                }
            }
            for (int s = 0; s < EPS && s < i; s++) {
                const int last = i - 1 - ((i - 1 - s) % EPS);
                if (!mbar_wait(&ep_full[s], (last / EPS) & 1, nullptr)) *abort_flag = 1;
            }
        }
    } else if (warp == 1) {
        // MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32();
            int i = 0, lt = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, lt++) {
                const int buf = lt & 1;
                if (lt >= 2 && !mbar_wait(&acc_empty[buf], ((lt >> 1) - 1) & 1, abort_flag)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * 2 * TBN);  // a_h b_h
                const uint32_t dsm = d + (uint32_t)TBN;               // the five small products
                bool ok = true;
                for (int kb = 0; kb < nkb; kb++, i++) {
                    const int s = i % OPS;
                    if (!mbar_wait(&op_full[s], (i / OPS) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint8_t *st = sOp + s * OP_BYTES;
                    uint64_t ad[3], bd[3];
#pragma unroll
                    for (int q = 0; q < 3; q++) {
                        ad[q] = smem_desc_sw64(st + q * A_BYTES);
                        bd[q] = smem_desc_sw64(st + 3 * A_BYTES + q * B_BYTES);
                    }
                    // parts (0 = h, 1 = m, 2 = l) of the five small products
                    constexpr int PA[5] = {1, 2, 0, 1, 0}, PB[5] = {1, 0, 2, 0, 1};
#pragma unroll
                    for (int kk = 0; kk < TBK / 8; kk++) {  // 8 TF32 = 32 bytes = 2 descriptor units per step
                        const uint32_t first = (kb > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
                        for (int t = 0; t < 5; t++)
                            umma_tf32(dsm, ad[PA[t]] + 2 * kk, bd[PB[t]] + 2 * kk, idesc, (first || t > 0) ? 1u : 0u);
                        umma_tf32(d, ad[0] + 2 * kk, bd[0] + 2 * kk, idesc, first);
                    }
                    umma_commit(&op_empty[s]);
                }
                if (!ok) break;
                umma_commit(&acc_full[buf]);  // arrives when this tile's MMAs have completed
            }
            // every MMA issued has completed before TMEM is freed
            umma_commit(mma_done);
            if (!mbar_wait(mma_done, 0, nullptr)) *abort_flag = 1;
        }
    } else if (warp >= 4) {
        // epilogue: thread = one row of the tile
        const int q = warp - 4;
        const int r = q * 32 + lane;
        const float beta = (float)a.ctrl->beta, tau = (float)a.ctrl->tau, thS = (float)a.ctrl->theta_S;
        int i = 0, lt = 0;
        for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, lt++) {
            const int buf = lt & 1;
            const int rb = (t / tiles_n) * TBM, cb = (t % tiles_n) * TBN;
            const int row = rb + r;
            // the row's mask words for this tile, loaded before the wait so that
            // their latency overlaps it (one word per 32-column sub-tile)
            uint32_t words[TBN / HALF];
#pragma unroll
            for (int w = 0; w < TBN / HALF; w++) {
                const int c0 = cb + w * HALF;
                words[w] = (a.Q != nullptr && row < a.m && c0 < a.n) ? a.Q[(int64_t)row * a.ldq + (c0 >> 5)]
                                                                     : 0xffffffffu;
            }
            if (!mbar_wait(&acc_full[buf], (lt >> 1) & 1, abort_flag)) break;
            tc_fence_after();
            bool ok = true;
            for (int h = 0; h < TBN / HALF; h++, i++) {
                const int s = i % EPS;
                if (!mbar_wait(&ep_full[s], (i / EPS) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                float acc[HALF];
                {
                    float v[16], w[16];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 2 * TBN + h * HALF);
#pragma unroll
                    for (int half = 0; half < 2; half++) {
                        tmem_ld16(ta + 16 * half, v);
                        tmem_ld16(ta + TBN + 16 * half, w);
#pragma unroll
                        for (int j = 0; j < 16; j++) acc[16 * half + j] = nkb > 0 ? v[j] + w[j] : 0.f;
                    }
                }
                const uint8_t *tD = sEp + s * EP_BYTES;
                const uint8_t *tS = tD + EP_TILE;
                const uint8_t *tP = a.has_sp ? tD + 2 * EP_TILE : tS;
                const int c0 = cb + h * HALF;
                if (row < a.m) {
                    const uint32_t word = words[h];  // 32 columns, one word
#pragma unroll
                    for (int c4 = 0; c4 < HALF / 4; c4++) {
                        const int col = c0 + 4 * c4;
                        if (col >= a.n) break;
                        const float4 dv = *swz4(tD, r, c4), sk = *swz4(tS, r, c4), sp = *swz4(tP, r, c4);
                        const float d4[4] = {dv.x, dv.y, dv.z, dv.w};
                        const float k4[4] = {sk.x, sk.y, sk.z, sk.w};
                        const float p4[4] = {sp.x, sp.y, sp.z, sp.w};
                        float so[4], mo[4];
#pragma unroll
                        for (int j = 0; j < 4; j++) {
                            const bool obs = (word >> (4 * c4 + j)) & 1u;
                            const float sh = beta != 0.f ? k4[j] + beta * (k4[j] - p4[j]) : k4[j];
                            const float l = acc[4 * c4 + j];
                            const float g = obs ? ((l - d4[j]) + sh) : 0.f;
                            so[j] = shrink(sh - tau * g, thS);
                            mo[j] = l - tau * g;
                        }
                        if (col + 3 < a.n) {
                            *reinterpret_cast<float4 *>(a.Sout + (int64_t)row * a.ldso + col) =
                                make_float4(so[0], so[1], so[2], so[3]);
                            *reinterpret_cast<float4 *>(a.M + (int64_t)row * a.ldm + col) =
                                make_float4(mo[0], mo[1], mo[2], mo[3]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; j++)
                                if (col + j < a.n) {
                                    a.Sout[(int64_t)row * a.ldso + col + j] = so[j];
                                    a.M[(int64_t)row * a.ldm + col + j] = mo[j];
                                }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&ep_empty[s]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
            if (!ok) break;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(a.err, 1);
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// A^ = [(1 + beta) A_k, -beta A_{k-1}] and B^ = [B_k, B_{k-1}] split into
// three TF32 parts each (P[0] high, P[1] middle, P[2] low; zero padding of the
// live K to the next 16)
struct SplitOut {
    float *a[3], *b[3];
};

__global__ void tf32_split_kernel(int m, int n, const float *__restrict__ Ak, const float *__restrict__ Ap,
                                  int64_t lda, const float *__restrict__ Bk, const float *__restrict__ Bp,
                                  int64_t ldb, const int *rk_p, const int *rp_p, const Ctrl *ctrl, SplitOut o,
                                  int64_t ldk)
{
    const int rk = rk_p ? *rk_p : 0;
    const int rp = (rp_p && ctrl->beta != 0.0) ? *rp_p : 0;
    const int K = rk + rp, Kp = (K + TBK - 1) / TBK * TBK;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Kp) return;
    const float ck = (float)(1.0 + ctrl->beta), cp = (float)(-ctrl->beta);
    const int rows = max(m, n);
    for (int row = blockIdx.y; row < rows; row += gridDim.y) {  // rows beyond the 65535 grid rows loop
        if (row < m) {
            const float v =
                c < rk ? Ak[(int64_t)row * lda + c] * ck : (c < K ? Ap[(int64_t)row * lda + c - rk] * cp : 0.f);
            const float h = tf32_rn(v), r1 = v - h, md = tf32_rn(r1);
            o.a[0][(int64_t)row * ldk + c] = h;
            o.a[1][(int64_t)row * ldk + c] = md;
            o.a[2][(int64_t)row * ldk + c] = tf32_rn(r1 - md);
        }
        if (row < n) {
            const float v = c < rk ? Bk[(int64_t)row * ldb + c] : (c < K ? Bp[(int64_t)row * ldb + c - rk] : 0.f);
            const float h = tf32_rn(v), r1 = v - h, md = tf32_rn(r1);
            o.b[0][(int64_t)row * ldk + c] = h;
            o.b[1][(int64_t)row * ldk + c] = md;
            o.b[2][(int64_t)row * ldk + c] = tf32_rn(r1 - md);
        }
    }
}

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

// fp32 row-major (rows x cols, leading dimension ld) map with boxes of
// box_rows x box_cols (32 columns: 128-byte swizzle; 16 columns: 64-byte)
bool make_map_f32(CUtensorMap *map, const float *base, uint64_t cols, uint64_t rows, uint64_t ld, uint32_t box_rows,
                  uint32_t box_cols = 32)
{
    EncodeTiledFn fn = encode_fn();
    if (fn == nullptr) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 4) % 16 != 0) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * 4};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t es[2] = {1, 1};
    const CUtensorMapSwizzle sw = box_cols == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cudaGetLastError();
    }
    return n;
}

}  // namespace

// three parts, each rows x round16(2 kmax)
size_t pass_tc_split_elems(int rows, int kmax) { return 3 * (size_t)rows * (size_t)((2 * kmax + TBK - 1) / TBK * TBK); }

// The fused fine pass on the tensor cores; false (nothing launched) when an
// operand does not meet the TMA rules (16-byte aligned bases and strides) or
// the tensor maps cannot be made.  A3 (m rows) and B3 (n rows) are scratch of
// pass_tc_split_elems each: three parts of leading dimension ldk =
// round16(2 kmax).
bool launch_pass_tc(const PassArgs<float> &p, int kmax, float *A3, float *B3, int *err, cudaStream_t st)
{
    if (p.M == nullptr || p.Sout == nullptr || p.Ak == nullptr || p.Bk == nullptr) return false;
    if (p.ldfa != p.ldfap || p.ldfb != p.ldfbp) return false;
    const int64_t ldk = (2 * kmax + TBK - 1) / TBK * TBK;
    const bool has_sp = p.Sp != nullptr && p.Sp != p.Sk;
    TcMaps maps;
    SplitOut so;
    for (int q = 0; q < 3; q++) {
        so.a[q] = A3 + (size_t)q * p.m * ldk;
        so.b[q] = B3 + (size_t)q * p.n * ldk;
        if (!make_map_f32(&maps.a[q], so.a[q], (uint64_t)ldk, (uint64_t)p.m, (uint64_t)ldk, TBM, TBK)) return false;
        if (!make_map_f32(&maps.b[q], so.b[q], (uint64_t)ldk, (uint64_t)p.n, (uint64_t)ldk, TBN, TBK)) return false;
    }
    if (!make_map_f32(&maps.d, p.D, (uint64_t)p.n, (uint64_t)p.m, (uint64_t)p.ldd, TBM)) return false;
    if (!make_map_f32(&maps.sk, p.Sk, (uint64_t)p.n, (uint64_t)p.m, (uint64_t)p.lds, TBM)) return false;
    if (!make_map_f32(&maps.sp, has_sp ? p.Sp : p.Sk, (uint64_t)p.n, (uint64_t)p.m, (uint64_t)p.lds, TBM))
        return false;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(pass_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES) !=
            cudaSuccess)
            return false;
        attr = true;
    }
    // split factors (one launch; threads over the padded live K), then the
    // persistent pass
    {
        dim3 grid((unsigned)((ldk + 127) / 128), (unsigned)std::min(std::max(p.m, p.n), 65535));
        CPCP_COUNT_LAUNCH();
        tf32_split_kernel<<<grid, 128, 0, st>>>(p.m, p.n, p.Ak, p.Ap ? p.Ap : p.Ak, p.ldfa, p.Bk, p.Bp ? p.Bp : p.Bk,
                                                p.ldfb, p.rk, p.Ap ? p.rp : nullptr, p.ctrl, so, ldk);
    }
    TcArgs a;
    a.m = p.m;
    a.n = p.n;
    a.Q = p.Q;
    a.ldq = p.ldq;
    a.Sout = p.Sout;
    a.ldso = p.ldso;
    a.M = p.M;
    a.ldm = p.ldm;
    a.rk = p.rk;
    a.rp = p.Ap ? p.rp : nullptr;
    a.ctrl = p.ctrl;
    a.has_sp = has_sp ? 1 : 0;
    a.err = err;
    const int tiles = ((p.m + TBM - 1) / TBM) * ((p.n + TBN - 1) / TBN);
    const int grid = std::min(tiles, sm_count());
    CPCP_COUNT_LAUNCH();
    pass_tc_kernel<<<grid, NT, SMEM_BYTES, st>>>(maps, a);
    return true;
}

}  // namespace cpcp
