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
// epilogue adds the two in fp32.
//
// The split happens in shared memory: TMA brings a 16-wide K slice of the
// fp32 factors (A_k or A_{k-1}, and B_k or B_{k-1}: the K blocks of A^ walk
// the columns of A_k first, then those of A_{k-1}) into a raw stage;
// converter warps scale it by (1 + beta) or -beta, zero the columns beyond
// the live rank, and write the three parts into an operand stage (the same
// swizzled offset in each part's slot), then hand that stage to the MMA
// issuer, which pairs the parts: six MMAs per K step of 8.  Raw and operand
// stages are separate rings, so TMA runs ahead of the converters and they
// run ahead of the tensor cores.  The operands cross L2 once, as fp32, and
// no split copy of the factors exists.
//
// Measured alternatives, each worse on the 2000 x 2000 rank-50 workload:
// splitting the factors into three TF32 copies in global memory by a
// separate launch (6.3 us, and three times the operand bytes through L2);
// converting in place in the operand stage (TMA, conversion and MMA then
// share two buffers and their latencies add) with two epilogue groups on
// alternate quarters (while both compute, no epilogue input is in flight):
// 37.5 us against 30.2 us + 6.3 us; the same with separate raw and operand
// rings and one epilogue group storing each row's float4 directly (32 lines
// per warp-wide store): 36.3 us; with TMA stores but two raw stages and two
// 32-column epilogue stages: 33.2 us, where a %globaltimer trace showed each
// 16-wide K stage taking about 1 us (a raw TMA from L2 takes about 1.1 us,
// its conversion about 0.5 us, and two raw stages let only one be in flight
// while the other converts) against 0.4 us of tensor-core work; a third raw
// stage changed nothing: four converter warps rounding with cvt.rna.tf32 took
// 1 us per stage (three conversions per element on a reduced-rate pipe);
// two-term splitting (a_h b_h + a_h b_l + a_l b_h) represents a factor only
// to 2^-22, and one accumulator shared by all six products loses the small
// terms' low bits to the large running sum; both left a rel-KKT floor near
// 1.7e-6, because the momentum step cancels most of L-hat.  Laying the six
// products out as one contraction over an extended K = 6 K re-read the
// operands six times from L2.
//
// One persistent CTA per SM walks 128 x 128 output tiles.  Warp roles:
//   warp 0   TMA producer of the raw stages (fp32 slices of A and B)
//   warp 1   MMA issuer: tcgen05.mma kind::tf32, M = 128, N = 128, K = 8
//   warp 2   TMEM allocator (per buffer a 128-column accumulator for a_h b_h and
//            one for the small products; two buffers: all 512 columns), then
//            TMA store issuer of the results
//   warp 3   TMA producer of the epilogue tiles: D, S_k, S_{k-1} in 16-column
//            slices (64-byte swizzle), three stages
//   warps 4-11 epilogue, two groups of four on the two 8-column halves of
//            each 16-column slice: tcgen05.ld of the accumulator (one TMEM
//            lane quarter per warp, one row per thread), the elementwise step;
//            S_{k+1} and M are written over the D and S_k slots of the stage
//            they came from (each thread rewrites what it read) and leave by
//            TMA store, so the row-per-thread layout never meets the LSU
//   warps 12-19 converters: the TF32 split of each raw stage.
// So the HBM stream of the epilogue inputs runs while the tensor cores work
// on the next tile, and the operands (L2-resident factors) never touch the
// SIMT pipes.
//
// Every mbarrier wait is bounded (about one second of %globaltimer) and also
// ends when another role has given up (a shared abort flag); the kernel then
// raises the error flag that the host turns into CPCP_ERR_TIMEOUT, drains the
// copies it issued and frees its TMEM.
#include <cuda.h>

#include <algorithm>

#include <mutex>

#include "common.cuh"

namespace cpcp {

namespace {

constexpr int TBM = 128;   // tile rows = TMEM lanes
constexpr int TBN = 128;   // tile columns = accumulator columns
constexpr int TBK = 16;    // K per operand stage: 64 bytes of fp32
constexpr int HALF = 16;   // epilogue sub-tile columns (64 bytes of fp32)
constexpr int OPS = 2;     // operand stages
constexpr int EPS = 3;     // epilogue sub-tile buffers
constexpr int NT = 640;
constexpr int EPI_W0 = 4;   // first epilogue warp (two groups of four)
constexpr int CVT_W0 = 12;  // first converter warp
constexpr int CVT_NW = 8;   // converter warps
constexpr uint32_t A_BYTES = TBM * TBK * 4;             // 8 KB per part
constexpr uint32_t B_BYTES = TBN * TBK * 4;             // 8 KB per part
constexpr uint32_t OP_BYTES = 3 * A_BYTES + 3 * B_BYTES;  // three parts of each
constexpr uint32_t OP_TX = A_BYTES + B_BYTES;             // bytes TMA brings per stage (fp32 slices)
static_assert(A_BYTES == B_BYTES, "the converters address the parts of A and B with one stride");
constexpr uint32_t EP_TILE = TBM * HALF * 4;            // 8 KB per array
constexpr uint32_t EP_BYTES = 3 * EP_TILE;              // D, S_k, S_{k-1}
constexpr uint32_t TMEM_COLS = 4 * TBN;  // two buffers x (large, small)
constexpr int RS = 3;       // raw stages (fp32 slices as TMA brings them)
constexpr size_t SMEM_BYTES = 1024 + OPS * (size_t)OP_BYTES + EPS * (size_t)EP_BYTES + RS * (size_t)OP_TX + 256;
static_assert(SMEM_BYTES <= 232448, "shared memory per block");

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

// tile store from shared memory (bulk group of the issuing thread); the box
// is clipped at the tensor's bounds
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(smem_u32(src)), "r"(x), "r"(y)
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

// 8 columns of two accumulators (at taddr and taddr + off) for this thread's
// row, with one wait for both loads; the wait is in the same asm statement so
// that no use of the registers can be scheduled before it
__device__ __forceinline__ void tmem_ld8x2(uint32_t taddr, uint32_t off, float (&v)[8], float (&w)[8])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr), "r"(taddr + off)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) {
        v[i] = __uint_as_float(r[i]);
        w[i] = __uint_as_float(r[8 + i]);
    }
}

// nearest TF32 value of a finite x (11 significant bits), ties away from zero:
// half an ulp of the 11-bit significand added to the magnitude bits, then the
// 13 low bits cleared (a carry into the exponent is the correct rounding).
// Integer ALU work at full rate.
__device__ __forceinline__ float tf32_round(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// live ranks of the contraction (the same on every role): K blocks [0, nk1)
// walk the columns of A_k / B_k, blocks [nk1, nk1 + nk2) those of A_{k-1} /
// B_{k-1}
struct LiveK {
    int rk, rp, nk1, nkb;
};
__device__ __forceinline__ LiveK live_k(const int *rk, const int *rp, const Ctrl *ctrl)
{
    LiveK l;
    l.rk = rk ? *rk : 0;
    l.rp = (rp && ctrl->beta != 0.0) ? *rp : 0;
    l.nk1 = (l.rk + TBK - 1) / TBK;
    l.nkb = l.nk1 + (l.rp + TBK - 1) / TBK;
    return l;
}

struct TcMaps {
    CUtensorMap a[2], b[2];  // fp32 factors: current, previous (K-major, 16-column boxes, 64-byte swizzle)
    CUtensorMap d, sk, sp;   // epilogue inputs (16-column boxes, 64-byte swizzle)
    CUtensorMap so, mo;      // results S_{k+1} and M (same boxes)
};

struct TcArgs {
    int m, n;
    const uint32_t *Q;
    int64_t ldq;
    const int *rk, *rp;
    const Ctrl *ctrl;
    int has_sp;
    int *err;
};

// 16-byte chunk c4 (0..3) of row r of a 128-row x 16-column fp32 TMA box with
// 64-byte swizzle: chunk bits [4, 6) of the offset XOR bits [7, 9)
__device__ __forceinline__ float4 *swz4(uint8_t *tile, int r, int c4)
{
    return reinterpret_cast<float4 *>(tile + r * 64 + ((c4 ^ ((r >> 1) & 3)) << 4));
}

__global__ void __launch_bounds__(NT, 1) pass_tc_kernel(const __grid_constant__ TcMaps maps, TcArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sOp = smem;                        // OPS x [A h | A m | A l | B h | B m | B l]
    uint8_t *sEp = smem + OPS * OP_BYTES;       // EPS x [D | S_k | S_{k-1}]
    uint8_t *sRaw = sEp + EPS * EP_BYTES;       // RS x [A | B] (fp32)
    uint64_t *bars = reinterpret_cast<uint64_t *>(sRaw + RS * OP_TX);
    uint64_t *raw_full = bars, *raw_empty = bars + RS;
    uint64_t *op_empty = bars + 2 * RS, *cvt_full = op_empty + OPS;
    uint64_t *ep_full = cvt_full + OPS, *ep_empty = ep_full + EPS;
    uint64_t *st_full = ep_empty + EPS;  // results of a stage written, ready to store
    uint64_t *acc_full = st_full + EPS, *acc_empty = acc_full + 2;
    uint64_t *mma_done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_n = (a.n + TBN - 1) / TBN;
    const int ntiles = ((a.m + TBM - 1) / TBM) * tiles_n;
    const LiveK lk = live_k(a.rk, a.rp, a.ctrl);
    const int nkb = lk.nkb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RS; s++) {
            mbar_init(&raw_full[s], 1);
            mbar_init(&raw_empty[s], CVT_NW);  // one arrival per converter warp
        }
        for (int s = 0; s < OPS; s++) {
            mbar_init(&op_empty[s], 1);
            mbar_init(&cvt_full[s], CVT_NW);
        }
        for (int s = 0; s < EPS; s++) {
            mbar_init(&ep_full[s], 1);
            mbar_init(&ep_empty[s], 1);  // the store issuer, once the stores have read the stage
            mbar_init(&st_full[s], 8);   // one arrival per epilogue warp
        }
        for (int s = 0; s < 2; s++) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 8);  // one arrival per epilogue warp
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
                    const int s = i % RS;
                    if (i >= RS && !mbar_wait(&raw_empty[s], ((i / RS) & 1) ^ 1, abort_flag)) break;
                    uint8_t *st = sRaw + s * OP_TX;
                    const int src = kb < lk.nk1 ? 0 : 1;
                    const int x = (kb < lk.nk1 ? kb : kb - lk.nk1) * TBK;
                    mbar_expect_tx(&raw_full[s], OP_TX);
                    tma_load_2d(st, &maps.a[src], &raw_full[s], x, rb);
                    tma_load_2d(st + A_BYTES, &maps.b[src], &raw_full[s], x, cb);
                }
            }
            // drain: the last phase issued on each stage has landed (time bound
            // only: no copy may still be in flight when the CTA exits)
            for (int s = 0; s < RS && s < i; s++) {
                const int last = i - 1 - ((i - 1 - s) % RS);
                if (!mbar_wait(&raw_full[s], (last / RS) & 1, nullptr)) *abort_flag = 1;
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
                    if (!mbar_wait(&cvt_full[s], (i / OPS) & 1, abort_flag)) {
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
    } else if (warp == 2) {
        // store issuer: S_{k+1} (D slot) and M (S_k slot) of each finished
        // slice; the stage goes back to the producer once the stores have
        // read it
        if (lane == 0) {
            int i = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
                const int rb = (t / tiles_n) * TBM, cb = (t % tiles_n) * TBN;
                bool ok = true;
                for (int h = 0; h < TBN / HALF; h++, i++) {
                    const int s = i % EPS;
                    if (!mbar_wait(&st_full[s], (i / EPS) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint8_t *tD = sEp + s * EP_BYTES;
                    tma_store_2d(&maps.so, tD, cb + h * HALF, rb);
                    tma_store_2d(&maps.mo, tD + EP_TILE, cb + h * HALF, rb);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    mbar_arrive(&ep_empty[s]);
                }
                if (!ok) break;
            }
            // every store has completed before the CTA exits
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        }
    } else if (warp >= EPI_W0 && warp < CVT_W0) {
        // epilogue: thread = one row of the tile; group g takes columns
        // [8 g, 8 g + 8) of every 16-column slice
        const int grp = (warp - EPI_W0) >> 2, q = (warp - EPI_W0) & 3;
        const int r = q * 32 + lane;
        const float beta = (float)a.ctrl->beta, tau = (float)a.ctrl->tau, thS = (float)a.ctrl->theta_S;
        int i = 0, lt = 0;
        for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, lt++) {
            const int buf = lt & 1;
            const int rb = (t / tiles_n) * TBM, cb = (t % tiles_n) * TBN;
            const int row = rb + r;
            // the row's mask words for this tile, loaded before the wait so that
            // their latency overlaps it (one word per 32 columns)
            uint32_t words[TBN / 32];
#pragma unroll
            for (int w = 0; w < TBN / 32; w++) {
                const int c0 = cb + w * 32;
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
                float acc[HALF / 2];
                {
                    float v[HALF / 2], w[HALF / 2];
                    const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) +
                                        (uint32_t)(buf * 2 * TBN + h * HALF + grp * (HALF / 2));
                    tmem_ld8x2(ta, (uint32_t)TBN, v, w);
#pragma unroll
                    for (int j = 0; j < HALF / 2; j++) acc[j] = nkb > 0 ? v[j] + w[j] : 0.f;
                }
                uint8_t *tD = sEp + s * EP_BYTES;
                uint8_t *tS = tD + EP_TILE;
                uint8_t *tP = a.has_sp ? tD + 2 * EP_TILE : tS;
                const int c0 = cb + h * HALF + grp * (HALF / 2);
                if (row < a.m) {
                    const uint32_t word = words[(h * HALF) / 32] >> ((h * HALF) % 32 + grp * (HALF / 2));
#pragma unroll
                    for (int c4 = 0; c4 < HALF / 8; c4++) {
                        const int col = c0 + 4 * c4;
                        if (col >= a.n) break;  // clipped by the store
                        const int cc = grp * (HALF / 8) + c4;  // 16-byte chunk within the 16-column row
                        float4 *pd = swz4(tD, r, cc);
                        float4 *ps = swz4(tS, r, cc);
                        const float4 dv = *pd, sk = *ps, sp = *swz4(tP, r, cc);
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
                        *pd = make_float4(so[0], so[1], so[2], so[3]);  // S_{k+1} over D
                        *ps = make_float4(mo[0], mo[1], mo[2], mo[3]);  // M over S_k
                    }
                }
                // the results are read by the TMA stores (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&st_full[s]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
            if (!ok) break;
        }
    } else if (warp >= CVT_W0) {
        // converters: the TF32 split of each raw stage into an operand stage.
        // A raw stage holds 512 float4 of A, then 512 of B; float4 g sits in
        // tile row g / 4 at the 16-byte chunk (g % 4) ^ ((row / 2) % 4) of the
        // 64-byte swizzle, i.e. K columns 4 ((g % 4) ^ ((row / 2) % 4)) ...;
        // the parts go to the same offset of their slots
        const int ct = threadIdx.x - CVT_W0 * 32;
        const float ck = (float)(1.0 + a.ctrl->beta), cp = (float)(-a.ctrl->beta);
        int i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok && !*abort_flag; t += gridDim.x) {
            for (int kb = 0; kb < nkb; kb++, i++) {
                const int s = i % OPS, sr = i % RS;
                if (!mbar_wait(&raw_full[sr], (i / RS) & 1, abort_flag) ||
                    (i >= OPS && !mbar_wait(&op_empty[s], ((i / OPS) & 1) ^ 1, abort_flag))) {
                    ok = false;
                    break;
                }
                const uint8_t *rw = sRaw + sr * OP_TX;
                uint8_t *st = sOp + s * OP_BYTES;
                const bool cur = kb < lk.nk1;
                const int k0 = (cur ? kb : kb - lk.nk1) * TBK;
                const int lim = cur ? lk.rk : lk.rp;
                const float ca = cur ? ck : cp;
#pragma unroll
                for (int u = 0; u < (2 * 512) / (CVT_NW * 32); u++) {
                    const int f = ct + u * CVT_NW * 32;
                    const int opnd = f >> 9, g = f & 511;
                    uint8_t *p0 = st + (opnd ? 3 * A_BYTES : 0) + g * 16;
                    const uint8_t *src = rw + (opnd ? A_BYTES : 0) + g * 16;
                    const int tr = g >> 2;
                    const int kc = k0 + 4 * ((g & 3) ^ ((tr >> 1) & 3));
                    const float coef = opnd ? 1.f : ca;
                    const float4 x = *reinterpret_cast<const float4 *>(src);
                    const float xv[4] = {x.x, x.y, x.z, x.w};
                    float hv[4], mv[4], lv[4];
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const float v = kc + j < lim ? xv[j] * coef : 0.f;
                        const float hi = tf32_round(v), r1 = v - hi, md = tf32_round(r1);
                        hv[j] = hi;
                        mv[j] = md;
                        lv[j] = tf32_round(r1 - md);
                    }
                    *reinterpret_cast<float4 *>(p0) = make_float4(hv[0], hv[1], hv[2], hv[3]);
                    *reinterpret_cast<float4 *>(p0 + A_BYTES) = make_float4(mv[0], mv[1], mv[2], mv[3]);
                    *reinterpret_cast<float4 *>(p0 + 2 * A_BYTES) = make_float4(lv[0], lv[1], lv[2], lv[3]);
                }
                // the parts are read by the tensor cores (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&cvt_full[s]);
                    mbar_arrive(&raw_empty[sr]);
                }
            }
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

// ---------------------------------------------------------------------------
// The products of the subspace iteration with the (restricted) iterate M,
//     Y = M Omega   (rows P = m, K = n: A = M, K-major)
//     Z = M^T Q     (rows P = n, K = m: A = M^T, read from M as stored)
// on the tensor cores, with the three-part TF32 split of the fused pass (six
// MMAs per K step of 8, the five small products and a_h b_h in separate fp32
// accumulators).  One CTA per (128-row output tile, K range): the long K of
// these tall-skinny products is split over CTAs so that about one CTA runs per
// SM, each writing a partial tile that a fixed-order reduction sums.  TMA
// brings 16-wide K slices of M and of the thin operand (Omega or Q, n x KM or
// m x KM) as fp32; the converter warps split them and, for the operands not
// already K-major (M^T, and the thin operand, whose K runs down its rows),
// transpose them into the K-major operand layout on the way.  The live width
// k (device value) sets the MMA's N = round16(k) <= 128; the converters zero
// the thin operand's columns beyond k.
//
// The tensor cores add into an fp32 accumulator by aligning to the largest
// term and dropping the bits below it, a one-sided error that grows with the
// number of MMAs chained into one accumulator.  So an accumulator lives for
// PP_DR stages only: the MMA warp alternates between two TMEM buffers, and the
// epilogue warps drain each finished buffer into a round-to-nearest fp32 sum
// in shared memory while the next one fills.
//
// Warp roles (512 threads): warp 0 TMA producer, warp 1 MMA issuer, warp 2
// TMEM allocator, warps 4-7 epilogue (one TMEM lane quarter each, one output
// row per thread while draining, one row per warp-wide store at the end),
// warps 8-15 converters.  Every mbarrier wait is bounded as in the fused pass;
// a timeout raises the error flag.
constexpr int PP_M = 128;    // output rows per tile
constexpr int PP_NB = 128;   // thin-operand columns a stage holds (the MMA's N is round16(k))
constexpr int PP_K = 16;     // K per stage
constexpr int PP_RS = 4;     // raw stages
constexpr int PP_OPS = 2;    // operand stages
constexpr int PP_DR = 2;     // stages per accumulator lifetime
constexpr int PP_NT = 512;
constexpr int PP_EPI_W0 = 4;
constexpr int PP_CVT_W0 = 8;
constexpr int PP_CVT_NW = 8;
constexpr uint32_t PP_A = PP_M * PP_K * 4;    // 8 KB: one part of A, or the raw A slice
constexpr uint32_t PP_B = PP_NB * PP_K * 4;   // 8 KB: one part of B, or the raw B slice
constexpr uint32_t PP_RAW = PP_A + PP_B;
constexpr uint32_t PP_OP = 3 * PP_A + 3 * PP_B;
constexpr int PP_ACC_LD = PP_M + 1;           // running sums, column-major, padded against bank conflicts
constexpr uint32_t PP_ACC = PP_NB * PP_ACC_LD * 4;
constexpr uint32_t PP_TMEM = 4 * PP_NB;       // two buffers x (a_h b_h, the small products)
constexpr size_t PP_SMEM = 1024 + PP_OPS * (size_t)PP_OP + PP_RS * (size_t)PP_RAW + PP_ACC + 256;
static_assert(PP_SMEM <= 232448, "shared memory per block");

struct ProdMaps {
    CUtensorMap a;  // M: [P rows][16-col boxes], 64-byte swizzle (Y); [16 rows][128-col boxes], no swizzle (Z)
    CUtensorMap b;  // thin operand: [16 rows][128-col boxes], no swizzle
};

struct ProdArgs {
    int P, K, ldc, stages_per_split, total_stages;
    int bcols;         // columns of the thin operand's TMA box: min(its leading dimension, 128)
    int tn;            // 1: A = M^T
    const int *kdyn;   // live width k
    float *part;       // partial tiles: split s at part + s * slice, row-major with ld ldc
    int64_t slice;
    int *err;
};

__device__ __forceinline__ void split3(float v, float &h, float &m, float &l)
{
    h = tf32_round(v);
    const float r1 = v - h;
    m = tf32_round(r1);
    l = tf32_round(r1 - m);
}

__global__ void __launch_bounds__(PP_NT, 1) prod_tc_kernel(const __grid_constant__ ProdMaps maps, ProdArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sOp = smem;                          // PP_OPS x [A h | A m | A l | B h | B m | B l]
    uint8_t *sRaw = sOp + PP_OPS * PP_OP;         // PP_RS x [A | B] (fp32 as TMA brings them)
    float *sAcc = reinterpret_cast<float *>(sRaw + PP_RS * PP_RAW);  // [column][PP_ACC_LD]
    uint64_t *bars = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(sAcc) + PP_ACC);
    uint64_t *raw_full = bars, *raw_empty = bars + PP_RS;
    uint64_t *op_empty = bars + 2 * PP_RS, *cvt_full = op_empty + PP_OPS;
    uint64_t *acc_full = cvt_full + PP_OPS, *acc_empty = acc_full + 2, *mma_done = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p0 = blockIdx.x * PP_M;
    const int s0 = blockIdx.y * a.stages_per_split;
    const int s1 = min(a.total_stages, s0 + a.stages_per_split);
    const int nst = max(0, s1 - s0);
    const int k = min(*a.kdyn, PP_NB);
    const int nmma = max(16, (k + 15) / 16 * 16);  // the MMA's N
    const int nch = (nst + PP_DR - 1) / PP_DR;      // accumulator lifetimes

    if (threadIdx.x == 0) {
        for (int s = 0; s < PP_RS; s++) {
            mbar_init(&raw_full[s], 1);
            mbar_init(&raw_empty[s], PP_CVT_NW);
        }
        for (int s = 0; s < PP_OPS; s++) {
            mbar_init(&op_empty[s], 1);
            mbar_init(&cvt_full[s], PP_CVT_NW);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(PP_TMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int i = 0;
            for (; i < nst && !*abort_flag; i++) {
                const int s = i % PP_RS;
                if (i >= PP_RS && !mbar_wait(&raw_empty[s], ((i / PP_RS) & 1) ^ 1, abort_flag)) break;
                uint8_t *st = sRaw + s * PP_RAW;
                const int kk = (s0 + i) * PP_K;
                mbar_expect_tx(&raw_full[s], PP_A + (uint32_t)(PP_K * a.bcols * 4));
                if (a.tn)
                    tma_load_2d(st, &maps.a, &raw_full[s], p0, kk);  // M rows kk.., columns p0..
                else
                    tma_load_2d(st, &maps.a, &raw_full[s], kk, p0);  // M rows p0.., columns kk..
                tma_load_2d(st + PP_A, &maps.b, &raw_full[s], 0, kk);
            }
            for (int s = 0; s < PP_RS && s < i; s++) {
                const int last = i - 1 - ((i - 1 - s) % PP_RS);
                if (!mbar_wait(&raw_full[s], (last / PP_RS) & 1, nullptr)) *abort_flag = 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // kind::tf32, fp32 accumulator, M = 128, N = round16(k)
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(nmma >> 3) << 17) |
                                   ((uint32_t)(PP_M >> 4) << 24);
            for (int i = 0; i < nst; i++) {
                const int s = i % PP_OPS, c = i / PP_DR, b = c & 1;
                const bool cfirst = (i % PP_DR) == 0;
                // buffer b was last filled by lifetime c - 2: wait for its drain
                if (cfirst && c >= 2 && !mbar_wait(&acc_empty[b], ((c >> 1) & 1) ^ 1, abort_flag)) break;
                if (!mbar_wait(&cvt_full[s], (i / PP_OPS) & 1, abort_flag)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * 2 * PP_NB), dsm = d + (uint32_t)PP_NB;
                const uint8_t *st = sOp + s * PP_OP;
                uint64_t ad[3], bd[3];
#pragma unroll
                for (int q = 0; q < 3; q++) {
                    ad[q] = smem_desc_sw64(st + q * PP_A);
                    bd[q] = smem_desc_sw64(st + 3 * PP_A + q * PP_B);
                }
                constexpr int PA[5] = {1, 2, 0, 1, 0}, PB[5] = {1, 0, 2, 0, 1};
#pragma unroll
                for (int kk = 0; kk < PP_K / 8; kk++) {
                    const uint32_t acc = (!cfirst || kk > 0) ? 1u : 0u;
#pragma unroll
                    for (int t = 0; t < 5; t++)
                        umma_tf32(dsm, ad[PA[t]] + 2 * kk, bd[PB[t]] + 2 * kk, idesc, (acc || t > 0) ? 1u : 0u);
                    umma_tf32(d, ad[0] + 2 * kk, bd[0] + 2 * kk, idesc, acc);
                }
                umma_commit(&op_empty[s]);
                if (i % PP_DR == PP_DR - 1 || i == nst - 1) umma_commit(&acc_full[b]);
            }
            umma_commit(mma_done);
            if (!mbar_wait(mma_done, 0, nullptr)) *abort_flag = 1;
        }
    } else if (warp >= PP_EPI_W0 && warp < PP_EPI_W0 + 4) {
        // drain each accumulator lifetime into the running sums (one row per
        // thread: the row's columns of both accumulators, summed in fp32)
        const int q = warp - PP_EPI_W0;
        const int rl = q * 32 + lane;
        bool ok = true;
        for (int c = 0; c < nch; c++) {
            const int b = c & 1;
            if (!mbar_wait(&acc_full[b], (c >> 1) & 1, abort_flag)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 2 * PP_NB);
            for (int c0 = 0; c0 < nmma; c0 += 8) {
                float v[8], w[8];
                tmem_ld8x2(ta + (uint32_t)c0, (uint32_t)PP_NB, v, w);
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    float *p = sAcc + (c0 + j) * PP_ACC_LD + rl;
                    const float t = v[j] + w[j];
                    *p = c == 0 ? t : *p + t;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
        // the warp's 32 rows, one row per store instruction
        __syncwarp();
        const bool have = ok && nch > 0;
        for (int r = q * 32; r < q * 32 + 32; r++) {
            const int row = p0 + r;
            if (row >= a.P) break;
            float *out = a.part + (int64_t)blockIdx.y * a.slice + (int64_t)row * a.ldc;
            for (int cc = lane; cc < k; cc += 32) out[cc] = have ? sAcc[cc * PP_ACC_LD + r] : 0.f;
        }
    } else if (warp >= PP_CVT_W0) {
        // the TF32 split of each raw stage into an operand stage.  Operand
        // tiles are K-major with the 64-byte swizzle: the 16-byte chunk at
        // physical position c4 of row r holds K columns 4 (c4 ^ ((r / 2) % 4)) ..
        const int ct = threadIdx.x - PP_CVT_W0 * 32;
        for (int i = 0; i < nst && !*abort_flag; i++) {
            const int s = i % PP_OPS, sr = i % PP_RS;
            if (!mbar_wait(&raw_full[sr], (i / PP_RS) & 1, abort_flag) ||
                (i >= PP_OPS && !mbar_wait(&op_empty[s], ((i / PP_OPS) & 1) ^ 1, abort_flag)))
                break;
            const uint8_t *rw = sRaw + sr * PP_RAW;
            const float *rB = reinterpret_cast<const float *>(rw + PP_A);
            uint8_t *st = sOp + s * PP_OP;
            // A: 128 rows x 4 chunks
            for (int g = ct; g < PP_M * 4; g += PP_CVT_NW * 32) {
                float xv[4];
                uint8_t *dst;
                if (!a.tn) {
                    // M rows as TMA brought them (same swizzle as the operand)
                    const float4 x = *reinterpret_cast<const float4 *>(rw + g * 16);
                    xv[0] = x.x;
                    xv[1] = x.y;
                    xv[2] = x.z;
                    xv[3] = x.w;
                    dst = st + g * 16;
                } else {
                    // M^T: output row r gathers column r of the raw [16 K][128] slice
                    const int r = g & (PP_M - 1), c4 = g >> 7;
                    const int kc = 4 * (c4 ^ ((r >> 1) & 3));
                    const float *rA = reinterpret_cast<const float *>(rw);
#pragma unroll
                    for (int j = 0; j < 4; j++) xv[j] = rA[(kc + j) * PP_M + r];
                    dst = st + r * 64 + c4 * 16;
                }
                float hv[4], mv[4], lv[4];
#pragma unroll
                for (int j = 0; j < 4; j++) split3(xv[j], hv[j], mv[j], lv[j]);
                *reinterpret_cast<float4 *>(dst) = make_float4(hv[0], hv[1], hv[2], hv[3]);
                *reinterpret_cast<float4 *>(dst + PP_A) = make_float4(mv[0], mv[1], mv[2], mv[3]);
                *reinterpret_cast<float4 *>(dst + 2 * PP_A) = make_float4(lv[0], lv[1], lv[2], lv[3]);
            }
            // B: row c of the operand gathers column c of the raw [16 K][128]
            // slice of the thin operand (zero beyond the live width; k <= bcols)
            for (int g = ct; g < nmma * 4; g += PP_CVT_NW * 32) {
                const int r = g % nmma, c4 = g / nmma;
                const int kc = 4 * (c4 ^ ((r >> 1) & 3));
                float xv[4];
#pragma unroll
                for (int j = 0; j < 4; j++) xv[j] = r < k ? rB[(kc + j) * a.bcols + r] : 0.f;
                float hv[4], mv[4], lv[4];
#pragma unroll
                for (int j = 0; j < 4; j++) split3(xv[j], hv[j], mv[j], lv[j]);
                uint8_t *dst = st + 3 * PP_A + r * 64 + c4 * 16;
                *reinterpret_cast<float4 *>(dst) = make_float4(hv[0], hv[1], hv[2], hv[3]);
                *reinterpret_cast<float4 *>(dst + PP_B) = make_float4(mv[0], mv[1], mv[2], mv[3]);
                *reinterpret_cast<float4 *>(dst + 2 * PP_B) = make_float4(lv[0], lv[1], lv[2], lv[3]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&cvt_full[s]);
                mbar_arrive(&raw_empty[sr]);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(a.err, 1);
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PP_TMEM) : "memory");
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

// fp32 row-major map with boxes of box_rows x box_cols and no swizzle (rows of
// box_cols * 4 bytes, a multiple of 16; at most 256 columns)
bool make_map_f32_plain(CUtensorMap *map, const float *base, uint64_t cols, uint64_t rows, uint64_t ld,
                        uint32_t box_rows, uint32_t box_cols)
{
    EncodeTiledFn fn = encode_fn();
    if (fn == nullptr) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * 4) % 16 != 0) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * 4};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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

// The fused fine pass on the tensor cores; false (nothing launched) when an
// operand does not meet the TMA rules (16-byte aligned bases and strides) or
// the tensor maps cannot be made.
bool launch_pass_tc(const PassArgs<float> &p, int *err, cudaStream_t st)
{
    if (p.M == nullptr || p.Sout == nullptr || p.Ak == nullptr || p.Bk == nullptr) return false;
    if (p.ldfa != p.ldfap || p.ldfb != p.ldfbp) return false;
    const bool has_sp = p.Sp != nullptr && p.Sp != p.Sk;
    TcMaps maps;
    const float *Ap = p.Ap ? p.Ap : p.Ak, *Bp = p.Bp ? p.Bp : p.Bk;
    if (!make_map_f32(&maps.a[0], p.Ak, (uint64_t)p.ldfa, (uint64_t)p.m, (uint64_t)p.ldfa, TBM, TBK)) return false;
    if (!make_map_f32(&maps.a[1], Ap, (uint64_t)p.ldfa, (uint64_t)p.m, (uint64_t)p.ldfa, TBM, TBK)) return false;
    if (!make_map_f32(&maps.b[0], p.Bk, (uint64_t)p.ldfb, (uint64_t)p.n, (uint64_t)p.ldfb, TBN, TBK)) return false;
    if (!make_map_f32(&maps.b[1], Bp, (uint64_t)p.ldfb, (uint64_t)p.n, (uint64_t)p.ldfb, TBN, TBK)) return false;
    if (!make_map_f32(&maps.d, p.D, (uint64_t)p.n, (uint64_t)p.m, (uint64_t)p.ldd, TBM, HALF)) return false;
    if (!make_map_f32(&maps.sk, p.Sk, (uint64_t)p.n, (uint64_t)p.m, (uint64_t)p.lds, TBM, HALF)) return false;
    if (!make_map_f32(&maps.sp, has_sp ? p.Sp : p.Sk, (uint64_t)p.n, (uint64_t)p.m, (uint64_t)p.lds, TBM, HALF))
        return false;
    if (!make_map_f32(&maps.so, p.Sout, (uint64_t)p.n, (uint64_t)p.m, (uint64_t)p.ldso, TBM, HALF)) return false;
    if (!make_map_f32(&maps.mo, p.M, (uint64_t)p.n, (uint64_t)p.m, (uint64_t)p.ldm, TBM, HALF)) return false;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(pass_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES) !=
            cudaSuccess)
            return false;
        attr = true;
    }
    TcArgs a;
    a.m = p.m;
    a.n = p.n;
    a.Q = p.Q;
    a.ldq = p.ldq;
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

// C (P x k) = A B for the products of the subspace iteration on the tensor
// cores (see prod_tc_kernel): tn = 0: A = M (P x K), tn = 1: A = M^T with M
// (K x P); M with leading dimension ldm; B (K x k, leading dimension ldb <= 128
// columns used) the thin operand.  Writes `splits` partial slices of part
// (slice floats apart, leading dimension ldc) and returns their number, or 0
// (nothing launched) when an operand does not meet the TMA rules.
int gpu_sm_count() { return sm_count(); }

int prod_tc_ctas(int P, int K, int max_splits, int max_ctas)
{
    // about one CTA per SM (or max_ctas), at least 4 stages per CTA
    const int tiles = (P + PP_M - 1) / PP_M;
    const int total = (K + PP_K - 1) / PP_K;
    const int budget = max_ctas > 0 ? std::min(max_ctas, sm_count()) : sm_count();
    int splits = std::max(1, std::min({budget / tiles, max_splits, std::max(1, total / 4)}));
    const int per = (total + splits - 1) / splits;
    splits = (total + per - 1) / per;
    return tiles * splits;
}

int launch_prod_tc(int tn, int P, int K, const float *M, int64_t ldm, const float *B, int64_t ldb, int bcols_max,
                   const int *kdyn, float *part, int64_t ldc, int64_t slice, int max_splits, int *err, cudaStream_t st,
                   int max_ctas)
{
    if (P < 1 || K < 1 || bcols_max < 1 || bcols_max > PP_NB) return 0;
    ProdMaps maps;
    const int bcols = (int)std::min<int64_t>(ldb, PP_NB);
    if (tn) {
        if (!make_map_f32_plain(&maps.a, M, (uint64_t)P, (uint64_t)K, (uint64_t)ldm, PP_K, PP_M)) return 0;
    } else {
        if (!make_map_f32(&maps.a, M, (uint64_t)K, (uint64_t)P, (uint64_t)ldm, PP_M, PP_K)) return 0;
    }
    if (!make_map_f32_plain(&maps.b, B, (uint64_t)bcols, (uint64_t)K, (uint64_t)ldb, PP_K, (uint32_t)bcols)) return 0;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(prod_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PP_SMEM) !=
            cudaSuccess)
            return 0;
        attr = true;
    }
    const int tiles = (P + PP_M - 1) / PP_M;
    const int total = (K + PP_K - 1) / PP_K;
    const int splits = prod_tc_ctas(P, K, max_splits, max_ctas) / tiles;
    const int per = (total + splits - 1) / splits;
    ProdArgs a;
    a.P = P;
    a.K = K;
    a.ldc = (int)ldc;
    a.stages_per_split = per;
    a.total_stages = total;
    a.bcols = bcols;
    a.tn = tn;
    a.kdyn = kdyn;
    a.part = part;
    a.slice = slice;
    a.err = err;
    CPCP_COUNT_LAUNCH();
    prod_tc_kernel<<<dim3((unsigned)tiles, (unsigned)splits), PP_NT, PP_SMEM, st>>>(maps, a);
    return splits;
}

}  // namespace cpcp
