// k_pass.cu -- the m x n passes of one iteration.
//
// One kernel template covers four passes that share the same tile shape:
//   STEP_FINE / STEP_COARSE  the fused iteration pass (momentum extrapolation,
//       masked gradient eq. (cpcp-grad-LS), S shrink (Alg. 3 threshold), and
//       M = Lhat - tau G, written dense on the fine level or restricted to
//       M_H = M R on a coarse level (Sec. 3.1 / Alg. 4 restriction step));
//   CHECK  the same quantities at (L_k, S_k) with the final weight, plus the
//       S part of the gradient-mapping residual and ||P_Q D||;
//   DIFF   ||A_k B_k^T - A_p B_p^T||_F^2 (L part of the residual).
//
// L is never stored densely: each 64 x 64 tile of Lhat is rebuilt on chip
// from the low-rank factors (a K = r_k + r_{k-1} contraction) and consumed in
// the epilogue, so the pass moves D, S_k, S_{k-1}, the mask bits and S_{k+1}
// through HBM once.
#include "common.cuh"

namespace cpcp {

namespace {

constexpr int BM = 64, BN = 64, KC = 16, NT = 256;
constexpr int NSLOT = 3;

// STEP_COARSE_G is STEP_COARSE plus, for the coarse-gradient test of the
// level switch, the restriction G R of the gradient and ||G||_F^2.
enum Mode { STEP_FINE = 0, STEP_COARSE = 1, CHECK = 2, DIFF = 3, RECON = 4, STEP_COARSE_G = 5 };

template <typename T, bool GM>
struct Smem {
    union {
        struct {
            T As[KC][BM + 4];
            T Bs[KC][BN + 4];
        } g;
        struct {
            T Ms[BM][BN + 1];
            T Gs[GM ? BM : 1][BN + 1];
        } e;
    } u;
    int j0[BN];
    T w0[BN], w1[BN];
    double red[NT / 32][NSLOT];
};

template <typename T>
__device__ __forceinline__ bool is_finite_val(T x)
{
    return isfinite(x);
}

// Accumulate coef * A[rows, 0:r] B[cols, 0:r]^T into acc.  With COMP the sum
// is compensated (Ogita-Rump-Oishi Dot2: exact products by FMA, TwoSum on the
// running sum, errors gathered in lo), so acc + lo carries about twice the
// working precision; the residual check needs this because it subtracts two
// reconstructions of nearly equal matrices.
template <typename T, bool COMP, typename SM>
__device__ __forceinline__ void accumulate_factor(SM &sm, T acc[4][4], T lo[4][4], const T *A, int64_t lda,
                                                  const T *B, int64_t ldb, int r, T coef, int m, int n, int rb,
                                                  int cb)
{
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    for (int c0 = 0; c0 < r; c0 += KC) {
        // load: 64 rows x 16 columns of A and of B, 4 values per thread
        {
            int row = t >> 2, kk = (t & 3) * 4;
            int gr = rb + row, gc = cb + row;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                int c = c0 + kk + u;
                T av = (gr < m && c < r) ? A[(int64_t)gr * lda + c] : T(0);
                T bv = (gc < n && c < r) ? B[(int64_t)gc * ldb + c] : T(0);
                sm.u.g.As[kk + u][row] = av * coef;
                sm.u.g.Bs[kk + u][row] = bv;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; kk++) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = sm.u.g.As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = sm.u.g.Bs[kk][4 * tx + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if constexpr (COMP) {
                        T p = a[i] * b[j];
                        T e = fma(a[i], b[j], -p);
                        T s = acc[i][j] + p;
                        T z = s - acc[i][j];
                        T q = (acc[i][j] - (s - z)) + (p - z);
                        acc[i][j] = s;
                        lo[i][j] += q + e;
                    } else {
                        acc[i][j] = fma(a[i], b[j], acc[i][j]);
                    }
                }
        }
        __syncthreads();
    }
}

template <typename T>
__device__ __forceinline__ void load4(const T *p, int64_t off, int col, int n, bool vec, T v[4])
{
    if (vec && col + 3 < n) {
        if constexpr (sizeof(T) == 4) {
            float4 q = *reinterpret_cast<const float4 *>(p + off);
            v[0] = q.x;
            v[1] = q.y;
            v[2] = q.z;
            v[3] = q.w;
        } else {
            double2 q0 = *reinterpret_cast<const double2 *>(p + off);
            double2 q1 = *reinterpret_cast<const double2 *>(p + off + 2);
            v[0] = q0.x;
            v[1] = q0.y;
            v[2] = q1.x;
            v[3] = q1.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++) v[j] = (col + j < n) ? p[off + j] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void store4(T *p, int64_t off, int col, int n, bool vec, const T v[4])
{
    if (vec && col + 3 < n) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(p + off) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            *reinterpret_cast<double2 *>(p + off) = make_double2(v[0], v[1]);
            *reinterpret_cast<double2 *>(p + off + 2) = make_double2(v[2], v[3]);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            if (col + j < n) p[off + j] = v[j];
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(NT) pass_kernel(PassArgs<T> a, int vec_flags)
{
    const int *rk_ptr = a.rk, *rp_ptr = a.rp;
    constexpr bool COARSE = (MODE == STEP_COARSE || MODE == STEP_COARSE_G);
    constexpr bool GM = (MODE == STEP_COARSE_G);
    using SM = Smem<T, GM>;
    extern __shared__ __align__(16) unsigned char smraw[];
    SM &sm = *reinterpret_cast<SM *>(smraw);
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int cb = blockIdx.x * BN, rb = blockIdx.y * BM;
    const int m = a.m, n = a.n;
    const Ctrl &C = *a.ctrl;

    T coef_k, coef_p;
    if (MODE == STEP_FINE || COARSE) {
        coef_k = T(1.0 + C.beta);
        coef_p = T(-C.beta);
    } else if (MODE == CHECK) {
        coef_k = T(1);
        coef_p = T(0);
    } else if (MODE == DIFF) {
        coef_k = T(1);
        coef_p = T(-1);
    } else {
        coef_k = T(1);
        coef_p = T(0);
    }
    const int rk = rk_ptr ? *rk_ptr : 0;
    const int rp = (rp_ptr && coef_p != T(0)) ? *rp_ptr : 0;

    // fp32 residual passes use compensated sums (see accumulate_factor)
    constexpr bool COMP = (MODE == CHECK || MODE == DIFF) && sizeof(T) == 4;
    T acc[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = lo[i][j] = T(0);
    if (rk > 0) accumulate_factor<T, COMP>(sm, acc, lo, a.Ak, a.ldfa, a.Bk, a.ldfb, rk, coef_k, m, n, rb, cb);
    if (rp > 0) accumulate_factor<T, COMP>(sm, acc, lo, a.Ap, a.ldfap, a.Bp, a.ldfbp, rp, coef_p, m, n, rb, cb);
    double gsq = 0.0;

    const int col = cb + 4 * tx;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;

    if (MODE == RECON) {
        const bool vM = vec_flags & 8;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            int row = rb + ty + 16 * i;
            if (row < m) store4(a.M, (int64_t)row * a.ldm + col, col, n, vM, acc[i]);
        }
        return;
    }
    if (MODE == DIFF) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            int row = rb + ty + 16 * i;
            if (row >= m) continue;
            T part = T(0);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                T dv = acc[i][j] + lo[i][j];
                if (col + j < n) part += dv * dv;
            }
            s0 += (double)part;
        }
    } else {
        const bool vD = vec_flags & 1, vS = vec_flags & 2, vO = vec_flags & 4, vM = vec_flags & 8;
        const T tau = T(C.tau);
        const T beta = (MODE == CHECK) ? T(0) : T(C.beta);
        const T thS = (MODE == CHECK) ? T(C.tau * C.lam * C.mu_bar) : T(C.theta_S);
        if (COARSE) __syncthreads();  // smem tile reused below
#pragma unroll
        for (int i = 0; i < 4; i++) {
            int lr = ty + 16 * i, row = rb + lr;
            if (row >= m) continue;
            T d[4], sk[4], sp[4];
            load4(a.D, (int64_t)row * a.ldd + col, col, n, vD, d);
            if (a.Sk) {
                load4(a.Sk, (int64_t)row * a.lds + col, col, n, vS, sk);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) sk[j] = T(0);
            }
            if (MODE != CHECK && a.Sp && beta != T(0)) {
                load4(a.Sp, (int64_t)row * a.lds + col, col, n, vS, sp);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) sp[j] = sk[j];
            }
            uint32_t bits = 0xffffffffu;
            if (a.Q && col < n) bits = a.Q[(int64_t)row * a.ldq + (col >> 5)] >> (col & 31);
            T so[4], mo[4], go[4];
            T ps = T(0), pd = T(0), pg = T(0);
            int nf = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                bool obs = (bits >> j) & 1u;
                bool inb = col + j < n;
                T sh = sk[j] + beta * (sk[j] - sp[j]);
                // L + S - D with the large terms cancelled first (lo = 0
                // unless the sum is compensated)
                T g = obs ? (((acc[i][j] - d[j]) + sh) + lo[i][j]) : T(0);
                T sn = shrink(sh - tau * g, thS);
                so[j] = sn;
                mo[j] = (acc[i][j] + lo[i][j]) - tau * g;
                go[j] = g;
                if (GM && inb) pg += g * g;
                if (MODE == CHECK && inb) {
                    T e = sk[j] - sn;
                    ps += e * e;
                    if (obs) {
                        if (is_finite_val(d[j]))
                            pd += d[j] * d[j];
                        else
                            nf++;
                    }
                }
            }
            if (MODE == STEP_FINE || COARSE)
                store4(a.Sout, (int64_t)row * a.ldso + col, col, n, vO, so);
            if (MODE == STEP_FINE || MODE == CHECK) {
                store4(a.M, (int64_t)row * a.ldm + col, col, n, vM, mo);
            } else if (COARSE) {
#pragma unroll
                for (int j = 0; j < 4; j++) sm.u.e.Ms[lr][4 * tx + j] = mo[j];
                if constexpr (GM) {
#pragma unroll
                    for (int j = 0; j < 4; j++) sm.u.e.Gs[lr][4 * tx + j] = go[j];
                    gsq += (double)pg;
                }
            }
            if (MODE == CHECK) {
                s0 += (double)ps;
                s1 += (double)pd;
                s2 += (double)nf;
            }
        }
    }

    if (COARSE) {
        // restriction of the tile: M_H[row, c] += sum_j M[row, j] R[j, c]
        if (t < BN) {
            int j = cb + t;
            if (j < n) {
                sm.j0[t] = a.tr.j0[j];
                sm.w0[t] = a.tr.w0[j];
                sm.w1[t] = a.tr.w1[j];
            } else {
                sm.j0[t] = -4;
                sm.w0[t] = T(0);
                sm.w1[t] = T(0);
            }
        }
        __syncthreads();
        const int jlast = min(cb + BN, n) - 1;
        const int c_lo = a.tr.j0[cb];
        const int c_hi = min(a.tr.j0[jlast] + 1, a.tr.nh - 1);
        const int ncol = c_hi - c_lo + 1;
        const int rows = min(BM, m - rb);
        for (int p = t; p < rows * ncol; p += NT) {
            int lr = p / ncol, c = c_lo + p % ncol;
            int jlo = max(a.tr.clo[c], cb), jhi = min(a.tr.chi[c], jlast);
            T s = T(0), sg = T(0);
            for (int j = jlo; j <= jhi; j++) {
                int lj = j - cb;
                T w = (sm.j0[lj] == c) ? sm.w0[lj] : ((sm.j0[lj] + 1 == c) ? sm.w1[lj] : T(0));
                s = fma(sm.u.e.Ms[lr][lj], w, s);
                if constexpr (GM) sg = fma(sm.u.e.Gs[lr][lj], w, sg);
            }
            if (jlo <= jhi) {
                atomicAdd(&a.MH[(int64_t)(rb + lr) * a.ldh + c], s);
                if constexpr (GM) atomicAdd(&a.GH[(int64_t)(rb + lr) * a.ldh + c], sg);
            }
        }
    }
    if constexpr (GM) {
        s0 = gsq;
        s1 = 0.0;
        s2 = 0.0;
    }

    if (MODE == CHECK || MODE == DIFF || GM) {
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if ((t & 31) == 0) {
            sm.red[t >> 5][0] = s0;
            sm.red[t >> 5][1] = s1;
            sm.red[t >> 5][2] = s2;
        }
        __syncthreads();
        if (t < NSLOT) {
            double v = 0.0;
            for (int w = 0; w < NT / 32; w++) v += sm.red[w][t];
            a.partial[((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * NSLOT + t] = v;
        }
    }
}

template <typename T>
int vec_flags_for(const PassArgs<T> &a)
{
    auto al = [](const void *p, int64_t ld) {
        return p == nullptr || ((reinterpret_cast<uintptr_t>(p) % 16 == 0) && (ld % (16 / (int64_t)sizeof(T)) == 0));
    };
    int f = 0;
    if (al(a.D, a.ldd)) f |= 1;
    if (al(a.Sk, a.lds) && al(a.Sp, a.lds)) f |= 2;
    if (al(a.Sout, a.ldso)) f |= 4;
    if (al(a.M, a.ldm)) f |= 8;
    return f;
}

template <typename T, int MODE>
int launch_mode(const PassArgs<T> &a, cudaStream_t st)
{
    using SM = Smem<T, MODE == STEP_COARSE_G>;
    if constexpr (sizeof(SM) > 48 * 1024) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(pass_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM));
            attr = true;
        }
    }
    dim3 grid((a.n + BN - 1) / BN, (a.m + BM - 1) / BM);
    CPCP_COUNT_LAUNCH();
    pass_kernel<T, MODE><<<grid, NT, sizeof(SM), st>>>(a, vec_flags_for(a));
    return grid.x * grid.y;
}

__global__ void sum_partials_kernel(const double *partial, int nblocks, int nslots, double *out)
{
    __shared__ double red[32];
    for (int s = 0; s < nslots; s++) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[(int64_t)b * nslots + s];
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += red[w];
            out[s] = tot;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// fine-level step pass, fp32, 128 x 128 tiles
// ---------------------------------------------------------------------------
// The fine pass is a K = r_k + r_{k-1} contraction (the Lhat tile from the
// factors) with an elementwise epilogue.  With 64 x 64 tiles and 4 x 4
// register tiles the contraction is bound by shared-memory loads; here each
// thread holds an 8 x 8 tile (four 16-byte shared loads feed 64 FMAs; its
// columns are 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3, so neighbouring
// threads read neighbouring 16-byte chunks, in shared and in global memory), the
// next K chunk of A and B is fetched into registers (16-byte loads) while the
// current one is multiplied, and the shared staging rows are padded so the
// transposed stores do not conflict.  Requires 16-byte aligned operands and
// leading dimensions that are multiples of 4 (checked by the launcher).
constexpr int FBM = 128, FBN = 128, FKC = 8, FNT = 256, FPAD = 4;

struct FineSmem {
    float As[FKC][FBM + FPAD];
    float Bs[FKC][FBN + FPAD];
};

__global__ void __launch_bounds__(FNT, 2) pass_fine_f32_kernel(PassArgs<float> a)
{
    __shared__ __align__(16) FineSmem sm;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int cb = blockIdx.x * FBN, rb = blockIdx.y * FBM;
    const int m = a.m, n = a.n;
    const Ctrl &C = *a.ctrl;
    const float beta = (float)C.beta;
    const float coef_k = (float)(1.0 + C.beta), coef_p = (float)(-C.beta);
    const int rk = a.rk ? *a.rk : 0;
    const int rp = (a.rp && coef_p != 0.f) ? *a.rp : 0;
    const int ck = (rk + FKC - 1) / FKC, cp = (rp + FKC - 1) / FKC, nchunk = ck + cp;

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = 0.f;

    // staging: thread t loads 4 consecutive K values of row t/2 of the A and
    // the B chunk (columns (t%2)*4 .. +3 of the chunk)
    const int srow = t >> 1, skk = (t & 1) * 4;
    float4 ra, rb4;
    auto fetch = [&](int ch) {
        const bool second = ch >= ck;
        const float *A = second ? a.Ap : a.Ak;
        const float *B = second ? a.Bp : a.Bk;
        const int64_t lda = second ? a.ldfap : a.ldfa, ldb = second ? a.ldfbp : a.ldfb;
        const int r = second ? rp : rk;
        const float coef = second ? coef_p : coef_k;
        const int c0 = (second ? ch - ck : ch) * FKC + skk;
        const int gr = rb + srow, gc = cb + srow;
        float av[4] = {0.f, 0.f, 0.f, 0.f}, bv[4] = {0.f, 0.f, 0.f, 0.f};
        if (c0 + 3 < r) {
            if (gr < m) {
                const float4 q = *reinterpret_cast<const float4 *>(A + (int64_t)gr * lda + c0);
                av[0] = q.x; av[1] = q.y; av[2] = q.z; av[3] = q.w;
            }
            if (gc < n) {
                const float4 q = *reinterpret_cast<const float4 *>(B + (int64_t)gc * ldb + c0);
                bv[0] = q.x; bv[1] = q.y; bv[2] = q.z; bv[3] = q.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (c0 + u < r) {
                    if (gr < m) av[u] = A[(int64_t)gr * lda + c0 + u];
                    if (gc < n) bv[u] = B[(int64_t)gc * ldb + c0 + u];
                }
            }
        }
        ra = make_float4(av[0] * coef, av[1] * coef, av[2] * coef, av[3] * coef);
        rb4 = make_float4(bv[0], bv[1], bv[2], bv[3]);
    };
    auto stage = [&]() {
        sm.As[skk + 0][srow] = ra.x;
        sm.As[skk + 1][srow] = ra.y;
        sm.As[skk + 2][srow] = ra.z;
        sm.As[skk + 3][srow] = ra.w;
        sm.Bs[skk + 0][srow] = rb4.x;
        sm.Bs[skk + 1][srow] = rb4.y;
        sm.Bs[skk + 2][srow] = rb4.z;
        sm.Bs[skk + 3][srow] = rb4.w;
    };
    if (nchunk > 0) {
        fetch(0);
        stage();
    }
    __syncthreads();
    for (int ch = 0; ch < nchunk; ch++) {
        const bool more = ch + 1 < nchunk;
        if (more) fetch(ch + 1);
#pragma unroll
        for (int kk = 0; kk < FKC; kk++) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&sm.As[kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&sm.As[kk][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&sm.Bs[kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&sm.Bs[kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 8; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
        if (more) stage();
        __syncthreads();
    }

    // epilogue: rows rb + ty*8 + i; columns cb + 4 tx .. +3 (h = 0) and
    // cb + 64 + 4 tx .. +3 (h = 1), each group inside one mask word
    const float tau = (float)C.tau, thS = (float)C.theta_S;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int row = rb + ty * 8 + i;
        if (row >= m) continue;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int c4 = cb + 64 * h + tx * 4;
            if (c4 >= n) continue;
            const bool full = c4 + 3 < n;
            uint32_t bits = 0xffffffffu;
            if (a.Q) bits = a.Q[(int64_t)row * a.ldq + (c4 >> 5)] >> (c4 & 31);
            float d[4], sk[4], sp[4], so[4], mo[4];
            if (full) {
                const float4 qd = *reinterpret_cast<const float4 *>(a.D + (int64_t)row * a.ldd + c4);
                const float4 qs = *reinterpret_cast<const float4 *>(a.Sk + (int64_t)row * a.lds + c4);
                d[0] = qd.x; d[1] = qd.y; d[2] = qd.z; d[3] = qd.w;
                sk[0] = qs.x; sk[1] = qs.y; sk[2] = qs.z; sk[3] = qs.w;
                if (a.Sp && beta != 0.f) {
                    const float4 qp = *reinterpret_cast<const float4 *>(a.Sp + (int64_t)row * a.lds + c4);
                    sp[0] = qp.x; sp[1] = qp.y; sp[2] = qp.z; sp[3] = qp.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++) sp[j] = sk[j];
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const bool in = c4 + j < n;
                    d[j] = in ? a.D[(int64_t)row * a.ldd + c4 + j] : 0.f;
                    sk[j] = in ? a.Sk[(int64_t)row * a.lds + c4 + j] : 0.f;
                    sp[j] = (in && a.Sp && beta != 0.f) ? a.Sp[(int64_t)row * a.lds + c4 + j] : sk[j];
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const bool obs = (bits >> j) & 1u;
                const float sh = sk[j] + beta * (sk[j] - sp[j]);
                const float l = acc[i][4 * h + j];
                const float g = obs ? ((l - d[j]) + sh) : 0.f;
                so[j] = shrink(sh - tau * g, thS);
                mo[j] = l - tau * g;
            }
            if (full) {
                *reinterpret_cast<float4 *>(a.Sout + (int64_t)row * a.ldso + c4) = make_float4(so[0], so[1], so[2], so[3]);
                *reinterpret_cast<float4 *>(a.M + (int64_t)row * a.ldm + c4) = make_float4(mo[0], mo[1], mo[2], mo[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if (c4 + j < n) {
                        a.Sout[(int64_t)row * a.ldso + c4 + j] = so[j];
                        a.M[(int64_t)row * a.ldm + c4 + j] = mo[j];
                    }
                }
            }
        }
    }
}

bool fine_f32_ok(const PassArgs<float> &a)
{
    auto al = [](const void *p, int64_t ld) {
        return p == nullptr || ((reinterpret_cast<uintptr_t>(p) % 16 == 0) && (ld % 4 == 0));
    };
    return a.Sk != nullptr && al(a.D, a.ldd) && al(a.Sk, a.lds) && al(a.Sp, a.lds) && al(a.Sout, a.ldso) &&
           al(a.M, a.ldm) && al(a.Ak, a.ldfa) && al(a.Bk, a.ldfb) && al(a.Ap, a.ldfap) && al(a.Bp, a.ldfbp);
}

}  // namespace

template <typename T>
int launch_step_pass(const PassArgs<T> &a, bool coarse, cudaStream_t st)
{
    if (coarse && a.GH != nullptr) return launch_mode<T, STEP_COARSE_G>(a, st);
    if (coarse) return launch_mode<T, STEP_COARSE>(a, st);
    if constexpr (sizeof(T) == 4) {
        if (fine_f32_ok(a)) {
            dim3 grid((a.n + FBN - 1) / FBN, (a.m + FBM - 1) / FBM);
            CPCP_COUNT_LAUNCH();
            pass_fine_f32_kernel<<<grid, FNT, 0, st>>>(a);
            return grid.x * grid.y;
        }
    }
    return launch_mode<T, STEP_FINE>(a, st);
}

// sum of squares of a rows x cols matrix (leading dimension ld): fixed grid,
// one fp64 partial per block, reduced in a fixed order by sum_partials
constexpr int SUMSQ_BLOCKS = 304;

template <typename T>
__global__ void __launch_bounds__(256) sumsq_kernel(int rows, int cols, const T *__restrict__ X, int64_t ld,
                                                    double *__restrict__ partial)
{
    __shared__ double red[8];
    double s = 0.0;
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = idx / cols, c = idx % cols;
        const double v = (double)X[r * ld + c];
        s += v * v;
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[w];
        partial[blockIdx.x] = t;
    }
}

template <typename T>
int launch_sumsq(int rows, int cols, const T *X, int64_t ld, double *partial, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    sumsq_kernel<T><<<SUMSQ_BLOCKS, 256, 0, st>>>(rows, cols, X, ld, partial);
    return SUMSQ_BLOCKS;
}

template <typename T>
int launch_check_pass(const PassArgs<T> &a, cudaStream_t st)
{
    return launch_mode<T, CHECK>(a, st);
}

template <typename T>
int launch_diff_pass(const PassArgs<T> &a, cudaStream_t st)
{
    return launch_mode<T, DIFF>(a, st);
}

template <typename T>
void launch_reconstruct(const PassArgs<T> &a, cudaStream_t st)
{
    launch_mode<T, RECON>(a, st);
}

void launch_sum_partials(const double *partial, int nblocks, int nslots, double *out, cudaStream_t st)
{
    CPCP_COUNT_LAUNCH();
    sum_partials_kernel<<<1, 256, 0, st>>>(partial, nblocks, nslots, out);
}

template int launch_step_pass<float>(const PassArgs<float> &, bool, cudaStream_t);
template int launch_step_pass<double>(const PassArgs<double> &, bool, cudaStream_t);
template int launch_sumsq<float>(int, int, const float *, int64_t, double *, cudaStream_t);
template int launch_sumsq<double>(int, int, const double *, int64_t, double *, cudaStream_t);
template int launch_check_pass<float>(const PassArgs<float> &, cudaStream_t);
template int launch_check_pass<double>(const PassArgs<double> &, cudaStream_t);
template int launch_diff_pass<float>(const PassArgs<float> &, cudaStream_t);
template int launch_diff_pass<double>(const PassArgs<double> &, cudaStream_t);
template void launch_reconstruct<float>(const PassArgs<float> &, cudaStream_t);
template void launch_reconstruct<double>(const PassArgs<double> &, cudaStream_t);

}  // namespace cpcp
