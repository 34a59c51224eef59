// k_small.cu -- the k x k stages of the subspace-iteration SVD and the
// per-iteration scalar schedule.  Each runs as a single CTA with its matrices
// in shared memory (k <= small_kmax<T>()).
//
//   chol      Gram reduction + Cholesky of the column-equilibrated Gram matrix
//             (CholeskyQR pass): X = Q R with Q = X R^{-1}.  Columns that are
//             numerically dependent are dropped (zero column in Q, zero row
//             in R) instead of breaking down.
//   jacobi    one-sided Jacobi SVD of the small triangular factor: the core
//             SVD of the Rayleigh-Ritz step, with singular values sorted.
//   svt_small singular value thresholding on the factors (Sec. 2.1, Alg. 1 /
//             Sec. 3.2): keeps sigma > theta, scales the kept left vectors by
//             sigma - theta, and picks the next subspace width.
//   ctrl      momentum weight, continuation weight and thresholds.
#include <cfloat>

#include "common.cuh"

namespace cpcp {

template <typename T>
constexpr int small_kmax()
{
    return sizeof(T) == 4 ? 128 : 80;
}

namespace {

template <typename T>
__device__ __forceinline__ T eps_of();
template <>
__device__ __forceinline__ float eps_of<float>()
{
    return FLT_EPSILON;
}
template <>
__device__ __forceinline__ double eps_of<double>()
{
    return DBL_EPSILON;
}

// ---------------------------------------------------------------------------
// Cholesky pass of CholeskyQR
// ---------------------------------------------------------------------------
constexpr int CHOL_NT = 512;

template <typename T>
__global__ void __launch_bounds__(CHOL_NT) chol_kernel(const T *__restrict__ partial, int splits, int kmax,
                                                       const int *kdyn, T *__restrict__ R, T *__restrict__ Rinv,
                                                       const T *__restrict__ Rprev, T *__restrict__ Rtot, int ldr)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = *kdyn;
    const int ld = k + 1;
    T *G = reinterpret_cast<T *>(smraw);  // equilibrated Gram -> upper Cholesky factor (off-diagonal)
    T *Ri = G + k * ld;                   // inverse of the factor
    T *P = Ri + k * ld;                   // Rprev (when combining two passes)
    T *d = P + k * ld;                    // column scales
    T *diag = d + k;                      // diagonal of the factor
    int *drop = reinterpret_cast<int *>(diag + k);
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

    // Gram matrix from the row-split partial sums, in a fixed order (four
    // independent chains keep several loads in flight)
    const int64_t slice = (int64_t)kmax * kmax;
    for (int idx = tid; idx < k * k; idx += nt) {
        int p = idx / k, c = idx % k;
        const T *src = partial + (int64_t)p * kmax + c;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int q = 0;
        for (; q + 3 < splits; q += 4) {
            s0 += src[q * slice];
            s1 += src[(q + 1) * slice];
            s2 += src[(q + 2) * slice];
            s3 += src[(q + 3) * slice];
        }
        for (; q < splits; q++) s0 += src[q * slice];
        G[p * ld + c] = (s0 + s1) + (s2 + s3);
    }
    if (Rprev != nullptr)
        for (int idx = tid; idx < k * k; idx += nt) P[(idx / k) * ld + idx % k] = Rprev[(int64_t)(idx / k) * ldr + idx % k];
    __syncthreads();
    for (int p = tid; p < k; p += nt) {
        T g = G[p * ld + p];
        d[p] = (g > T(0) && isfinite(g)) ? sqrt(g) : T(0);
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += nt) {
        int p = idx / k, c = idx % k;
        T dp = d[p], dc = d[c];
        G[p * ld + c] = (dp > T(0) && dc > T(0)) ? G[p * ld + c] / dp / dc : T(0);
    }
    __syncthreads();

    // right-looking Cholesky of the equilibrated Gram matrix.  Only a
    // non-positive (or denormal) pivot is a breakdown and drops the column; a
    // tiny positive pivot gives a noise direction that the next CholeskyQR
    // pass cleans up.
    const T tol = eps_of<T>() * eps_of<T>();
    for (int j = 0; j < k; j++) {
        const T piv = G[j * ld + j];
        const bool dj = !(piv > tol);
        const T inv = dj ? T(0) : T(1) / sqrt(piv);
        for (int c = j + 1 + tid; c < k; c += nt) G[j * ld + c] *= inv;
        if (tid == 0) {
            diag[j] = dj ? T(0) : sqrt(piv);
            drop[j] = dj;
        }
        __syncthreads();
        const int w = k - j - 1;
        for (int idx = tid; idx < w * w; idx += nt) {
            int a = j + 1 + idx / w, b = j + 1 + idx % w;
            if (a <= b) G[a * ld + b] -= G[j * ld + a] * G[j * ld + b];
        }
        __syncthreads();
    }

    // inverse of the factor by back substitution, one warp per column; a
    // dropped index gets a zero column (Q gets a zero column there)
    for (int c = warp; c < k; c += nw) {
        if (drop[c]) {
            for (int i = lane; i < k; i += 32) Ri[i * ld + c] = T(0);
            continue;
        }
        for (int i = c + 1 + lane; i < k; i += 32) Ri[i * ld + c] = T(0);
        if (lane == 0) Ri[c * ld + c] = T(1) / diag[c];
        __syncwarp();
        for (int i = c - 1; i >= 0; i--) {
            if (drop[i]) {
                if (lane == 0) Ri[i * ld + c] = T(0);
                __syncwarp();
                continue;
            }
            T s = T(0);
            for (int p = i + 1 + lane; p <= c; p += 32) s = fma(G[i * ld + p], Ri[p * ld + c], s);
            s = warp_sum(s);
            if (lane == 0) Ri[i * ld + c] = -s / diag[i];
            __syncwarp();
        }
    }
    __syncthreads();

    // undo the equilibration: R = Rt D, R^{-1} = D^{-1} Rt^{-1}; Rtot = R Rprev
    for (int idx = tid; idx < k * k; idx += nt) {
        int i = idx / k, c = idx % k;
        T rv = T(0), iv = T(0);
        if (c >= i && !drop[i]) rv = (c == i ? diag[i] : G[i * ld + c]) * d[c];
        if (c >= i && d[i] > T(0)) iv = Ri[i * ld + c] / d[i];
        R[(int64_t)i * ldr + c] = rv;
        Rinv[(int64_t)i * ldr + c] = iv;
        if (Rprev != nullptr) {
            T s = T(0);
            if (c >= i && !drop[i])
                for (int p = i; p <= c; p++) s = fma((p == i ? diag[i] : G[i * ld + p]) * d[p], P[p * ld + c], s);
            Rtot[(int64_t)i * ldr + c] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// one-sided Jacobi SVD of C = Rz^T (k x k): C = Ut diag(sig) Wt^T
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) jacobi_kernel(const T *__restrict__ Rz, int ldr, const int *kdyn,
                                                      T *__restrict__ Ut, T *__restrict__ Wt, T *__restrict__ sig)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int k = *kdyn;
    const int ld = k + 1;
    const int N = k + (k & 1);
    T *X = reinterpret_cast<T *>(smraw);  // X[c * ld + i]: column c of C
    T *V = X + k * ld;
    T *sv = V + k * ld;                   // squared column norms, then singular values
    int *pos = reinterpret_cast<int *>(sv + k);
    __shared__ int rot_count;
    __shared__ T amax;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;

    for (int idx = tid; idx < k * k; idx += nt) {
        int c = idx / k, i = idx % k;
        X[c * ld + i] = Rz[(int64_t)c * ldr + i];  // column c of Rz^T = row c of Rz
        V[c * ld + i] = (c == i) ? T(1) : T(0);
    }
    __syncthreads();

    // a pair is rotated when |x_p . x_q| exceeds the rounding bound of the
    // warp dot product (k/32 sequential terms per lane + a 5-level tree)
    const T tol = T(2) * T((k + 31) / 32 + 8) * eps_of<T>();
    // columns whose norm is below the rounding noise of the largest one carry
    // no information; rotating them against large columns only moves noise
    const T negl = (T(4) * T(k) * eps_of<T>()) * (T(4) * T(k) * eps_of<T>());
    for (int sweep = 0; sweep < 30; sweep++) {
        // exact squared norms at the start of each sweep; rotations then
        // update them by a' = a - t g, b' = b + t g (Rutishauser)
        for (int c = warp; c < k; c += nw) {
            T s = T(0);
            for (int i = lane; i < k; i += 32) s = fma(X[c * ld + i], X[c * ld + i], s);
            s = warp_sum(s);
            if (lane == 0) sv[c] = s;
        }
        if (tid == 0) rot_count = 0;
        __syncthreads();
        if (warp == 0) {
            T v = T(0);
            for (int c = lane; c < k; c += 32) v = max(v, sv[c]);
            for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
            if (lane == 0) amax = v;
        }
        __syncthreads();
        const T small = negl * amax;
        for (int round = 0; round < N - 1; round++) {
            // round-robin (circle) schedule: slot 0 holds column 0, slot s > 0
            // holds column 1 + (s - 1 + round) mod (N - 1); slot t meets N-1-t
            for (int pr = warp; pr < N / 2; pr += nw) {
                int sa = pr, sb = N - 1 - pr;
                int p = sa == 0 ? 0 : 1 + (sa - 1 + round) % (N - 1);
                int q = 1 + (sb - 1 + round) % (N - 1);
                if (p >= k || q >= k) continue;
                T *xp = X + p * ld, *xq = X + q * ld;
                T g = T(0);
                for (int i = lane; i < k; i += 32) g = fma(xp[i], xq[i], g);
                g = warp_sum(g);
                const T a = sv[p], b = sv[q];
                if (!(a > small) || !(b > small)) continue;
                if (fabs(g) <= tol * sqrt(a) * sqrt(b)) continue;
                T zeta = (b - a) / (T(2) * g);
                // t = sign(z) / (|z| + sqrt(1 + z^2)), or 1/(2 z) where z^2 would overflow
                T az = fabs(zeta);
                T tt = az > T(1e15) ? T(0.5) / zeta
                                    : (zeta >= T(0) ? T(1) : T(-1)) / (az + sqrt(T(1) + zeta * zeta));
                T cs = T(1) / sqrt(T(1) + tt * tt), sn = cs * tt;
                T *vp = V + p * ld, *vq = V + q * ld;
                for (int i = lane; i < k; i += 32) {
                    T u = xp[i], v = xq[i];
                    xp[i] = cs * u - sn * v;
                    xq[i] = sn * u + cs * v;
                    u = vp[i];
                    v = vq[i];
                    vp[i] = cs * u - sn * v;
                    vq[i] = sn * u + cs * v;
                }
                __syncwarp();
                if (lane == 0) {
                    sv[p] = max(a - tt * g, T(0));
                    sv[q] = b + tt * g;
                    atomicAdd(&rot_count, 1);
                }
            }
            __syncthreads();
        }
        int done = (rot_count == 0);
        __syncthreads();
        if (done) break;
    }

    for (int c = warp; c < k; c += nw) {
        T s = T(0);
        for (int i = lane; i < k; i += 32) s = fma(X[c * ld + i], X[c * ld + i], s);
        s = warp_sum(s);
        if (lane == 0) sv[c] = sqrt(s);
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
        int p = 0;
        for (int c2 = 0; c2 < k; c2++) p += (sv[c2] > sv[c]) || (sv[c2] == sv[c] && c2 < c);
        pos[c] = p;
        sig[p] = sv[c];
    }
    __syncthreads();
    for (int idx = tid; idx < k * k; idx += nt) {
        int c = idx / k, i = idx % k;
        int p = pos[c];
        T s = sv[c];
        Ut[(int64_t)i * ldr + p] = s > T(0) ? X[c * ld + i] / s : T(0);
        Wt[(int64_t)i * ldr + p] = V[c * ld + i];
    }
}

// ---------------------------------------------------------------------------
// SVT on the factors + subspace width for the next iteration
// ---------------------------------------------------------------------------
template <typename T>
__global__ void svt_small_kernel(const T *__restrict__ Ut, const T *__restrict__ sig, int ldr, Ctrl *ctrl,
                                 T *__restrict__ Us, double *sig64)
{
    __shared__ int s_r;
    const int k = ctrl->k;
    const T th = T(ctrl->theta_L);
    if (threadIdx.x == 0) s_r = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
        if (sig[c] > th) atomicAdd(&s_r, 1);
        if (sig64) sig64[c] = (double)sig[c];
    }
    __syncthreads();
    const int r = s_r;  // sig is sorted, so the kept values are the first r
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        int i = idx / k, c = idx % k;
        Us[(int64_t)i * ldr + c] = c < r ? Ut[(int64_t)i * ldr + c] * (sig[c] - th) : T(0);
    }
    if (threadIdx.x == 0) {
        ctrl->r_new = r;
        int kn = r + ctrl->oversample;
        if (kn < 1) kn = 1;
        if (kn > ctrl->kcap) kn = ctrl->kcap;
        if (r >= k && k < ctrl->kcap) ctrl->flags |= 1;
        ctrl->k_next = kn;
    }
}

// Random start columns of the subspace block: columns [k, k_next) and the
// columns whose singular value came out exactly zero (dropped directions).
template <typename T>
__global__ void fill_random_kernel(T *Omega, int64_t ldo, int rows, const Ctrl *ctrl, int all_cols,
                                   const T *__restrict__ sig, int kmax, uint64_t salt)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y;
    if (j >= rows || c >= kmax) return;
    int kc = all_cols ? 0 : ctrl->k;
    int kn = all_cols ? ctrl->k : ctrl->k_next;
    if (c >= kn) return;
    bool fill = (c >= kc) || (sig != nullptr && sig[c] == T(0));
    if (!fill) return;
    uint64_t key = ctrl->seed * 0x9E3779B97F4A7C15ull + salt * 0xD1B54A32D192ED03ull + (uint64_t)ctrl->iter * 7919ull;
    Omega[(int64_t)j * ldo + c] = T(hash_uniform(key ^ ((uint64_t)j * 1000003ull + (uint64_t)c * 0x100000001B3ull)));
}

__global__ void ctrl_begin_kernel(Ctrl *c)
{
    double mu = c->mu0 * pow(c->eta, (double)c->iter);
    if (mu < c->mu_bar) mu = c->mu_bar;
    double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * c->t * c->t));
    c->mu_k = mu;
    c->t_next = t1;
    c->beta = (c->t - 1.0) / t1;
    c->theta_L = c->tau * mu;
    c->theta_S = c->tau * c->lam * mu;
}

__global__ void ctrl_take_width_kernel(Ctrl *c) { c->k = c->k_next; }

// residual check at weight mu_c: thresholds of the check, and a width of at
// least rank(L_k) + p so that the fine SVT is not truncated
__global__ void ctrl_set_check_kernel(Ctrl *chk, const Ctrl *it, double mu_c)
{
    chk->mu_bar = mu_c;
    chk->mu_k = mu_c;
    chk->theta_L = chk->tau * mu_c;
    chk->theta_S = chk->tau * chk->lam * mu_c;
    int k = max(chk->k_next, it->rk + chk->oversample);
    chk->k_next = min(k, chk->kcap);  // columns [k, k_next) get random vectors, then k = k_next
}

__global__ void ctrl_end_kernel(Ctrl *c)
{
    c->t = c->t_next;
    c->rp = c->rk;
    c->rk = c->r_new;
    c->k = c->k_next;
    c->iter += 1;
}

template <typename T>
size_t chol_smem(int kmax)
{
    return (size_t)3 * kmax * (kmax + 1) * sizeof(T) + 2 * kmax * sizeof(T) + kmax * sizeof(int) + 16;
}

template <typename T>
size_t jacobi_smem(int kmax)
{
    return (size_t)2 * kmax * (kmax + 1) * sizeof(T) + kmax * sizeof(T) + kmax * sizeof(int) + 16;
}

template <typename T>
void ensure_small_attrs()
{
    static bool done = false;
    if (done) return;
    cudaFuncSetAttribute(chol_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)chol_smem<T>(small_kmax<T>()));
    cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)jacobi_smem<T>(small_kmax<T>()));
    done = true;
}

}  // namespace

template <typename T>
void launch_chol(const T *partialG, int splits, int kmax, const int *kdyn, T *R, T *Rinv, const T *Rprev, T *Rtot,
                 int ldr, cudaStream_t st)
{
    ensure_small_attrs<T>();
    chol_kernel<T><<<1, CHOL_NT, chol_smem<T>(kmax), st>>>(partialG, splits, kmax, kdyn, R, Rinv, Rprev, Rtot, ldr);
}

template <typename T>
void launch_jacobi(const T *Rz, int ldr, const int *kdyn, T *Ut, T *Wt, T *sig, int kmax, cudaStream_t st)
{
    ensure_small_attrs<T>();
    jacobi_kernel<T><<<1, 1024, jacobi_smem<T>(kmax), st>>>(Rz, ldr, kdyn, Ut, Wt, sig);
}

template <typename T>
void launch_svt_small(const T *Ut, const T *sig, int ldr, Ctrl *ctrl, T *Us, double *sig64, cudaStream_t st)
{
    svt_small_kernel<T><<<1, 256, 0, st>>>(Ut, sig, ldr, ctrl, Us, sig64);
}

template <typename T>
void launch_fill_random(T *Omega, int64_t ldo, int rows, const Ctrl *ctrl, int all_cols, const T *sig, int kmax,
                        uint64_t salt, cudaStream_t st)
{
    dim3 grid((kmax + 63) / 64, rows);
    fill_random_kernel<T><<<grid, 64, 0, st>>>(Omega, ldo, rows, ctrl, all_cols, sig, kmax, salt);
}

void launch_ctrl_begin(Ctrl *c, cudaStream_t st) { ctrl_begin_kernel<<<1, 1, 0, st>>>(c); }
void launch_ctrl_end(Ctrl *c, cudaStream_t st) { ctrl_end_kernel<<<1, 1, 0, st>>>(c); }
void launch_ctrl_take_width(Ctrl *c, cudaStream_t st) { ctrl_take_width_kernel<<<1, 1, 0, st>>>(c); }
void launch_ctrl_set_check(Ctrl *chk, const Ctrl *it, double mu_c, cudaStream_t st)
{
    ctrl_set_check_kernel<<<1, 1, 0, st>>>(chk, it, mu_c);
}

int small_kmax_f32() { return small_kmax<float>(); }
int small_kmax_f64() { return small_kmax<double>(); }

#define INST(T)                                                                                                      \
    template void launch_chol<T>(const T *, int, int, const int *, T *, T *, const T *, T *, int, cudaStream_t);      \
    template void launch_jacobi<T>(const T *, int, const int *, T *, T *, T *, int, cudaStream_t);                    \
    template void launch_svt_small<T>(const T *, const T *, int, Ctrl *, T *, double *, cudaStream_t);               \
    template void launch_fill_random<T>(T *, int64_t, int, const Ctrl *, int, const T *, int, uint64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cpcp
