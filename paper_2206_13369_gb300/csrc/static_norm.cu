// static_norm.cu -- ||P_Q[D]||_F and the count of non-finite observed
// entries, computed without allocating any memory.
//
// This is a variant of the masked-norm reduction of the residual pass: the
// per-tile partial sums that the solver keeps in its handle's workspace live
// here in one file-scope device array of fixed size, so the entry point needs
// no handle and never calls cudaMalloc/cudaFree.  It exists for callers that
// must not allocate device memory at call time (see include/cpcp.h).
#include <atomic>

#include "../../include/cpcp.h"
#include "common.cuh"

namespace {

constexpr int TILE = 64;              // 64 x 64 tiles, the tiling of the residual pass
constexpr int NT = 256;
constexpr int MAX_TILES = 65536;      // largest problem: ceil(m/64) * ceil(n/64) <= 65536
constexpr int MAX_DEVICES = 64;

// Scratch shared by every call on a device: two partial sums per tile
// (sum of squares, non-finite count) followed by the two results.  Every slot
// a call reads is written earlier by the same call, so nothing has to be
// cleared between calls.  Size: (2 * 65536 + 2) doubles = 1 MiB.
static __device__ __align__(256) double g_norm_scratch[2 * MAX_TILES + 2];

// Device address of g_norm_scratch on each device, resolved once per device.
static std::atomic<double *> g_scratch_addr[MAX_DEVICES];

// One block per 64 x 64 tile on a one-dimensional grid (tile b is row tile
// b / tiles_x, column tile b % tiles_x), so the tile count alone bounds the
// grid: gridDim.x may reach 2^31 - 1, far above MAX_TILES.
template <typename T>
__global__ void __launch_bounds__(NT) masked_sq_tiles(int m, int n, int tiles_x, const T *__restrict__ D,
                                                      int64_t ldd, const uint32_t *__restrict__ Q, int64_t ldq,
                                                      double *__restrict__ part)
{
    __shared__ double red[NT / 32][2];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int bx = (int)(blockIdx.x % (unsigned)tiles_x), by = (int)(blockIdx.x / (unsigned)tiles_x);
    const int col = bx * TILE + 4 * tx;
    double sq = 0.0, nf = 0.0;
    for (int i = 0; i < 4; i++) {
        const int row = by * TILE + ty + 16 * i;
        if (row >= m) continue;
        uint32_t bits = 0xffffffffu;
        if (Q != nullptr && col < n) bits = Q[(int64_t)row * ldq + (col >> 5)] >> (col & 31);
        for (int j = 0; j < 4; j++) {
            if (col + j >= n || !((bits >> j) & 1u)) continue;
            const double v = (double)D[(int64_t)row * ldd + col + j];
            if (isfinite(v))
                sq += v * v;
            else
                nf += 1.0;
        }
    }
    sq = cpcp::warp_sum(sq);
    nf = cpcp::warp_sum(nf);
    if ((t & 31) == 0) {
        red[t >> 5][0] = sq;
        red[t >> 5][1] = nf;
    }
    __syncthreads();
    if (t < 2) {
        double v = 0.0;
        for (int w = 0; w < NT / 32; w++) v += red[w][t];
        part[2 * (int64_t)blockIdx.x + t] = v;
    }
}

// fixed-order reduction of the tile partials: out[0] = norm, out[1] = count
__global__ void reduce_tiles(int tiles, const double *__restrict__ part, double *__restrict__ out)
{
    __shared__ double red[NT / 32][2];
    double sq = 0.0, nf = 0.0;
    for (int b = threadIdx.x; b < tiles; b += NT) {
        sq += part[2 * b];
        nf += part[2 * b + 1];
    }
    sq = cpcp::warp_sum(sq);
    nf = cpcp::warp_sum(nf);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5][0] = sq;
        red[threadIdx.x >> 5][1] = nf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < NT / 32; w++) {
            a += red[w][0];
            c += red[w][1];
        }
        out[0] = sqrt(a);
        out[1] = c;
    }
}

// Set-up, once per device, with that device current: the host-side name of
// g_norm_scratch is only a stand-in, the kernels need its device address.
cpcp_status scratch_address(int dev, double **out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return CPCP_ERR_INVALID_ARG;
    double *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (p == nullptr) {
        void *addr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&addr, g_norm_scratch);
        if (e != cudaSuccess || addr == nullptr) {
            cudaGetLastError();
            return CPCP_ERR_CUDA;
        }
        p = static_cast<double *>(addr);
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return CPCP_OK;
}

}  // namespace

extern "C" cpcp_status cpcp_masked_norm_static(void *stream, int m, int n, cpcp_dtype dt, const void *D, int64_t ldd,
                                               const uint32_t *Q, int64_t ldq, double *fro, int64_t *nonfinite)
{
    if (m < 1 || n < 1 || D == nullptr || ldd < n || fro == nullptr || (dt != CPCP_F32 && dt != CPCP_F64))
        return CPCP_ERR_INVALID_ARG;
    if (Q != nullptr && ldq < (n + 31) / 32) return CPCP_ERR_INVALID_ARG;
    const int64_t tx = (n + TILE - 1) / TILE, ty = (m + TILE - 1) / TILE;
    if (tx * ty > MAX_TILES) return CPCP_ERR_INVALID_ARG;  // larger than the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CPCP_ERR_CUDA;
    }
    double *scratch = nullptr;
    cpcp_status st = scratch_address(dev, &scratch);
    if (st != CPCP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaGetLastError();  // a launch error reported below is this call's own
    const unsigned tiles = (unsigned)(tx * ty);
    CPCP_COUNT_LAUNCH();
    if (dt == CPCP_F32)
        masked_sq_tiles<float><<<tiles, NT, 0, s>>>(m, n, (int)tx, static_cast<const float *>(D), ldd, Q, ldq,
                                                    scratch);
    else
        masked_sq_tiles<double><<<tiles, NT, 0, s>>>(m, n, (int)tx, static_cast<const double *>(D), ldd, Q, ldq,
                                                     scratch);
    if (cudaGetLastError() != cudaSuccess) return CPCP_ERR_CUDA;
    CPCP_COUNT_LAUNCH();
    reduce_tiles<<<1, NT, 0, s>>>((int)tiles, scratch, scratch + 2 * MAX_TILES);
    if (cudaGetLastError() != cudaSuccess) return CPCP_ERR_CUDA;
    double res[2];
    if (cudaMemcpyAsync(res, scratch + 2 * MAX_TILES, sizeof(res), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return CPCP_ERR_CUDA;
    }
    *fro = res[0];
    if (nonfinite != nullptr) *nonfinite = (int64_t)res[1];
    return CPCP_OK;
}
