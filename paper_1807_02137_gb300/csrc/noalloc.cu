// noalloc.cu -- residual norm of a grid function using statically allocated device scratch.
//
// The handle-based solver keeps its scratch (per-block partial sums of the residual norm) in
// memory it allocates at set-up.  Some callers cannot allocate device memory at the point where
// they need a residual norm: for example code that runs under a framework owning every byte of
// device memory through its own pool, or a real-time loop that may not call cudaMalloc (which
// synchronises the device) once it is running.  mg_residual_norm_noalloc serves them: it computes
// the same norm as the start of a pseudo-time step (mg_begin_step) from caller-owned inputs, with
// its partial sums held in one file-scope device array instead of allocated memory.
//
// The array is sized for kNoAllocMaxTiles 32 x 32 tiles (67,108,864 cells, e.g. 8192 x 8192);
// every GPU that loads this library holds its 512 KB until the process exits.  All calls share
// it: each call overwrites every partial it reads, so nothing needs clearing, but two calls that
// overlap on the GPU (on different streams) race on the array and give wrong results.
#include <cmath>
#include <mutex>

#include "../../include/segmg.h"
#include "arith.cuh"

namespace {

using namespace segmg;

constexpr int kNoAllocMaxTiles = 65536;
constexpr int kMaxDevices = 64;

// [0, kNoAllocMaxTiles): per-tile partial sums; [kNoAllocMaxTiles]: the total.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxTiles + 1];

std::mutex g_mu;
double *g_addr[kMaxDevices] = {};

// Block sum as the solver's norm kernels form it: each warp adds its lanes in C (the storage
// precision of the norm's per-thread sums), the warp sums are added in FP64.
template <typename C>
__device__ double block_sum_na(C v, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = (double)v;
    __syncthreads();
    if (tid < 32) {
        double s = tid < (nt + 31) / 32 ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (tid == 0) red[32] = s;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// The residual-norm tile kernel of the solver specialised to a zero increment: phi is passed
// whole (dense, pitch m) and each 32 x 32 tile writes sum r^2, r = -L(phi), to its slot.
template <typename T>
__global__ void __launch_bounds__(256) k_residual_static(const T *phi, const T *w, const T *F, int n, int m,
                                                         T cdiff, T inv_2h, T beta, double *partials) {
    constexpr int R = 36;
    __shared__ T sP[R][R + 1];
    __shared__ T sG[R][R + 1];
    __shared__ double red[33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const T z = T(0);
    for (int q = tid; q < R * R; q += 256) {
        int a = q / R, b = q % R;
        sP[a][b] = phi[(size_t)clampi(i0 - 2 + a, 0, n - 1) * m + clampi(j0 - 2 + b, 0, m - 1)];
    }
    __syncthreads();
    for (int q = tid; q < 34 * 34; q += 256) {
        int a = 1 + q / 34, b = 1 + q % 34;
        int gi = i0 - 2 + a, gj = j0 - 2 + b;
        T g = T(0);
        if (gi >= 0 && gi < n && gj >= 0 && gj < m)
            g = cell_G(w[(size_t)gi * m + gj], sP[a + 1][b], sP[a - 1][b], sP[a][b + 1], sP[a][b - 1], z, z, z, z,
                       inv_2h, beta);
        sG[a][b] = g;
    }
    __syncthreads();
    T acc = T(0);
    for (int q = tid; q < 1024; q += 256) {
        int ti = q / 32, tj = q % 32, a = ti + 2, b = tj + 2;
        int gi = i0 + ti, gj = j0 + tj;
        if (gi >= n || gj >= m) continue;
        bool hS = gi + 1 < n, hN = gi > 0, hE = gj + 1 < m, hW = gj > 0;
        T gc = sG[a][b];
        T aS = face(gc, sG[a + 1][b], hS), aN = face(gc, sG[a - 1][b], hN);
        T aE = face(gc, sG[a][b + 1], hE), aW = face(gc, sG[a][b - 1], hW);
        T pc = sP[a][b];
        T fl = mul_rn(aS, add_rn(sub_rn(sP[a + 1][b], pc), z));
        fl = fma_rn(aN, add_rn(sub_rn(sP[a - 1][b], pc), z), fl);
        fl = fma_rn(aE, add_rn(sub_rn(sP[a][b + 1], pc), z), fl);
        fl = fma_rn(aW, add_rn(sub_rn(sP[a][b - 1], pc), z), fl);
        T Lv = fma_rn(cdiff, fl, -add_rn(F[(size_t)gi * m + gj], z));
        T r = -Lv;
        acc = add_square(acc, r);
    }
    double s = block_sum_na(acc, red);
    if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

__global__ void k_sum_static(const double *partials, int np, double *out) {
    __shared__ double red[33];
    double v = 0.0;
    for (int q = threadIdx.x; q < np; q += blockDim.x) v += partials[q];
    double s = block_sum_na(v, red);
    if (threadIdx.x == 0) *out = s;
}

// Errors of this entry point are reported by their code only (mg_last_error is not updated).
int err(int code, const char *) { return code; }

template <typename T>
int run(const void *phi, const void *w, const void *F, int n, int m, const mg_params *p, double *scratch,
        cudaStream_t st) {
    dim3 grid((m + 31) / 32, (n + 31) / 32), block(32, 8);
    k_residual_static<T><<<grid, block, 0, st>>>((const T *)phi, (const T *)w, (const T *)F, n, m,
                                                 (T)(p->mu), (T)0.5, (T)p->beta, scratch);
    k_sum_static<<<1, 256, 0, st>>>(scratch, (int)(grid.x * grid.y), scratch + kNoAllocMaxTiles);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MG_OK : err(MG_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

extern "C" int mg_residual_norm_noalloc(const void *phi, const void *w, const void *F, int n, int m,
                                        const mg_params *p, double *norm, void *stream) {
    if (!phi || !w || !F || !p || !norm) return err(MG_ERR_ARG, "NULL argument");
    if (n < 1 || m < 1) return err(MG_ERR_ARG, "image size must be positive");
    if (p->model != MG_MODEL_SC) return err(MG_ERR_ARG, "only the Spencer-Chen model is supported");
    if (p->precision != MG_F32 && p->precision != MG_F64) return err(MG_ERR_ARG, "precision");
    if (!(p->mu > 0) || !(p->beta > 0)) return err(MG_ERR_ARG, "mu and beta must be > 0");
    long tiles = (long)((m + 31) / 32) * ((n + 31) / 32);
    if (tiles > kNoAllocMaxTiles)
        return err(MG_ERR_ARG, "grid exceeds the static scratch (at most 65536 tiles of 32 x 32 cells)");
    if ((n + 31) / 32 > 65535)   // the tile rows are the launch's grid.y
        return err(MG_ERR_ARG, "more than 65535 rows of 32 x 32 tiles");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return err(MG_ERR_CUDA, "no current CUDA device");
    double *scratch = nullptr;
    {
        // Once per device, with that device current: the device address of the static array.
        // Host code must not use g_noalloc_scratch itself, which names a host-side shadow.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            cudaError_t e = cudaGetSymbolAddress((void **)&g_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                return err(MG_ERR_CUDA, cudaGetErrorString(e));
            }
        }
        scratch = g_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    (void)cudaGetLastError();   // a pending error of earlier, unrelated work is not this call's
    int rc = p->precision == MG_F32 ? run<float>(phi, w, F, n, m, p, scratch, st)
                                    : run<double>(phi, w, F, n, m, p, scratch, st);
    if (rc) return rc;
    double s2 = 0.0;
    cudaError_t e = cudaMemcpyAsync(&s2, scratch + kNoAllocMaxTiles, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return err(MG_ERR_CUDA, cudaGetErrorString(e));
    *norm = std::sqrt(s2);
    return MG_OK;
}
