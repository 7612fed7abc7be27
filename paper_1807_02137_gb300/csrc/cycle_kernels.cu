// cycle_kernels.cu -- residual, grid transfers and the coarsest solve of the FAS V-cycle
// (Sec. 3.1, Algorithm 1).
#include "arith.cuh"

namespace segmg {

namespace {

// Sum of a per-thread double over the block (blockDim.x * blockDim.y <= 1024); the result is
// returned to every thread.  Fixed reduction order: deterministic.
__device__ double block_sum(double v, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
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

__device__ double block_max(double v, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        double s = tid < (nt + 31) / 32 ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
        if (tid == 0) red[32] = s;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------------------
// Residual of L (the row-scaled operator of one pseudo-time step) on 32 x 32 tiles:
//   L(phi) = mu/h^2 sum_X G_X ((pn_X - pn) + (u_X - u)) - F - area - u / tau,
// mode 0: out = rhs - L(pn + uin) and a per-block FP64 partial of sum out^2;
// mode 1: out += L(pn + uin)   (the FAS right-hand side f^{2h} = N^{2h} phi^{2h} + r^{2h}).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_residual(LevelView<T> L, const T *uin, const double *area,
                                                  T *out, int mode, double *partials) {
    constexpr int R = 36;
    __shared__ T sP[R][R + 1];
    __shared__ T sU[R][R + 1];
    __shared__ T sG[R][R + 1];
    // FP32 stages w and F in shared memory too; FP64 reads them from global memory
    constexpr bool kStage = sizeof(T) == 4;
    constexpr int RW = kStage ? R : 1, FW = kStage ? 32 : 1;
    __shared__ T sW[RW][RW + 1];
    __shared__ T sF[FW][FW + 1];
    __shared__ double red[33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int n = L.n, m = L.m, p = L.pitch;
    // stage pn, uin (mirror-clamped), w and F (FP32 only) with vector loads
    load_halo2<T>(sP, L.pn, sU, uin, i0, j0, n, m, p, tid);
    if (kStage) {
        if (!L.wb) load_halo2<T>(reinterpret_cast<T (*)[37]>(sW), L.w, nullptr, nullptr, i0, j0, n, m, p, tid);
        load_tile32<T>(reinterpret_cast<T (*)[33]>(sF), L.F, nullptr, nullptr, i0, j0, n, m, p, tid);
    }
    __syncthreads();
    for (int q = tid; q < 34 * 34; q += 256) {
        int a = 1 + q / 34, b = 1 + q % 34;
        int gi = i0 - 2 + a, gj = j0 - 2 + b;
        T g = T(0);
        if (gi >= 0 && gi < n && gj >= 0 && gj < m)
            g = cell_G((L.wb || !kStage) ? weight_at(L, (size_t)gi * p + gj) : sW[kStage ? a : 0][kStage ? b : 0],
                       sP[a + 1][b], sP[a - 1][b],
                       sP[a][b + 1], sP[a][b - 1], sU[a + 1][b], sU[a - 1][b], sU[a][b + 1], sU[a][b - 1],
                       L.inv_2h, L.beta);
        sG[a][b] = g;
    }
    __syncthreads();
    const T ar = area ? T(area[L.level]) : T(0);
    T acc = T(0);
    for (int q = tid; q < 1024; q += 256) {
        int ti = q / 32, tj = q % 32, a = ti + 2, b = tj + 2;
        int gi = i0 + ti, gj = j0 + tj;
        if (gi >= n || gj >= m) continue;
        bool hS = gi + 1 < n, hN = gi > 0, hE = gj + 1 < m, hW = gj > 0;
        T gc = sG[a][b];
        T aS = face(gc, sG[a + 1][b], hS), aN = face(gc, sG[a - 1][b], hN);
        T aE = face(gc, sG[a][b + 1], hE), aW = face(gc, sG[a][b - 1], hW);
        T pc = sP[a][b], uc = sU[a][b];
        T fl = mul_rn(aS, add_rn(sub_rn(sP[a + 1][b], pc), sub_rn(sU[a + 1][b], uc)));
        fl = fma_rn(aN, add_rn(sub_rn(sP[a - 1][b], pc), sub_rn(sU[a - 1][b], uc)), fl);
        fl = fma_rn(aE, add_rn(sub_rn(sP[a][b + 1], pc), sub_rn(sU[a][b + 1], uc)), fl);
        fl = fma_rn(aW, add_rn(sub_rn(sP[a][b - 1], pc), sub_rn(sU[a][b - 1], uc)), fl);
        size_t o = (size_t)gi * p + gj;
        T Fv = kStage ? sF[kStage ? ti : 0][kStage ? tj : 0] : L.F[o];
        T Lv = sub_rn(fma_rn(L.cdiff, fl, -add_rn(Fv, ar)), mul_rn(L.inv_tau, uc));
        if (mode == 0) {
            T r = L.has_rhs ? sub_rn(L.rhs[o], Lv) : -Lv;
            out[o] = r;
            acc = add_square(acc, r);
        } else {
            out[o] = add_rn(out[o], Lv);
        }
    }
    if (mode == 0) {
        double s = block_sum((double)acc, red);
        if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// Sums `np` partials in a fixed order into *out.
__global__ void k_sum_partials(const double *partials, int np, double *out) {
    __shared__ double red[33];
    double v = 0.0;
    for (int q = threadIdx.x; q < np; q += blockDim.x) v += partials[q];
    double s = block_sum(v, red);
    if (threadIdx.x == 0) *out = s;
}

// One-dimensional full-weighting taps (Sec. 3.1): coarse I sits on fine 2I+1; (1/4, 1/2, 1/4)
// on 2I, 2I+1, 2I+2, or (1/2, 1/2) on 2I, 2I+1 when fine 2I+2 does not exist.
__device__ __forceinline__ int fw_taps(int I, int n, int *idx, double *wt) {
    int q = 2 * I + 1;
    if (q + 1 < n) {
        idx[0] = q - 1; idx[1] = q; idx[2] = q + 1;
        wt[0] = 0.25; wt[1] = 0.5; wt[2] = 0.25;
        return 3;
    }
    idx[0] = q - 1; idx[1] = q;
    wt[0] = 0.5; wt[1] = 0.5;
    return 2;
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict(const T *f, int n, int m, int pf, T *c, T *c2, int pc) {
    const int J = blockIdx.x * 32 + threadIdx.x, I = blockIdx.y * 8 + threadIdx.y;
    const int nc = n / 2, mc = m / 2;
    if (I >= nc || J >= mc) return;
    int ri[3], ci[3];
    double rw[3], cw[3];
    int nr = fw_taps(I, n, ri, rw), nk = fw_taps(J, m, ci, cw);
    T s = T(0);
    for (int a = 0; a < nr; ++a) {
        T row = T(0);
        for (int b = 0; b < nk; ++b) row = fma_rn(T(cw[b]), f[(size_t)ri[a] * pf + ci[b]], row);
        s = fma_rn(T(rw[a]), row, s);
    }
    c[(size_t)I * pc + J] = s;
    if (c2) c2[(size_t)I * pc + J] = s;
}

// One-dimensional bilinear taps (Sec. 3.1): fine 2I+1 takes coarse I; fine 2I+2 the mean of
// coarse I and I+1; fine 0 (and fine n-1 for odd n) the single nearest coarse value.
__device__ __forceinline__ int bl_taps(int p, int nc, int *idx, double *wt) {
    if (p & 1) { idx[0] = (p - 1) / 2; wt[0] = 1.0; return 1; }
    if (p == 0) { idx[0] = 0; wt[0] = 1.0; return 1; }
    int I = p / 2 - 1;
    if (I + 1 < nc) { idx[0] = I; idx[1] = I + 1; wt[0] = 0.5; wt[1] = 0.5; return 2; }
    idx[0] = I; wt[0] = 1.0;
    return 1;
}

// Interpolation and correction: u_f += P (u_c - u0_c)  (Algorithm 1, "Interpolation").
template <typename T>
__global__ void __launch_bounds__(256) k_interp_add(LevelView<T> Lf, LevelView<T> Lc) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i >= Lf.n || j >= Lf.m) return;
    int ri[2], ci[2];
    double rw[2], cw[2];
    int nr = bl_taps(i, Lc.n, ri, rw), nk = bl_taps(j, Lc.m, ci, cw);
    T s = T(0);
    for (int a = 0; a < nr; ++a)
        for (int b = 0; b < nk; ++b) {
            size_t o = (size_t)ri[a] * Lc.pitch + ci[b];
            s = fma_rn(T(rw[a] * cw[b]), sub_rn(Lc.u[o], Lc.u0[o]), s);
        }
    size_t o = (size_t)i * Lf.pitch + j;
    Lf.u[o] = add_rn(Lf.u[o], s);
}

// ---------------------------------------------------------------------------------------
// Coarsest solve (Algorithm 1, "compute the exact solution"), one block, FP64.
// Picard on the frozen coefficients: each step solves
//   (mu/h^2 sum_X G_X + 1/tau) phi - mu/h^2 sum_X G_X phi_X = -(F - pn/tau + area + rhs)
// (symmetric positive definite) by banded Cholesky with cells ordered along the shorter side,
// until the nonlinear residual falls below tol times its initial value, a step changes no
// value by more than 1e-14 of the largest, or maxit steps.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_coarse(LevelView<T> L, ModelParams mp, double A1frac,
                                                double h2nm, int maxit, double tol, double *scratch,
                                                Scalars *sc) {
    extern __shared__ double smem_coarse[];
    if (!scratch) scratch = smem_coarse;          // small grids: everything in shared memory
    __shared__ double red[33];
    __shared__ int s_err;
    const int n = L.n, m = L.m, p = L.pitch, N = n * m;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool colmajor = m > n;
    const int bw = colmajor ? n : m, bw1 = bw + 1;
    double *x = scratch, *G = x + N, *b = G + N, *y = b + N, *band = y + N;
    const double hinv = 2.0 * (double)L.inv_2h;
    const double cdiff = mp.mu * hinv * hinv;
    const double inv_tau = (double)L.inv_tau, inv_2h = (double)L.inv_2h, beta = (double)L.beta;
    auto idx = [&](int i, int j) { return colmajor ? j * n + i : i * m + j; };
    if (tid == 0) s_err = 0;
    for (int q = tid; q < N; q += nt) {
        int i = q / m, j = q % m;
        x[idx(i, j)] = (double)L.pn[(size_t)i * p + j] + (double)L.u[(size_t)i * p + j];
    }
    __syncthreads();
    // G at x and the Rada-Chen area term; returns the area term
    auto coeffs = [&]() -> double {
        double area = 0.0;
        if (mp.model == 1) {
            double hs = 0.0;
            for (int q = tid; q < N; q += nt) hs += 0.5 + atan(x[q] / mp.eps) / M_PI;
            hs = block_sum(hs, red);
            area = 2.0 * mp.nu * (h2nm * hs - A1frac);
        }
        for (int q = tid; q < N; q += nt) {
            int i = q / m, j = q % m;
            int iS = min(i + 1, n - 1), iN = max(i - 1, 0), jE = min(j + 1, m - 1), jW = max(j - 1, 0);
            double gy = (x[idx(iS, j)] - x[idx(iN, j)]) * inv_2h;
            double gx = (x[idx(i, jE)] - x[idx(i, jW)]) * inv_2h;
            G[idx(i, j)] = (double)weight_at(L, (size_t)i * p + j) / sqrt(gx * gx + gy * gy + beta);
        }
        __syncthreads();
        return area;
    };
    auto faceG = [&](int i, int j, int i2, int j2) { return 0.5 * (G[idx(i, j)] + G[idx(i2, j2)]); };
    auto resnorm = [&]() -> double {
        double area = coeffs();
        double acc = 0.0;
        for (int q = tid; q < N; q += nt) {
            int i = q / m, j = q % m;
            double xc = x[idx(i, j)], fl = 0.0;
            if (i + 1 < n) fl += faceG(i, j, i + 1, j) * (x[idx(i + 1, j)] - xc);
            if (i > 0) fl += faceG(i, j, i - 1, j) * (x[idx(i - 1, j)] - xc);
            if (j + 1 < m) fl += faceG(i, j, i, j + 1) * (x[idx(i, j + 1)] - xc);
            if (j > 0) fl += faceG(i, j, i, j - 1) * (x[idx(i, j - 1)] - xc);
            size_t o = (size_t)i * p + j;
            double pn = (double)L.pn[o];
            double Lv = cdiff * fl - (double)L.F[o] - area - inv_tau * (xc - pn);
            double r = (L.has_rhs ? (double)L.rhs[o] : 0.0) - Lv;
            acc += r * r;
        }
        return sqrt(block_sum(acc, red));
    };
    const double r0 = resnorm();
    double res = r0;
    int it = 0;
    while (it < maxit) {
        if (it > 0) {
            res = resnorm();
            if (res <= tol * r0 || res == 0.0) break;
        }
        if (r0 == 0.0) break;
        double area = coeffs();
        for (int q = tid; q < N * bw1; q += nt) band[q] = 0.0;
        __syncthreads();
        for (int q = tid; q < N; q += nt) {
            int i = q / m, j = q % m, r = idx(i, j);
            double diag = 0.0;
            auto off = [&](int i2, int j2) {
                double a = cdiff * faceG(i, j, i2, j2);
                diag += a;
                int c = idx(i2, j2);
                if (c < r) band[(size_t)r * bw1 + (r - c)] = -a;
            };
            if (i + 1 < n) off(i + 1, j);
            if (i > 0) off(i - 1, j);
            if (j + 1 < m) off(i, j + 1);
            if (j > 0) off(i, j - 1);
            band[(size_t)r * bw1] = diag + inv_tau;
            size_t o = (size_t)i * p + j;
            b[r] = -((double)L.F[o] - inv_tau * (double)L.pn[o] + area + (L.has_rhs ? (double)L.rhs[o] : 0.0));
        }
        __syncthreads();
        // right-looking banded Cholesky: band[r*bw1 + (r-c)] = L(r, c)
        for (int k = 0; k < N && !s_err; ++k) {
            if (tid == 0) {
                double d = band[(size_t)k * bw1];
                if (!(d > 0.0)) s_err = 1;
                else band[(size_t)k * bw1] = sqrt(d);
            }
            __syncthreads();
            if (s_err) break;
            const double lkk = band[(size_t)k * bw1];
            const int last = min(k + bw, N - 1), cnt = last - k;
            for (int t = tid; t < cnt; t += nt) band[(size_t)(k + 1 + t) * bw1 + (1 + t)] /= lkk;
            __syncthreads();
            for (int t = tid; t < cnt * cnt; t += nt) {
                // the trailing triangle: rows ii >= columns jj (integer indexing only)
                const int ii = t / cnt, jj = t - ii * cnt;
                if (jj > ii) continue;
                int ri = k + 1 + ii, rj = k + 1 + jj;
                band[(size_t)ri * bw1 + (ri - rj)] -= band[(size_t)ri * bw1 + (ri - k)] * band[(size_t)rj * bw1 + (rj - k)];
            }
            __syncthreads();
        }
        if (s_err) break;
        // forward and backward substitution by warp 0
        if (tid < 32) {
            for (int r = 0; r < N; ++r) {
                double s = 0.0;
                for (int c = max(0, r - bw) + tid; c < r; c += 32) s += band[(size_t)r * bw1 + (r - c)] * y[c];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                if (tid == 0) y[r] = (b[r] - s) / band[(size_t)r * bw1];
                __syncwarp();
            }
            for (int r = N - 1; r >= 0; --r) {
                double s = 0.0;
                int c1 = min(N - 1, r + bw);
                for (int c = r + 1 + tid; c <= c1; c += 32) s += band[(size_t)c * bw1 + (c - r)] * b[c];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                if (tid == 0) b[r] = (y[r] - s) / band[(size_t)r * bw1];
                __syncwarp();
            }
        }
        __syncthreads();
        double dmax = 0.0, pmax = 1.0;
        for (int q = tid; q < N; q += nt) {
            dmax = fmax(dmax, fabs(b[q] - x[q]));
            pmax = fmax(pmax, fabs(b[q]));
        }
        dmax = block_max(dmax, red);
        pmax = block_max(pmax, red);
        for (int q = tid; q < N; q += nt) x[q] = b[q];
        __syncthreads();
        ++it;
        if (dmax <= 1e-14 * pmax) break;
    }
    for (int q = tid; q < N; q += nt) {
        int i = q / m, j = q % m;
        size_t o = (size_t)i * p + j;
        L.u[o] = (T)(x[idx(i, j)] - (double)L.pn[o]);
    }
    if (tid == 0) {
        sc->picard = it;
        sc->coarse_res = res;
        if (s_err) sc->err = 1;
    }
}

}  // namespace

int num_partials(int n, int m) { return ((m + 31) / 32) * ((n + 31) / 32); }

size_t coarse_scratch_doubles(int n, int m) {
    size_t N = (size_t)n * m, bw = (size_t)(m > n ? n : m);
    return 4 * N + N * (bw + 1);
}

template <typename T>
void launch_residual(const LevelView<T> &L, const T *uin, const double *area, T *out, int mode,
                     double *partials, int npart, double *norm_out, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32), block(32, 8);
    k_residual<T><<<grid, block, 0, st>>>(L, uin, area, out, mode, partials);
    if (mode == 0 && norm_out) k_sum_partials<<<1, 1024, 0, st>>>(partials, npart, norm_out);
}

template <typename T>
void launch_restrict(const T *f, int n, int m, int pf, T *c, T *c2, int pc, cudaStream_t st) {
    dim3 grid((m / 2 + 31) / 32, (n / 2 + 7) / 8), block(32, 8);
    k_restrict<T><<<grid, block, 0, st>>>(f, n, m, pf, c, c2, pc);
}

template <typename T>
void launch_interp_add(const LevelView<T> &Lf, const LevelView<T> &Lc, cudaStream_t st) {
    dim3 grid((Lf.m + 31) / 32, (Lf.n + 7) / 8), block(32, 8);
    k_interp_add<T><<<grid, block, 0, st>>>(Lf, Lc);
}

constexpr size_t kCoarseSmemMax = 200 * 1024;

void prepare_coarse_kernels() {
    cudaFuncSetAttribute(k_coarse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemMax);
    cudaFuncSetAttribute(k_coarse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemMax);
}

template <typename T>
void launch_coarse_solve(const LevelView<T> &L, const double *, ModelParams mp, double A1frac,
                         double h2nm, int maxit, double tol, double *scratch, Scalars *sc,
                         cudaStream_t st) {
    size_t bytes = coarse_scratch_doubles(L.n, L.m) * sizeof(double);
    if (bytes <= kCoarseSmemMax)
        k_coarse<T><<<1, 256, bytes, st>>>(L, mp, A1frac, h2nm, maxit, tol, nullptr, sc);
    else
        k_coarse<T><<<1, 256, 0, st>>>(L, mp, A1frac, h2nm, maxit, tol, scratch, sc);
}

#define INST(T)                                                                                    \
    template void launch_residual<T>(const LevelView<T> &, const T *, const double *, T *, int,    \
                                     double *, int, double *, cudaStream_t);                       \
    template void launch_restrict<T>(const T *, int, int, int, T *, T *, int, cudaStream_t);       \
    template void launch_interp_add<T>(const LevelView<T> &, const LevelView<T> &, cudaStream_t);  \
    template void launch_coarse_solve<T>(const LevelView<T> &, const double *, ModelParams, double, \
                                         double, int, double, double *, Scalars *, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace segmg
