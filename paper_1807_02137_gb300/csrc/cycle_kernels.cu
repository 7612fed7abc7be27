// cycle_kernels.cu -- residual, grid transfers and the coarsest solve of the FAS V-cycle
// (Sec. 3.1, Algorithm 1).
#include "arith.cuh"
#include "coarse_body.cuh"
#include "reduce.cuh"

namespace segmg {

namespace {

// ---------------------------------------------------------------------------------------
// Residual of L (the row-scaled operator of one pseudo-time step) on 32 x 32 tiles:
//   L(phi) = mu/h^2 sum_X G_X ((pn_X - pn) + (u_X - u)) - F - area - u / tau,
// mode 0: out = rhs - L(pn + uin) and, if partials is not NULL, a per-block FP64 partial of
// sum out^2;
// mode 1: out += L(pn + uin)   (the FAS right-hand side f^{2h} = N^{2h} phi^{2h} + r^{2h}).
// ---------------------------------------------------------------------------------------
// MINB > 1 asks the compiler for that many resident blocks per SM (FP32, fewer registers): used
// when it lets every tile of the grid be resident at once (a 1024^2 grid)
template <typename T, int MINB = 1>
__global__ void __launch_bounds__(256, MINB)
    k_residual(LevelView<T> L, const T *uin, const double *area, T *out, int mode, double *partials) {
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
        const size_t lim = (size_t)n * p;
        T Fv = kStage ? sF[kStage ? ti : 0][kStage ? tj : 0] : ldc(L.F, o, lim, kDbgResidual);
        T Lv = sub_rn(fma_rn(L.cdiff, fl, -add_rn(Fv, ar)), mul_rn(L.inv_tau, uc));
        if (mode == 0) {
            T r = L.has_rhs ? sub_rn(ldc(L.rhs, o, lim, kDbgResidual), Lv) : -Lv;
            stc(out, o, lim, kDbgResidual, r);
            acc = add_square(acc, r);
        } else {
            stc(out, o, lim, kDbgResidual, add_rn(ldc(out, o, lim, kDbgResidual), Lv));
        }
    }
    if (mode == 0 && partials) {
        double s = block_sum_warps(acc, red);
        if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// Loads the window dst[a][b] = src[clamp(r0 + a)][clamp(c0 + b)], a < ROWS, b < COLS, of one or
// two pitched FP32 grid functions (indices clamped into the grid: the mirror ghosts), with
// 16-byte vector loads where the window lies inside; c0 mod 4 == OFF.  NT threads.
template <int ROWS, int COLS, int OFF, int NT>
__device__ __forceinline__ void load_window(float (*dA)[COLS + 1], const float *sA, float (*dB)[COLS + 1],
                                            const float *sB, int r0, int c0, int n, int m, int p, int tid) {
    constexpr int NV = (COLS + OFF + 3) / 4, NVEC = ROWS * NV;
    for (int q = tid; q < NVEC; q += NT) {
        const int a = q / NV, k = q % NV, gi = r0 + a, gj = c0 - OFF + 4 * k;
        float xa[4], xb[4];
        if (gi >= 0 && gi < n && gj >= 0 && gj + 4 <= m && MG_DBG_OK((size_t)gi * p + gj + 3, (size_t)n * p, kDbgHaloLoad)) {
            const size_t o = (size_t)gi * p + gj;
            const float4 va = __ldg(reinterpret_cast<const float4 *>(sA + o));
            xa[0] = va.x; xa[1] = va.y; xa[2] = va.z; xa[3] = va.w;
            if (sB) {
                const float4 vb = __ldg(reinterpret_cast<const float4 *>(sB + o));
                xb[0] = vb.x; xb[1] = vb.y; xb[2] = vb.z; xb[3] = vb.w;
            }
        } else {
            const size_t ro = (size_t)clamp_idx(gi, n - 1) * p;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const size_t o = ro + clamp_idx(gj + e, m - 1);
                xa[e] = ldc(sA, o, (size_t)n * p, kDbgHaloLoad);
                if (sB) xb[e] = ldc(sB, o, (size_t)n * p, kDbgHaloLoad);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int b = 4 * k - OFF + e;
            if (b >= 0 && b < COLS) {
                dA[a][b] = xa[e];
                if (sB) dB[a][b] = xb[e];
            }
        }
    }
}

// The end of a pre-smoothing on an FP32 grid in one kernel: the residual r = rhs - L(pn + u)
// (the arithmetic of k_residual, mode 0) on the 32 x 32 fine tile plus one row and column,
// then the full weighting of r and of u onto the 16 x 16 coarse cells of the tile (the
// arithmetic of k_restrict): coarse rhs, u and u0.  r itself is not stored.
struct ResRestrictSmem {
    float P[37][38], U[37][38], W[37][38];   // rows i0-2 .. i0+34, columns j0-2 .. j0+34
    float G[35][36];                         // rows i0-1 .. i0+33
    float F[33][34], RH[33][34];             // rows i0 .. i0+32
    float R[33][34];
};

__global__ void __launch_bounds__(256) k_residual_restrict(LevelView<float> L, LevelView<float> C, const double *area) {
    extern __shared__ __align__(16) unsigned char smem_rr[];
    ResRestrictSmem &S = *reinterpret_cast<ResRestrictSmem *>(smem_rr);
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, tid = threadIdx.y * 32 + threadIdx.x;
    const int n = L.n, m = L.m, p = L.pitch;
    load_window<37, 37, 2, 256>(S.P, L.pn, S.U, L.u, i0 - 2, j0 - 2, n, m, p, tid);
    if (!L.wb) load_window<37, 37, 2, 256>(S.W, L.w, nullptr, nullptr, i0 - 2, j0 - 2, n, m, p, tid);
    load_window<33, 33, 0, 256>(S.F, L.F, L.has_rhs ? S.RH : nullptr, L.has_rhs ? L.rhs : nullptr, i0, j0, n, m, p,
                                tid);
    __syncthreads();
    for (int q = tid; q < 35 * 35; q += 256) {
        const int a = q / 35, b = q % 35, gi = i0 - 1 + a, gj = j0 - 1 + b;
        float g = 0.f;
        if (gi >= 0 && gi < n && gj >= 0 && gj < m) {
            const int A = a + 1, B = b + 1;
            const float w = L.wb ? weight_at(L, (size_t)gi * p + gj) : S.W[A][B];
            g = cell_G(w, S.P[A + 1][B], S.P[A - 1][B], S.P[A][B + 1], S.P[A][B - 1], S.U[A + 1][B], S.U[A - 1][B],
                       S.U[A][B + 1], S.U[A][B - 1], L.inv_2h, L.beta);
        }
        S.G[a][b] = g;
    }
    __syncthreads();
    const float ar = area ? float(area[L.level]) : 0.f;
    for (int q = tid; q < 33 * 33; q += 256) {
        const int ti = q / 33, tj = q % 33, gi = i0 + ti, gj = j0 + tj;
        float r = 0.f;
        if (gi < n && gj < m) {
            const int a = ti + 1, b = tj + 1;        // in G
            const int A = ti + 2, B = tj + 2;        // in P, U
            const bool hS = gi + 1 < n, hN = gi > 0, hE = gj + 1 < m, hW = gj > 0;
            const float gc = S.G[a][b];
            const float aS = face(gc, S.G[a + 1][b], hS), aN = face(gc, S.G[a - 1][b], hN);
            const float aE = face(gc, S.G[a][b + 1], hE), aW = face(gc, S.G[a][b - 1], hW);
            const float pc = S.P[A][B], uc = S.U[A][B];
            float fl = mul_rn(aS, add_rn(sub_rn(S.P[A + 1][B], pc), sub_rn(S.U[A + 1][B], uc)));
            fl = fma_rn(aN, add_rn(sub_rn(S.P[A - 1][B], pc), sub_rn(S.U[A - 1][B], uc)), fl);
            fl = fma_rn(aE, add_rn(sub_rn(S.P[A][B + 1], pc), sub_rn(S.U[A][B + 1], uc)), fl);
            fl = fma_rn(aW, add_rn(sub_rn(S.P[A][B - 1], pc), sub_rn(S.U[A][B - 1], uc)), fl);
            const float Lv = sub_rn(fma_rn(L.cdiff, fl, -add_rn(S.F[ti][tj], ar)), mul_rn(L.inv_tau, uc));
            r = L.has_rhs ? sub_rn(S.RH[ti][tj], Lv) : -Lv;
        }
        S.R[ti][tj] = r;
    }
    __syncthreads();
    // full weighting onto the coarse cells of this tile: one thread per coarse cell
    {
        const int I = blockIdx.y * 16 + tid / 16, J = blockIdx.x * 16 + tid % 16;
        if (I < C.n && J < C.m) {
            int ri[3], ci[3];
            float rw[3], cw[3];
            const int nr = fw_taps(I, n, ri, rw), nk = fw_taps(J, m, ci, cw);
            float sr = 0.f, su = 0.f;
            for (int a = 0; a < nr; ++a) {
                float rowr = 0.f, rowu = 0.f;
                for (int b = 0; b < nk; ++b) {
                    if (!MG_DBG_OK(ri[a] - i0, 33, kDbgResidual) || !MG_DBG_OK(ci[b] - j0, 33, kDbgResidual)) continue;
                    rowr = fma_rn(float(cw[b]), S.R[ri[a] - i0][ci[b] - j0], rowr);
                    rowu = fma_rn(float(cw[b]), S.U[ri[a] - i0 + 2][ci[b] - j0 + 2], rowu);
                }
                sr = fma_rn(float(rw[a]), rowr, sr);
                su = fma_rn(float(rw[a]), rowu, su);
            }
            const size_t o = (size_t)I * C.pitch + J, lc = (size_t)C.n * C.pitch;
            stc(C.rhs, o, lc, kDbgResidual, sr);
            stc(C.u, o, lc, kDbgResidual, su);
            stc(C.u0, o, lc, kDbgResidual, su);
        }
    }
}

// stage[k * gridDim.x + b] = sum of chunk b of the k-th array of np partials (blockIdx.y = k).
__global__ void __launch_bounds__(256) k_chunk_sums(const double *part, int np, double *stage) {
    __shared__ double red[33];
    const int b = blockIdx.x, k = blockIdx.y;
    const double s = chunk_sum(part + (size_t)k * np, b * kSumChunk, min(np, (b + 1) * kSumChunk), red);
    if (threadIdx.x == 0) stage[(size_t)k * gridDim.x + b] = s;
}

// Sums `np` partials in a fixed order into *out (one block).
__global__ void __launch_bounds__(256) k_sum_partials(const double *partials, int np, double *out) {
    __shared__ double red[33];
    const double s = chunk_sum(partials, 0, np, red);
    if (threadIdx.x == 0) *out = s;
}

// Full weighting of up to three fields of one grid in one launch (blockIdx.z picks the field).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(RestrictFields<T> F, int n, int m, int pf, int pc) {
    const int J = blockIdx.x * 32 + threadIdx.x, I = blockIdx.y * 8 + threadIdx.y;
    const int nc = n / 2, mc = m / 2;
    if (I >= nc || J >= mc) return;
    const T *f = F.f[blockIdx.z];
    T *c = F.c[blockIdx.z], *c2 = F.c2[blockIdx.z];
    int ri[3], ci[3];
    float rw[3], cw[3];
    int nr = fw_taps(I, n, ri, rw), nk = fw_taps(J, m, ci, cw);
    T s = T(0);
    for (int a = 0; a < nr; ++a) {
        T row = T(0);
        for (int b = 0; b < nk; ++b)
            row = fma_rn(T(cw[b]), ldc(f, (size_t)ri[a] * pf + ci[b], (size_t)n * pf, kDbgResidual), row);
        s = fma_rn(T(rw[a]), row, s);
    }
    stc(c, (size_t)I * pc + J, (size_t)nc * pc, kDbgResidual, s);
    if (c2) stc(c2, (size_t)I * pc + J, (size_t)nc * pc, kDbgResidual, s);
}

// Interpolation and correction: u_f += P (u_c - u0_c)  (Algorithm 1, "Interpolation").
template <typename T>
__global__ void __launch_bounds__(256) k_interp_add(LevelView<T> Lf, LevelView<T> Lc) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i >= Lf.n || j >= Lf.m) return;
    int ri[2], ci[2];
    float rw[2], cw[2];
    int nr = bl_taps(i, Lc.n, ri, rw), nk = bl_taps(j, Lc.m, ci, cw);
    T s = T(0);
    for (int a = 0; a < nr; ++a)
        for (int b = 0; b < nk; ++b) {
            size_t o = (size_t)ri[a] * Lc.pitch + ci[b], lc = (size_t)Lc.n * Lc.pitch;
            s = fma_rn(T(rw[a] * cw[b]), sub_rn(ldc(Lc.u, o, lc, kDbgInterp), ldc(Lc.u0, o, lc, kDbgInterp)), s);
        }
    size_t o = (size_t)i * Lf.pitch + j;
    stc(Lf.u, o, (size_t)Lf.n * Lf.pitch, kDbgInterp, add_rn(Lf.u[o], s));
}

// The coarsest solve (coarse_body.cuh) as its own one-block kernel.
template <typename T, typename C>
__global__ void __launch_bounds__(kCoarseThreads) k_coarse(LevelView<T> L, ModelParams mp, double A1frac,
                                                           double h2nm, int maxit, double tol, C *scratch,
                                                           Scalars *sc, int aos, double aos_dt) {
    extern __shared__ __align__(16) unsigned char smem_coarse[];
    if (!scratch) scratch = reinterpret_cast<C *>(smem_coarse);   // small grids: all in shared memory
    __shared__ double red[33];
    __shared__ int s_err;
    CoarseGrid<T> g{L.n, L.m, L.pitch, L.pn, L.u, L.w, L.wb, L.F, L.rhs, L.has_rhs, L.inv_2h, L.inv_tau, L.beta};
    int it;
    double res;
    (void)A1frac;   // the area of the initial contour is read from the device scalars (set by each reset,
                    // so a captured graph stays valid across resets)
    coarse_solve_block<T, C>(g, mp, sc->A1frac, h2nm, maxit, tol, scratch, red, &s_err, &it, &res, aos, aos_dt);
    if (threadIdx.x == 0) {
        sc->picard = it;
        sc->coarse_res = res;
        if (s_err) sc->err = 1;
    }
}

}  // namespace

int num_partials(int n, int m) { return ((m + 31) / 32) * ((n + 31) / 32); }


// Resident blocks per SM of the FP32 residual held to 8 blocks per SM, and the SM count
// (measured once at set-up, outside any capture).
struct ResOcc {
    int per_sm = 0, sms = 1;
    ResOcc() {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_residual<float, 8>, 256, 0) != cudaSuccess)
            per_sm = 0;
    }
};
const ResOcc &res_occ() {
    static const ResOcc o;
    return o;
}

template <typename T>
void launch_residual(const LevelView<T> &L, const T *uin, const double *area, T *out, int mode,
                     double *partials, int npart, double *norm_out, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32), block(32, 8);
    // the per-block partial sums (FP64, slow on this GPU) only when the norm is wanted; the
    // register-limited FP32 variant when it makes every tile resident at once (same operations,
    // same order)
    const ResOcc &o = res_occ();
    if (sizeof(T) == 4 && (long)grid.x * grid.y <= (long)o.sms * o.per_sm)
        k_residual<T, sizeof(T) == 4 ? 8 : 1><<<grid, block, 0, st>>>(L, uin, area, out, mode,
                                                                      norm_out ? partials : nullptr);
    else
        k_residual<T><<<grid, block, 0, st>>>(L, uin, area, out, mode, norm_out ? partials : nullptr);
    if (mode == 0 && norm_out) launch_sum_partials(partials, npart, norm_out, st);
}

template <typename T>
void launch_restrict(const T *f, int n, int m, int pf, T *c, T *c2, int pc, cudaStream_t st) {
    RestrictFields<T> F{};
    F.f[0] = f; F.c[0] = c; F.c2[0] = c2; F.nf = 1;
    launch_restrict_fields(F, n, m, pf, pc, st);
}

template <typename T>
void launch_restrict_fields(const RestrictFields<T> &F, int n, int m, int pf, int pc, cudaStream_t st) {
    dim3 grid((m / 2 + 31) / 32, (n / 2 + 7) / 8, F.nf), block(32, 8);
    k_restrict<T><<<grid, block, 0, st>>>(F, n, m, pf, pc);
}

template <typename T>
void launch_interp_add(const LevelView<T> &Lf, const LevelView<T> &Lc, cudaStream_t st) {
    dim3 grid((Lf.m + 31) / 32, (Lf.n + 7) / 8), block(32, 8);
    k_interp_add<T><<<grid, block, 0, st>>>(Lf, Lc);
}

constexpr size_t kCoarseSmemMax = 200 * 1024;

void launch_chunk_sums(const double *part, int np, int K, double *stage, cudaStream_t st) {
    k_chunk_sums<<<dim3(sum_blocks(np), K), 256, 0, st>>>(part, np, stage);
}

void launch_sum_partials(double *partials, int np, double *out, cudaStream_t st) {
    const int G = sum_blocks(np);
    if (G == 1) {
        k_sum_partials<<<1, 256, 0, st>>>(partials, np, out);
    } else {   // the chunk sums go to the G doubles after the partials
        launch_chunk_sums(partials, np, 1, partials + np, st);
        k_sum_partials<<<1, 256, 0, st>>>(partials + np, G, out);
    }
}

void launch_residual_restrict(const LevelView<float> &L, const LevelView<float> &C, const double *area,
                              cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32), block(32, 8);
    k_residual_restrict<<<grid, block, sizeof(ResRestrictSmem), st>>>(L, C, area);
}

void prepare_coarse_kernels() {
    (void)res_occ();
    cudaFuncSetAttribute(k_residual_restrict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ResRestrictSmem));
    cudaFuncSetAttribute(k_coarse<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemMax);
    cudaFuncSetAttribute(k_coarse<float, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemMax);
    cudaFuncSetAttribute(k_coarse<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemMax);
}

template <typename T, typename C>
static void coarse_launch(const LevelView<T> &L, ModelParams mp, double A1frac, double h2nm, int maxit,
                          double tol, double *scratch, Scalars *sc, int aos, double aos_dt, cudaStream_t st) {
    size_t bytes = coarse_scratch_elems(L.n, L.m) * sizeof(C);
    if (bytes <= kCoarseSmemMax)
        k_coarse<T, C><<<1, kCoarseThreads, bytes, st>>>(L, mp, A1frac, h2nm, maxit, tol, nullptr, sc, aos, aos_dt);
    else
        k_coarse<T, C><<<1, kCoarseThreads, 0, st>>>(L, mp, A1frac, h2nm, maxit, tol, reinterpret_cast<C *>(scratch),
                                                     sc, aos, aos_dt);
}

template <typename T>
void launch_coarse_solve(const LevelView<T> &L, int fp64, ModelParams mp, double A1frac,
                         double h2nm, int maxit, double tol, double *scratch, Scalars *sc,
                         int aos, double aos_dt, cudaStream_t st) {
    if (sizeof(T) == 8 || fp64) coarse_launch<T, double>(L, mp, A1frac, h2nm, maxit, tol, scratch, sc, aos, aos_dt, st);
    else coarse_launch<T, float>(L, mp, A1frac, h2nm, maxit, tol, scratch, sc, aos, aos_dt, st);
}

#define INST(T)                                                                                    \
    template void launch_residual<T>(const LevelView<T> &, const T *, const double *, T *, int,    \
                                     double *, int, double *, cudaStream_t);                       \
    template void launch_restrict<T>(const T *, int, int, int, T *, T *, int, cudaStream_t);       \
    template void launch_restrict_fields<T>(const RestrictFields<T> &, int, int, int, int, cudaStream_t); \
    template void launch_interp_add<T>(const LevelView<T> &, const LevelView<T> &, cudaStream_t);  \
    template void launch_coarse_solve<T>(const LevelView<T> &, int, ModelParams, double,            \
                                         double, int, double, double *, Scalars *, int, double,     \
                                         cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace segmg
