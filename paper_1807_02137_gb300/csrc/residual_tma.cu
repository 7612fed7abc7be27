// residual_tma.cu -- the residual kernels of the V-cycle (Algorithm 1: r = f - N(phi), the FAS
// right-hand side f^{2h} = N^{2h}(phi^{2h}) + R r, the full weighting of Sec. 3.1) for FP32
// storage, with their inputs staged into shared memory by the Tensor Memory Accelerator.
//
// Same per-cell operations, in the same order, as k_residual and k_residual_restrict in
// cycle_kernels.cu (the results are bitwise identical, the partial sums of the norm included:
// 256 threads per 32 x 32 tile, each thread owning the cells of one column in rows wy, wy + 8,
// ...); the work around them changes as in snapshot_tma.cu: one thread copies the pn, u (or u0)
// and w boxes and the F and rhs (or output) tiles, edge tiles mirror-clamp their ghost cells, and
// tiles whose stencil lies inside the grid run without per-cell bounds tests.  The one mbarrier
// wait is bounded (wait_limit try_wait rounds); on time-out the block records bit 4 in the
// handle's error word, drains and returns.
#include <cuda.h>

#include <type_traits>

#include "arith.cuh"
#include "reduce.cuh"
#include "tma.cuh"

namespace segmg {

namespace {

constexpr int kC = 40, kCb = 48;   // FP32 / BF16 box columns (from j0-4 / j0-8)
// resident blocks per SM asked of the compiler: 8 x 256 threads at most 32 registers (the
// residual's FP32 shared memory, 26 KB, fits 8 blocks); 6 for the residual with restriction
constexpr int kResMinB = 8, kRRMinB = 6;
constexpr long long kResDrain = 1LL << 22;

// ---------------------------------------------------------------------------------------
// r = rhs - L(pn + uin) and its per-tile sum of squares (MODE 0), or out += L(pn + uin) (MODE 1)
// ---------------------------------------------------------------------------------------
template <bool MIXED>
struct ResTmaSmem {
    alignas(128) float P[36][kC];
    alignas(128) float U[36][kC];
    alignas(128) float W[36][kC];   // FP32: w, overwritten in place by G (a cell reads only its own w)
    alignas(128) __nv_bfloat16 Wb[MIXED ? 36 : 1][kCb];   // mixed precision: w; G is then in W
    alignas(128) float F[32][32];
    alignas(128) float X[32][32];   // MODE 0: rhs; MODE 1: the output's values before the update
    double red[33];
    unsigned long long bar;
};

template <int MODE, bool MIXED, bool NORM, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_residual_tma(LevelView<float> L, const double *area, float *out, double *partials,
                   const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mU,
                   const __grid_constant__ CUtensorMap mW, const __grid_constant__ CUtensorMap mF,
                   const __grid_constant__ CUtensorMap mX, int *err, long long wait_limit) {
    using T = float;
    using Smem = ResTmaSmem<MIXED>;
    extern __shared__ unsigned char smem_res[];
    Smem &S = *reinterpret_cast<Smem *>(smem_res + ((128 - (smem_u32(smem_res) & 127)) & 127));
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32 + lane;
    const int n = L.n, m = L.m, p = L.pitch;
    const bool hasX = MODE == 1 || L.has_rhs;
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        fence_proxy_async();
        const unsigned wbytes = MIXED ? 36u * kCb * 2u : 36u * kC * 4u;
        mbar_expect_tx(&S.bar, 2u * 36u * kC * 4u + wbytes + 4096u + (hasX ? 4096u : 0u));
        tma_load(&S.P[0][0], &mP, j0 - 4, i0 - 2, &S.bar);
        tma_load(&S.U[0][0], &mU, j0 - 4, i0 - 2, &S.bar);
        if (MIXED) tma_load(&S.Wb[0][0], &mW, j0 - 8, i0 - 2, &S.bar);
        else tma_load(&S.W[0][0], &mW, j0 - 4, i0 - 2, &S.bar);
        tma_load(&S.F[0][0], &mF, j0, i0, &S.bar);
        if (hasX) tma_load(&S.X[0][0], &mX, j0, i0, &S.bar);
    }
    __syncthreads();
    bool ok = true;
    if (wy == 0) ok = mbar_wait(&S.bar, 0, wait_limit);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicOr(err, 4);
            mbar_wait(&S.bar, 0, kResDrain);
        }
        __syncthreads();
        return;
    }
    if (i0 < 2 || j0 < 4 || i0 + 34 > n || j0 + 36 > m) {   // mirror ghosts of pn and uin
        for (int q = tid; q < 36 * kC; q += 256) {
            const int a = q / kC, c = q - a * kC, gi = i0 - 2 + a, gj = j0 - 4 + c;
            const int ci = clamp_idx(gi, n - 1), cj = clamp_idx(gj, m - 1);
            if (ci != gi || cj != gj) {
                S.P[a][c] = S.P[ci - (i0 - 2)][cj - (j0 - 4)];
                S.U[a][c] = S.U[ci - (i0 - 2)][cj - (j0 - 4)];
            }
        }
        __syncthreads();
    }
    const bool interior = i0 >= 1 && j0 >= 1 && i0 + 33 <= n && j0 + 33 <= m;
    auto g_at = [&](int a, int c, bool check) {
        const int gi = i0 - 2 + a, gj = j0 - 4 + c;
        T g = T(0);
        if (!check || (gi >= 0 && gi < n && gj >= 0 && gj < m)) {
            const T w = MIXED ? __bfloat162float(S.Wb[MIXED ? a : 0][c + 4]) : S.W[a][c];
            g = cell_G(w, S.P[a + 1][c], S.P[a - 1][c], S.P[a][c + 1], S.P[a][c - 1], S.U[a + 1][c], S.U[a - 1][c],
                       S.U[a][c + 1], S.U[a][c - 1], L.inv_2h, L.beta);
        }
        S.W[a][c] = g;
    };
    if (interior) {
#pragma unroll
        for (int k = 0; k < 4; ++k) g_at(1 + wy + 8 * k, lane + 4, false);
        if (wy < 2) g_at(33 + wy, lane + 4, false);
        if (tid < 68) g_at(1 + (tid >> 1), (tid & 1) ? 36 : 3, false);
    } else {
        for (int a = 1 + wy; a <= 34; a += 8) g_at(a, lane + 4, true);
        if (tid < 68) g_at(1 + (tid >> 1), (tid & 1) ? 36 : 3, true);
    }
    __syncthreads();
    const T ar = area ? T(area[L.level]) : T(0);
    const T c2 = L.cdiff * T(0.5);
    const int gj = j0 + lane, c = lane + 4;
    const size_t lim = (size_t)n * p;
    T acc = T(0);
    auto cell = [&](int k, auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;
        const int ti = wy + 8 * k, a = ti + 2, gi = i0 + ti;
        if (!(IN || (gi < n && gj < m))) return;
        const bool hS = IN || gi + 1 < n, hN = IN || gi > 0, hE = IN || gj + 1 < m, hW = IN || gj > 0;
        const T gc = S.W[a][c];
        const T aS = face2(gc, S.W[a + 1][c], hS), aN = face2(gc, S.W[a - 1][c], hN);   // with c2 (arith.cuh)
        const T aE = face2(gc, S.W[a][c + 1], hE), aW = face2(gc, S.W[a][c - 1], hW);
        const T pc = S.P[a][c], uc = S.U[a][c];
        T fl = mul_rn(aS, add_rn(sub_rn(S.P[a + 1][c], pc), sub_rn(S.U[a + 1][c], uc)));
        fl = fma_rn(aN, add_rn(sub_rn(S.P[a - 1][c], pc), sub_rn(S.U[a - 1][c], uc)), fl);
        fl = fma_rn(aE, add_rn(sub_rn(S.P[a][c + 1], pc), sub_rn(S.U[a][c + 1], uc)), fl);
        fl = fma_rn(aW, add_rn(sub_rn(S.P[a][c - 1], pc), sub_rn(S.U[a][c - 1], uc)), fl);
        const T Lv = sub_rn(fma_rn(c2, fl, -add_rn(S.F[ti][lane], ar)), mul_rn(L.inv_tau, uc));
        const size_t o = (size_t)gi * p + gj;
        if (MODE == 0) {
            const T r = L.has_rhs ? sub_rn(S.X[ti][lane], Lv) : -Lv;
            if (out) stc(out, o, lim, kDbgResidual, r);
            acc = add_square(acc, r);
        } else {
            stc(out, o, lim, kDbgResidual, add_rn(S.X[ti][lane], Lv));
        }
    };
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (interior) cell(k, std::true_type{});
        else cell(k, std::false_type{});
    }
    if (NORM) {
        const double s = block_sum_warps(acc, S.red);
        if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------------------
// The end of a pre-smoothing: r = rhs - L(pn + u) on the tile plus one row and column, then the
// full weighting of r and u onto the tile's 16 x 16 coarse cells (rhs, u, u0 of the coarse grid)
// ---------------------------------------------------------------------------------------
template <bool MIXED>
struct RRTmaSmem {
    alignas(128) float P[37][kC];   // rows i0-2 .. i0+34, columns j0-4 .. j0+35
    alignas(128) float U[37][kC];
    alignas(128) float W[37][kC];   // FP32: w, overwritten in place by G; mixed: G
    alignas(128) __nv_bfloat16 Wb[MIXED ? 37 : 1][kCb];
    alignas(128) float F[33][36];   // rows i0 .. i0+32, columns j0 .. j0+35
    alignas(128) float RH[33][36];
    float R[33][34];
    unsigned long long bar;
};

template <bool MIXED, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_residual_restrict_tma(LevelView<float> L, LevelView<float> C, const double *area,
                            const __grid_constant__ CUtensorMap mP, const __grid_constant__ CUtensorMap mU,
                            const __grid_constant__ CUtensorMap mW, const __grid_constant__ CUtensorMap mF,
                            const __grid_constant__ CUtensorMap mR, int *err, long long wait_limit) {
    using Smem = RRTmaSmem<MIXED>;
    extern __shared__ unsigned char smem_rr2[];
    Smem &S = *reinterpret_cast<Smem *>(smem_rr2 + ((128 - (smem_u32(smem_rr2) & 127)) & 127));
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32 + lane;
    const int n = L.n, m = L.m;
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        fence_proxy_async();
        const unsigned wbytes = MIXED ? 37u * kCb * 2u : 37u * kC * 4u;
        mbar_expect_tx(&S.bar, 2u * 37u * kC * 4u + wbytes + 33u * 36u * 4u * (L.has_rhs ? 2u : 1u));
        tma_load(&S.P[0][0], &mP, j0 - 4, i0 - 2, &S.bar);
        tma_load(&S.U[0][0], &mU, j0 - 4, i0 - 2, &S.bar);
        if (MIXED) tma_load(&S.Wb[0][0], &mW, j0 - 8, i0 - 2, &S.bar);
        else tma_load(&S.W[0][0], &mW, j0 - 4, i0 - 2, &S.bar);
        tma_load(&S.F[0][0], &mF, j0, i0, &S.bar);
        if (L.has_rhs) tma_load(&S.RH[0][0], &mR, j0, i0, &S.bar);
    }
    __syncthreads();
    bool ok = true;
    if (wy == 0) ok = mbar_wait(&S.bar, 0, wait_limit);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicOr(err, 4);
            mbar_wait(&S.bar, 0, kResDrain);
        }
        __syncthreads();
        return;
    }
    if (i0 < 2 || j0 < 4 || i0 + 35 > n || j0 + 36 > m) {   // mirror ghosts of pn and u
        for (int q = tid; q < 37 * kC; q += 256) {
            const int a = q / kC, c = q - a * kC, gi = i0 - 2 + a, gj = j0 - 4 + c;
            const int ci = clamp_idx(gi, n - 1), cj = clamp_idx(gj, m - 1);
            if (ci != gi || cj != gj) {
                S.P[a][c] = S.P[ci - (i0 - 2)][cj - (j0 - 4)];
                S.U[a][c] = S.U[ci - (i0 - 2)][cj - (j0 - 4)];
            }
        }
        __syncthreads();
    }
    // G on rows i0-1 .. i0+33 and columns j0-1 .. j0+33 (box rows 1..35, columns 3..37)
    const bool gin = i0 >= 1 && j0 >= 1 && i0 + 34 <= n && j0 + 34 <= m;
    auto g_at = [&](int a, int c, bool check) {
        const int gi = i0 - 2 + a, gj = j0 - 4 + c;
        float g = 0.f;
        if (!check || (gi >= 0 && gi < n && gj >= 0 && gj < m)) {
            const float w = MIXED ? __bfloat162float(S.Wb[MIXED ? a : 0][c + 4]) : S.W[a][c];
            g = cell_G(w, S.P[a + 1][c], S.P[a - 1][c], S.P[a][c + 1], S.P[a][c - 1], S.U[a + 1][c], S.U[a - 1][c],
                       S.U[a][c + 1], S.U[a][c - 1], L.inv_2h, L.beta);
        }
        S.W[a][c] = g;
    };
    if (gin) {
#pragma unroll
        for (int k = 0; k < 4; ++k) g_at(1 + wy + 8 * k, lane + 3, false);
        if (wy < 3) g_at(33 + wy, lane + 3, false);
        if (tid < 105) g_at(1 + tid / 3, 35 + tid % 3, false);
    } else {
        for (int a = 1 + wy; a <= 35; a += 8) g_at(a, lane + 3, true);
        if (tid < 105) g_at(1 + tid / 3, 35 + tid % 3, true);
    }
    __syncthreads();
    // r on rows i0 .. i0+32, columns j0 .. j0+32 (zero outside the grid)
    const float ar = area ? float(area[L.level]) : 0.f;
    const float c2 = L.cdiff * 0.5f;
    const bool rin = gin;   // every r cell has its four faces and its G ring inside the grid
    auto r_at = [&](int ti, int tj, auto in_tag) {
        constexpr bool IN = decltype(in_tag)::value;
        const int gi = i0 + ti, gj = j0 + tj;
        float r = 0.f;
        if (IN || (gi < n && gj < m)) {
            const int a = ti + 2, c = tj + 4;   // box coordinates
            const bool hS = IN || gi + 1 < n, hN = IN || gi > 0, hE = IN || gj + 1 < m, hW = IN || gj > 0;
            const float gc = S.W[a][c];
            const float aS = face2(gc, S.W[a + 1][c], hS), aN = face2(gc, S.W[a - 1][c], hN);   // with c2
            const float aE = face2(gc, S.W[a][c + 1], hE), aW = face2(gc, S.W[a][c - 1], hW);
            const float pc = S.P[a][c], uc = S.U[a][c];
            float fl = mul_rn(aS, add_rn(sub_rn(S.P[a + 1][c], pc), sub_rn(S.U[a + 1][c], uc)));
            fl = fma_rn(aN, add_rn(sub_rn(S.P[a - 1][c], pc), sub_rn(S.U[a - 1][c], uc)), fl);
            fl = fma_rn(aE, add_rn(sub_rn(S.P[a][c + 1], pc), sub_rn(S.U[a][c + 1], uc)), fl);
            fl = fma_rn(aW, add_rn(sub_rn(S.P[a][c - 1], pc), sub_rn(S.U[a][c - 1], uc)), fl);
            const float Lv = sub_rn(fma_rn(c2, fl, -add_rn(S.F[ti][tj], ar)), mul_rn(L.inv_tau, uc));
            r = L.has_rhs ? sub_rn(S.RH[ti][tj], Lv) : -Lv;
        }
        S.R[ti][tj] = r;
    };
    if (rin) {
#pragma unroll
        for (int k = 0; k < 4; ++k) r_at(wy + 8 * k, lane, std::true_type{});
        if (wy == 0) r_at(32, lane, std::true_type{});
        if (tid < 33) r_at(tid, 32, std::true_type{});
    } else {
        for (int ti = wy; ti < 33; ti += 8) r_at(ti, lane, std::false_type{});
        if (tid < 33) r_at(tid, 32, std::false_type{});
    }
    __syncthreads();
    // full weighting onto the coarse cells of this tile: one thread per coarse cell
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
                rowu = fma_rn(float(cw[b]), S.U[ri[a] - i0 + 2][ci[b] - j0 + 4], rowu);
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

template <int MODE, bool MIXED, bool NORM>
size_t res_smem() { return sizeof(ResTmaSmem<MIXED>) + 128; }
template <bool MIXED>
size_t rr_smem() { return sizeof(RRTmaSmem<MIXED>) + 128; }

template <int MODE, bool MIXED, bool NORM>
void res_attr() {
    cudaFuncSetAttribute(k_residual_tma<MODE, MIXED, NORM, kResMinB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)res_smem<MODE, MIXED, NORM>());
}

const CUtensorMap *tm(const unsigned char *b) { return reinterpret_cast<const CUtensorMap *>(b); }

template <int MODE, bool MIXED, bool NORM>
void launch_res(const LevelView<float> &L, const double *area, float *out, double *partials, const SnapMaps &M,
                const unsigned char *mU, const unsigned char *mX, int *err, long long wl, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32), block(32, 8);
    k_residual_tma<MODE, MIXED, NORM, kResMinB><<<grid, block, res_smem<MODE, MIXED, NORM>(), st>>>(
        L, area, out, partials, *tm(M.P), *tm(mU), *tm(M.W), *tm(M.F), *tm(mX), err, wl);
}

template <bool MIXED>
void launch_res_mixed(const LevelView<float> &L, int uin_is_u0, const double *area, float *out, int mode,
                      double *partials, const SnapMaps &M, const ResMaps &R, int *err, long long wl, cudaStream_t st) {
    const unsigned char *mU = uin_is_u0 ? R.U0 : M.U;
    if (mode == 1) launch_res<1, MIXED, false>(L, area, out, nullptr, M, mU, M.R, err, wl, st);
    else if (partials) launch_res<0, MIXED, true>(L, area, out, partials, M, mU, L.has_rhs ? M.R : M.F, err, wl, st);
    else launch_res<0, MIXED, false>(L, area, out, nullptr, M, mU, L.has_rhs ? M.R : M.F, err, wl, st);
}

}  // namespace

void prepare_residual_tma() {
    res_attr<0, false, false>(); res_attr<0, false, true>(); res_attr<1, false, false>();
    res_attr<0, true, false>(); res_attr<0, true, true>(); res_attr<1, true, false>();
    cudaFuncSetAttribute(k_residual_restrict_tma<false, kRRMinB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rr_smem<false>());
    cudaFuncSetAttribute(k_residual_restrict_tma<true, kRRMinB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rr_smem<true>());
}

bool encode_residual_maps(const LevelView<float> &L, ResMaps *R) {
    bool ok = encode_map_2d(R->P37, L.pn, 4, L.n, L.m, L.pitch, 37, kC) &&
              encode_map_2d(R->U37, L.u, 4, L.n, L.m, L.pitch, 37, kC) &&
              encode_map_2d(R->F33, L.F, 4, L.n, L.m, L.pitch, 33, 36);
    if (L.wb) ok = ok && encode_map_2d(R->W37, (void *)L.wb, 2, L.n, L.m, L.pitch, 37, kCb);
    else ok = ok && encode_map_2d(R->W37, L.w, 4, L.n, L.m, L.pitch, 37, kC);
    if (L.rhs) ok = ok && encode_map_2d(R->R33, L.rhs, 4, L.n, L.m, L.pitch, 33, 36);
    if (L.u0) ok = ok && encode_map_2d(R->U0, L.u0, 4, L.n, L.m, L.pitch, 36, kC);
    return ok;
}

void launch_residual_tma(const LevelView<float> &L, int uin_is_u0, const double *area, float *out, int mode,
                         double *partials, int npart, double *norm_out, const SnapMaps &M, const ResMaps &R, int *err,
                         long long wait_limit, cudaStream_t st) {
    double *parts = mode == 0 && norm_out ? partials : nullptr;
    if (M.mixed) launch_res_mixed<true>(L, uin_is_u0, area, out, mode, parts, M, R, err, wait_limit, st);
    else launch_res_mixed<false>(L, uin_is_u0, area, out, mode, parts, M, R, err, wait_limit, st);
    if (parts) launch_sum_partials(partials, npart, norm_out, st);
}

void launch_residual_restrict_tma(const LevelView<float> &L, const LevelView<float> &C, const double *area,
                                  const ResMaps &R, int *err, long long wait_limit, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32), block(32, 8);
    const unsigned char *mR = L.has_rhs ? R.R33 : R.F33;
    if (L.wb)
        k_residual_restrict_tma<true, kRRMinB><<<grid, block, rr_smem<true>(), st>>>(L, C, area, *tm(R.P37), *tm(R.U37),
                                                                           *tm(R.W37), *tm(R.F33), *tm(mR), err,
                                                                           wait_limit);
    else
        k_residual_restrict_tma<false, kRRMinB><<<grid, block, rr_smem<false>(), st>>>(L, C, area, *tm(R.P37), *tm(R.U37),
                                                                             *tm(R.W37), *tm(R.F33), *tm(mR), err,
                                                                             wait_limit);
}

}  // namespace segmg
