// snapshot_tma.cu -- the coefficient snapshot of Hybrid Smoother 2 (Sec. 4.3: the lagged
// coefficients G = w / |grad phi|_beta of eq. abcdrc, the right-hand side f of the frozen system,
// the jump set D of Sec. 4.1 and the partial-line member masks) for FP32 storage, with its inputs
// staged into shared memory by the Tensor Memory Accelerator.
//
// Same tiles and the same per-cell operations as k_snapshot in smooth_kernels.cu (the results
// are bitwise identical); what changes is the work around them:
//   - one thread copies the boxes of pn, u, w (rows i0-2 .. i0+33, columns j0-4 .. j0+35; BF16
//     w from column j0-8 in mixed precision) and the 32 x 32 tiles of F and rhs with five
//     cp.async.bulk.tensor loads completing on one mbarrier; only edge tiles then overwrite the
//     box cells outside the grid with the clamped cells' values (the mirror ghosts; the copy
//     fills them with zeros);
//   - tiles whose G ring lies inside the grid run a main loop without per-cell bounds tests;
//   - the column member masks are collected as per-thread bit words (one bit per row a thread
//     owns) ORed across the warps, instead of a byte transpose in shared memory.
// On the finest grid of an 8192^2 image this takes the kernel from about 270 to about 150
// thread instructions per cell.  The one wait on the mbarrier is bounded (wait_limit try_wait
// rounds); on time-out the block records bit 4 in the handle's error word, drains and returns.
#include <cuda.h>

#include <type_traits>

#include "arith.cuh"
#include "reduce.cuh"
#include "tma.cuh"

namespace segmg {

namespace {

constexpr int kBR = 36, kBC = 40, kBCb = 48;   // box rows; FP32 and BF16 box columns
// coarse rows and columns the box rows 0..35 and columns 2..37 interpolate from (fine i0-2 ..
// i0+33 take coarse i0/2-2 .. i0/2+16)
constexpr int kCR = 20;
constexpr long long kSnapDrain = 1LL << 22;

template <int WARPS, bool MIXED>
struct SnapTmaSmem {
    alignas(128) float P[kBR][kBC];
    alignas(128) float U[kBR][kBC];
    alignas(128) float W[kBR][kBC];   // FP32: w, overwritten in place by G (a cell reads only its own w)
    alignas(128) __nv_bfloat16 Wb[MIXED ? kBR : 1][kBCb];      // mixed precision: w (from column j0-8); G in W
    alignas(128) float F[32][32];
    alignas(128) float R[32][32];
    uint32_t cm[2][WARPS][32];   // column member bits of sweeps C, D per warp
    double red[33];              // NORM: the block's sum of squares
    float E[kCR][kCR + 1];       // interpolating snapshot: u_c - u0_c on the coarse cells used
    unsigned long long bar;
};

// One 32 x 32 tile per block of WARPS warps; thread (wy, lane) owns tile column lane, rows
// wy, wy + WARPS, ....  Box coordinates: row a = tile row + 2, column c = tile column + 4.
// NORM (8 warps): the block also writes sum r^2 of its tile, r = rhs - L(pn + u) at the state
// the snapshot reads, to partials[block]: the operations and the order of k_residual_tma's norm
// (the same G box, faces, flux and per-thread order), so the partials are bitwise its partials.
// XT = 1, FAS (the first snapshot of a coarse grid's pre-smoothing, right after the
// restriction, when u = u0 there): the block also completes the grid's FAS right-hand side,
// rhs += L(pn + u0) (Algorithm 1), with the G it forms anyway, writes it and takes it into f,
// instead of a separate residual launch before the snapshot.  XT = 2, interpolation (the first
// snapshot of a grid's post-smoothing): the block first applies the coarse-grid correction
// u += P (u_c - u0_c) (Algorithm 1) to the box cells it reads and writes its tile's corrected u,
// instead of a separate interpolation launch.  Both take the separate launches' operations, so
// the values are the same.
template <int WARPS, int MINB, bool MIXED, bool NORM = false, int XT = 0>
__global__ void __launch_bounds__(32 * WARPS, MINB)
    k_snapshot_tma(LevelView<float> L, const double *area, const __grid_constant__ CUtensorMap mP,
                   const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mW,
                   const __grid_constant__ CUtensorMap mF, const __grid_constant__ CUtensorMap mR, int *err,
                   long long wait_limit, double *partials, LevelView<float> Cg) {
    constexpr bool FAS = XT == 1, INTERP = XT == 2;
    static_assert(!NORM || WARPS == 8, "the norm's thread-to-cell map is that of 8 warps per tile");
    using T = float;
    using Smem = SnapTmaSmem<WARPS, MIXED>;
    constexpr int NT = 32 * WARPS, RPW = 32 / WARPS;
    extern __shared__ unsigned char smem_snap[];
    Smem &S = *reinterpret_cast<Smem *>(smem_snap + ((128 - (smem_u32(smem_snap) & 127)) & 127));
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int lane = threadIdx.x, wy = threadIdx.y, tid = wy * 32 + lane;
    const int n = L.n, m = L.m, p = L.pitch;
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        fence_proxy_async();
        const unsigned wbytes = MIXED ? (unsigned)(kBR * kBCb * 2) : (unsigned)(kBR * kBC * 4);
        mbar_expect_tx(&S.bar, 2u * kBR * kBC * 4u + wbytes + 4096u + (L.has_rhs ? 4096u : 0u));
        tma_load(&S.P[0][0], &mP, j0 - 4, i0 - 2, &S.bar);
        tma_load(&S.U[0][0], &mU, j0 - 4, i0 - 2, &S.bar);
        if (MIXED) tma_load(&S.Wb[0][0], &mW, j0 - 8, i0 - 2, &S.bar);
        else tma_load(&S.W[0][0], &mW, j0 - 4, i0 - 2, &S.bar);
        tma_load(&S.F[0][0], &mF, j0, i0, &S.bar);
        if (L.has_rhs) tma_load(&S.R[0][0], &mR, j0, i0, &S.bar);
    }
    int I0 = 0, J0 = 0;   // INTERP: the first coarse row and column of E
    if (INTERP) {   // u_c - u0_c while the boxes are in flight
        I0 = max(0, i0 / 2 - 2);
        J0 = max(0, j0 / 2 - 2);
        const size_t lc = (size_t)Cg.n * Cg.pitch;
        for (int q = tid; q < kCR * kCR; q += NT) {
            const int r = q / kCR, cc = q - r * kCR, I = I0 + r, J = J0 + cc;
            float e = 0.f;
            if (I < Cg.n && J < Cg.m) {
                const size_t o = (size_t)I * Cg.pitch + J;
                e = sub_rn(ldc(Cg.u, o, lc, kDbgInterp), ldc(Cg.u0, o, lc, kDbgInterp));
            }
            S.E[r][cc] = e;
        }
    }
    __syncthreads();   // the barrier's initialisation is visible before anyone waits on it
    bool ok = true;
    if (wy == 0) ok = mbar_wait(&S.bar, 0, wait_limit);   // the other warps wait at the block barrier
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicOr(err, 4);
            mbar_wait(&S.bar, 0, kSnapDrain);   // no copy may still write once the block has ended
        }
        __syncthreads();
        return;
    }
    if (INTERP) {
        // u += P (u_c - u0_c) on the in-grid box cells of rows 0..35 and columns 2..37 (every u
        // the G box, the class and the residuals read), as k_interp_add: then the tile's cells
        // to u
        for (int q = tid; q < kBR * (kBC - 4); q += NT) {
            const int a = q / (kBC - 4), c = 2 + (q - a * (kBC - 4)), gi = i0 - 2 + a, gj = j0 - 4 + c;
            if (gi < 0 || gi >= n || gj < 0 || gj >= m) continue;
            int ri[2], ci[2];
            float rw[2], cw[2];
            const int nr = bl_taps(gi, Cg.n, ri, rw), nk = bl_taps(gj, Cg.m, ci, cw);
            T sacc = T(0);
            for (int x = 0; x < nr; ++x)
                for (int y = 0; y < nk; ++y) {
                    const int er = ri[x] - I0, ec = ci[y] - J0;
                    if (!MG_DBG_OK(er, kCR, kDbgInterp) || !MG_DBG_OK(ec, kCR, kDbgInterp)) continue;
                    sacc = fma_rn(T(rw[x] * cw[y]), S.E[er][ec], sacc);
                }
            S.U[a][c] = add_rn(S.U[a][c], sacc);
        }
        __syncthreads();
        const size_t lim = (size_t)n * p;
        for (int q = tid; q < 1024; q += NT) {
            const int ti = q >> 5, tj = q & 31, gi = i0 + ti, gj = j0 + tj;
            if (gi < n && gj < m) stc(L.u, (size_t)gi * p + gj, lim, kDbgInterp, S.U[ti + 2][tj + 4]);
        }
    }
    // edge tiles: box cells of pn and u outside the grid take the clamped cell's values (the
    // source is an in-grid cell of the box, never itself overwritten); w is read only at cells
    // inside the grid
    if (i0 < 2 || j0 < 4 || i0 + 34 > n || j0 + 36 > m) {
        for (int q = tid; q < kBR * kBC; q += NT) {
            const int a = q / kBC, c = q - a * kBC, gi = i0 - 2 + a, gj = j0 - 4 + c;
            const int ci = clamp_idx(gi, n - 1), cj = clamp_idx(gj, m - 1);
            if (ci != gi || cj != gj) {
                const int sa = ci - (i0 - 2), sc = cj - (j0 - 4);
                S.P[a][c] = S.P[sa][sc];
                S.U[a][c] = S.U[sa][sc];
            }
        }
        __syncthreads();
    }
    // G on the tile and its ring (box rows 1..34, columns 3..36)
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
        for (int k = 0; k < RPW; ++k) g_at(1 + wy + WARPS * k, lane + 4, false);
        if (wy < 2) g_at(33 + wy, lane + 4, false);
        if (tid < 68) g_at(1 + (tid >> 1), (tid & 1) ? 36 : 3, false);
    } else {
        for (int a = 1 + wy; a <= 34; a += WARPS) g_at(a, lane + 4, true);
        if (tid < 68) g_at(1 + (tid >> 1), (tid & 1) ? 36 : 3, true);
    }
    __syncthreads();
    const T ar = area ? T(area[L.level]) : T(0);
    const int gj = j0 + lane, c = lane + 4;
    const int lenr = min(32, m - j0), lenc = min(32, n - i0);
    T acc = T(0);   // NORM: this thread's sum of r^2
    const T c2 = L.cdiff * T(0.5);
    // f, G and the jump-set class of tile row wy + WARPS k (IN: no bounds tests needed)
    auto cell = [&](int k, auto in_tag) -> uint32_t {
        constexpr bool IN = decltype(in_tag)::value;
        const int ti = wy + WARPS * k, a = ti + 2, gi = i0 + ti;
        uint32_t star = 0;
        if (IN || (gi < n && gj < m)) {
            const bool hS = IN || gi + 1 < n, hN = IN || gi > 0, hE = IN || gj + 1 < m, hW = IN || gj > 0;
            const T gc = S.W[a][c];
            // twice the faces, with c2 = cdiff / 2 (face2 in arith.cuh: the same values)
            const T aS = face2(gc, S.W[a + 1][c], hS), aN = face2(gc, S.W[a - 1][c], hN);
            const T aE = face2(gc, S.W[a][c + 1], hE), aW = face2(gc, S.W[a][c - 1], hW);
            const T pc = S.P[a][c];
            T ds = mul_rn(aS, sub_rn(S.P[a + 1][c], pc));
            ds = fma_rn(aN, sub_rn(S.P[a - 1][c], pc), ds);
            ds = fma_rn(aE, sub_rn(S.P[a][c + 1], pc), ds);
            ds = fma_rn(aW, sub_rn(S.P[a][c - 1], pc), ds);
            const size_t o = (size_t)gi * p + gj, lim = (size_t)n * p;
            T base = add_rn(S.F[ti][lane], ar);
            if (FAS) {   // as k_residual_tma, mode 1, with uin = u (= u0 here)
                const T uc = S.U[a][c];
                T fl = mul_rn(aS, add_rn(sub_rn(S.P[a + 1][c], pc), sub_rn(S.U[a + 1][c], uc)));
                fl = fma_rn(aN, add_rn(sub_rn(S.P[a - 1][c], pc), sub_rn(S.U[a - 1][c], uc)), fl);
                fl = fma_rn(aE, add_rn(sub_rn(S.P[a][c + 1], pc), sub_rn(S.U[a][c + 1], uc)), fl);
                fl = fma_rn(aW, add_rn(sub_rn(S.P[a][c - 1], pc), sub_rn(S.U[a][c - 1], uc)), fl);
                const T Lv = sub_rn(fma_rn(c2, fl, -add_rn(S.F[ti][lane], ar)), mul_rn(L.inv_tau, uc));
                const T rn = add_rn(S.R[ti][lane], Lv);
                stc(L.rhs, o, lim, kDbgSnapshot, rn);
                base = add_rn(base, rn);
            } else if (L.has_rhs) {
                base = add_rn(base, S.R[ti][lane]);
            }
            stc(L.f, o, lim, kDbgSnapshot, fma_rn(-c2, ds, base));
            stc(L.G, o, lim, kDbgSnapshot, gc);
            // jump set D (Sec. 4.1): max > Sigma * min over the faces inside the domain; the
            // smallest coefficient, ties to the earlier of A, B, C, D (Sec. 4.1.3)
            const T big = T(3.0e38);
            const T vS = hS ? aS : big, vN = hN ? aN : big, vE = hE ? aE : big, vW = hW ? aW : big;
            const T mn = fmin(fmin(vS, vN), fmin(vE, vW));
            const T mx = fmax(fmax(hS ? aS : T(-1), hN ? aN : T(-1)), fmax(hE ? aE : T(-1), hW ? aW : T(-1)));
            const int am = vS == mn ? 0 : (vN == mn ? 1 : (vE == mn ? 2 : 3));
            const int cnt = (int)hS + (int)hN + (int)hE + (int)hW;
            if (cnt >= 2 && mx > mul_rn(L.Sigma, mn)) star = 1u << am;
            if (L.cls) stc(L.cls, o, lim, kDbgSnapshot, (uint8_t)star);
            if (NORM) {   // the residual of the cell at this state (as k_residual_tma, mode 0)
                const T uc = S.U[a][c];
                T fl = mul_rn(aS, add_rn(sub_rn(S.P[a + 1][c], pc), sub_rn(S.U[a + 1][c], uc)));
                fl = fma_rn(aN, add_rn(sub_rn(S.P[a - 1][c], pc), sub_rn(S.U[a - 1][c], uc)), fl);
                fl = fma_rn(aE, add_rn(sub_rn(S.P[a][c + 1], pc), sub_rn(S.U[a][c + 1], uc)), fl);
                fl = fma_rn(aW, add_rn(sub_rn(S.P[a][c - 1], pc), sub_rn(S.U[a][c - 1], uc)), fl);
                const T Lv = sub_rn(fma_rn(c2, fl, -add_rn(S.F[ti][lane], ar)), mul_rn(L.inv_tau, uc));
                const T r = L.has_rhs ? sub_rn(S.R[ti][lane], Lv) : -Lv;
                acc = add_square(acc, r);
            }
        }
        return star;
    };
    // row pieces (sweeps A, B): one ballot per row, finished by lanes 2k (A) and 2k+1 (B);
    // column pieces (sweeps C, D): bit ti of this thread's words
    uint32_t bits = 0, cC = 0, cD = 0;
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int ti = wy + WARPS * k;
        const uint32_t star = interior ? cell(k, std::true_type{}) : cell(k, std::false_type{});
        const uint32_t bA = __ballot_sync(0xffffffffu, star & 1u), bB = __ballot_sync(0xffffffffu, star & 2u);
        if (lane == 2 * k) bits = bA;
        if (lane == 2 * k + 1) bits = bB;
        cC |= ((star >> 2) & 1u) << ti;
        cD |= ((star >> 3) & 1u) << ti;
    }
    S.cm[0][wy][lane] = cC;
    S.cm[1][wy][lane] = cD;
    if (lane < 2 * RPW) {
        const int line = wy + WARPS * (lane >> 1), s = lane & 1;
        if (i0 + line < n)
            stc(L.mrow, ((size_t)s * n + i0 + line) * L.npm + (j0 >> 5), (size_t)2 * n * L.npm, kDbgMaskStore,
                members_of(bits, lenr));
    }
    __syncthreads();
    if (wy < 2 && j0 + lane < m) {   // warp 0: sweep C, warp 1: sweep D
        uint32_t v = 0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) v |= S.cm[wy][w][lane];
        stc(L.mcol, ((size_t)wy * m + j0 + lane) * L.npn + (i0 >> 5), (size_t)2 * m * L.npn, kDbgMaskStore,
            members_of(v, lenc));
    }
    if (NORM) {
        const double s = block_sum_warps(acc, S.red);
        if (tid == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
    }
}

template <int WARPS, int MINB, bool MIXED, bool NORM = false>
size_t snap_smem() {
    return sizeof(SnapTmaSmem<WARPS, MIXED>) + 128;
}

// Resident blocks per SM of the 32-, 16- and 8-warp variants (FP32 and mixed weights), measured
// once outside any capture, and the SM count.
struct SnapTmaOcc {
    int per_sm[2][3] = {{1, 1, 1}, {1, 1, 1}}, sms = 1;
};
SnapTmaOcc g_snap_occ;

template <int WARPS, int MINB, bool MIXED, bool NORM = false, int XT = 0>
int snap_attr() {
    const int smem = (int)snap_smem<WARPS, MINB, MIXED>();
    cudaFuncSetAttribute(k_snapshot_tma<WARPS, MINB, MIXED, NORM, XT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_snapshot_tma<WARPS, MINB, MIXED, NORM, XT>, 32 * WARPS, smem) !=
            cudaSuccess || v < 1)
        v = 1;
    return v;
}

template <int WARPS, int MINB, bool MIXED, bool NORM = false, int XT = 0>
void launch_v(const LevelView<float> &L, const double *area, const SnapMaps &M, int *err, long long wl,
              cudaStream_t st, double *partials = nullptr, const LevelView<float> *C = nullptr) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32), block(32, WARPS);
    const auto *mp = reinterpret_cast<const CUtensorMap *>(M.P);
    const auto *mu = reinterpret_cast<const CUtensorMap *>(M.U);
    const auto *mw = reinterpret_cast<const CUtensorMap *>(M.W);
    const auto *mf = reinterpret_cast<const CUtensorMap *>(M.F);
    const auto *mr = reinterpret_cast<const CUtensorMap *>(L.has_rhs ? M.R : M.F);
    k_snapshot_tma<WARPS, MINB, MIXED, NORM, XT><<<grid, block, snap_smem<WARPS, MINB, MIXED>(), st>>>(
        L, area, *mp, *mu, *mw, *mf, *mr, err, wl, partials, C ? *C : L);
}

template <bool MIXED, int XT = 0>
void launch_mixed(const LevelView<float> &L, const double *area, const SnapMaps &M, int *err, long long wl,
                  cudaStream_t st, const LevelView<float> *C = nullptr) {
    const long tiles = (long)((L.m + 31) / 32) * ((L.n + 31) / 32);
    const int *ps = g_snap_occ.per_sm[MIXED ? 1 : 0];
    // the most threads per tile with which every tile still gets a resident block
    if (tiles <= (long)g_snap_occ.sms * ps[0]) launch_v<32, 1, MIXED, false, XT>(L, area, M, err, wl, st, nullptr, C);
    else if (tiles <= (long)g_snap_occ.sms * ps[1]) launch_v<16, 1, MIXED, false, XT>(L, area, M, err, wl, st, nullptr, C);
    else launch_v<8, 7, MIXED, false, XT>(L, area, M, err, wl, st, nullptr, C);
}

}  // namespace

void prepare_snapshot_tma() {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_snap_occ.sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_snap_occ.sms < 1) g_snap_occ.sms = 1;
    g_snap_occ.per_sm[0][0] = snap_attr<32, 1, false>();
    g_snap_occ.per_sm[0][1] = snap_attr<16, 1, false>();
    g_snap_occ.per_sm[0][2] = snap_attr<8, 7, false>();
    g_snap_occ.per_sm[1][0] = snap_attr<32, 1, true>();
    g_snap_occ.per_sm[1][1] = snap_attr<16, 1, true>();
    g_snap_occ.per_sm[1][2] = snap_attr<8, 7, true>();
    (void)snap_attr<8, 7, false, true>();
    (void)snap_attr<8, 7, true, true>();
    (void)snap_attr<32, 1, false, false, 1>();
    (void)snap_attr<16, 1, false, false, 1>();
    (void)snap_attr<8, 7, false, false, 1>();
    (void)snap_attr<32, 1, true, false, 1>();
    (void)snap_attr<16, 1, true, false, 1>();
    (void)snap_attr<8, 7, true, false, 1>();
    (void)snap_attr<32, 1, false, false, 2>();
    (void)snap_attr<16, 1, false, false, 2>();
    (void)snap_attr<8, 7, false, false, 2>();
    (void)snap_attr<32, 1, true, false, 2>();
    (void)snap_attr<16, 1, true, false, 2>();
    (void)snap_attr<8, 7, true, false, 2>();
}

bool encode_snapshot_maps(const LevelView<float> &L, SnapMaps *M) {
    bool ok = encode_map_2d(M->P, L.pn, 4, L.n, L.m, L.pitch, kBR, kBC) &&
              encode_map_2d(M->U, L.u, 4, L.n, L.m, L.pitch, kBR, kBC) &&
              encode_map_2d(M->F, L.F, 4, L.n, L.m, L.pitch, 32, 32);
    if (L.wb) ok = ok && encode_map_2d(M->W, (void *)L.wb, 2, L.n, L.m, L.pitch, kBR, kBCb);
    else ok = ok && encode_map_2d(M->W, L.w, 4, L.n, L.m, L.pitch, kBR, kBC);
    if (L.rhs) ok = ok && encode_map_2d(M->R, L.rhs, 4, L.n, L.m, L.pitch, 32, 32);
    M->mixed = L.wb != nullptr;
    return ok;
}

void launch_snapshot_tma(const LevelView<float> &L, const double *area, const SnapMaps &M, int *err,
                         long long wait_limit, cudaStream_t st) {
    if (M.mixed) launch_mixed<true>(L, area, M, err, wait_limit, st);
    else launch_mixed<false>(L, area, M, err, wait_limit, st);
}

void launch_snapshot_fas_tma(const LevelView<float> &L, const double *area, const SnapMaps &M, int *err,
                             long long wait_limit, cudaStream_t st) {
    if (M.mixed) launch_mixed<true, 1>(L, area, M, err, wait_limit, st);
    else launch_mixed<false, 1>(L, area, M, err, wait_limit, st);
}

void launch_snapshot_interp_tma(const LevelView<float> &L, const LevelView<float> &C, const double *area,
                                const SnapMaps &M, int *err, long long wait_limit, cudaStream_t st) {
    if (M.mixed) launch_mixed<true, 2>(L, area, M, err, wait_limit, st, &C);
    else launch_mixed<false, 2>(L, area, M, err, wait_limit, st, &C);
}

void launch_snapshot_norm_tma(const LevelView<float> &L, const double *area, const SnapMaps &M, double *partials,
                              int *err, long long wait_limit, cudaStream_t st) {
    if (M.mixed) launch_v<8, 7, true, true>(L, area, M, err, wait_limit, st, partials);
    else launch_v<8, 7, false, true>(L, area, M, err, wait_limit, st, partials);
}

}  // namespace segmg
