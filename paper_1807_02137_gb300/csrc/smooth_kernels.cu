// smooth_kernels.cu -- Hybrid Smoother 2 (Sec. 4.3) on the GPU.
//
// One outer smoothing iteration = one coefficient snapshot (the "global" variant of Sec. 3.2:
// coefficients frozen at the start of the iteration) followed by four directional sweeps that
// lag A, B, C, D in turn.  The parallel ordering of a sweep k:
//   1. point updates (eq. gslexrc) of the non-member cells of one checkerboard colour, then of
//      the other (red = (i+j) even first for A and C, black first for B and D);
//   2. partial-line solves of the member groups on lines of one parity, then the other (even
//      first for A and C, odd first for B and D).  Groups run along rows for A, B and along
//      columns for C, D, cut at multiples of 32 cells; all groups of one phase read the values
//      from the start of the phase.
// Two implementations compute exactly the same sequence of IEEE operations per cell:
//   - the phased path launches one kernel per phase (the reference implementation);
//   - the fused path runs one kernel per sweep on 32 x 64 output tiles with a 4-cell halo,
//     recomputing the halo redundantly so that no tile depends on another within a sweep.
#include "arith.cuh"

namespace segmg {

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// ---------------------------------------------------------------------------------------
// Snapshot: G, f and the cls byte of every cell (32 x 32 tiles aligned to the 32-cell pieces
// of rows and columns, so every piece of every line lies inside exactly one tile).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_snapshot(LevelView<T> L, const double *area) {
    constexpr int R = 36;
    __shared__ T sP[R][R + 1];
    __shared__ T sU[R][R + 1];
    __shared__ T sG[R][R + 1];
    __shared__ uint8_t sStar[32][33];
    __shared__ uint8_t sMem[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int n = L.n, m = L.m, p = L.pitch;
    for (int q = tid; q < R * R; q += 256) {
        int a = q / R, b = q % R;
        int gi = clampi(i0 - 2 + a, 0, n - 1), gj = clampi(j0 - 2 + b, 0, m - 1);
        sP[a][b] = L.pn[(size_t)gi * p + gj];
        sU[a][b] = L.u[(size_t)gi * p + gj];
    }
    __syncthreads();
    for (int q = tid; q < 34 * 34; q += 256) {
        int a = 1 + q / 34, b = 1 + q % 34;
        int gi = i0 - 2 + a, gj = j0 - 2 + b;
        T g = T(0);
        if (gi >= 0 && gi < n && gj >= 0 && gj < m)
            g = cell_G(L.w[(size_t)gi * p + gj], sP[a + 1][b], sP[a - 1][b], sP[a][b + 1], sP[a][b - 1],
                       sU[a + 1][b], sU[a - 1][b], sU[a][b + 1], sU[a][b - 1], L.inv_2h, L.beta);
        sG[a][b] = g;
    }
    __syncthreads();
    const T ar = area ? T(area[L.level]) : T(0);
    for (int q = tid; q < 1024; q += 256) {
        int ti = q / 32, tj = q % 32, a = ti + 2, b = tj + 2;
        int gi = i0 + ti, gj = j0 + tj;
        uint8_t star = 0;
        if (gi < n && gj < m) {
            bool hS = gi + 1 < n, hN = gi > 0, hE = gj + 1 < m, hW = gj > 0;
            T gc = sG[a][b];
            T aS = face(gc, sG[a + 1][b], hS), aN = face(gc, sG[a - 1][b], hN);
            T aE = face(gc, sG[a][b + 1], hE), aW = face(gc, sG[a][b - 1], hW);
            T pc = sP[a][b];
            T ds = mul_rn(aS, sub_rn(sP[a + 1][b], pc));
            ds = fma_rn(aN, sub_rn(sP[a - 1][b], pc), ds);
            ds = fma_rn(aE, sub_rn(sP[a][b + 1], pc), ds);
            ds = fma_rn(aW, sub_rn(sP[a][b - 1], pc), ds);
            size_t o = (size_t)gi * p + gj;
            T base = add_rn(L.F[o], ar);
            if (L.has_rhs) base = add_rn(base, L.rhs[o]);
            L.f[o] = fma_rn(-L.cdiff, ds, base);
            L.G[o] = gc;
            // jump set D (Sec. 4.1): max > Sigma * min over the faces inside the domain;
            // smallest coefficient with ties to the earlier of A, B, C, D (Sec. 4.1.3).
            const T big = T(3.0e38);
            const T vS = hS ? aS : big, vN = hN ? aN : big, vE = hE ? aE : big, vW = hW ? aW : big;
            const T mn = fmin(fmin(vS, vN), fmin(vE, vW));
            const T mx = fmax(fmax(hS ? aS : T(-1), hN ? aN : T(-1)), fmax(hE ? aE : T(-1), hW ? aW : T(-1)));
            const int am = vS == mn ? 0 : (vN == mn ? 1 : (vE == mn ? 2 : 3));
            const int cnt = (int)hS + (int)hN + (int)hE + (int)hW;
            if (cnt >= 2 && mx > mul_rn(L.Sigma, mn))
                star = (uint8_t)((1u << am) | kInD | (am << 5));
        }
        sStar[ti][tj] = star;
    }
    __syncthreads();
    const int warp = tid / 32, lane = tid % 32;
    const int lenr = min(32, m - j0), lenc = min(32, n - i0);
    for (int r = warp; r < 32; r += 8) {             // row pieces: sweeps A, B
        uint8_t s = sStar[r][lane];
        uint32_t mA = members_of(__ballot_sync(0xffffffffu, s & 1u), lenr);
        uint32_t mB = members_of(__ballot_sync(0xffffffffu, s & 2u), lenr);
        sMem[r][lane] = (uint8_t)((s & 0xf0u) | ((mA >> lane) & 1u) | (((mB >> lane) & 1u) << 1));
    }
    __syncthreads();
    for (int c = warp; c < 32; c += 8) {             // column pieces: sweeps C, D
        uint8_t s = sStar[lane][c];
        uint32_t mC = members_of(__ballot_sync(0xffffffffu, s & 4u), lenc);
        uint32_t mD = members_of(__ballot_sync(0xffffffffu, s & 8u), lenc);
        sMem[lane][c] |= (uint8_t)((((mC >> lane) & 1u) << 2) | (((mD >> lane) & 1u) << 3));
    }
    __syncthreads();
    for (int q = tid; q < 1024; q += 256) {
        int ti = q / 32, tj = q % 32, gi = i0 + ti, gj = j0 + tj;
        if (gi < n && gj < m) L.cls[(size_t)gi * p + gj] = sMem[ti][tj];
    }
}

// ---------------------------------------------------------------------------------------
// Phased path
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_rb(LevelView<T> L, int colour, int sweep) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    const int n = L.n, m = L.m, p = L.pitch;
    if (i >= n || j >= m || ((i + j) & 1) != colour) return;
    size_t o = (size_t)i * p + j;
    if ((L.cls[o] >> sweep) & 1u) return;
    bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
    size_t oS = hS ? o + p : o, oN = hN ? o - p : o, oE = hE ? o + 1 : o, oW = hW ? o - 1 : o;
    T gc = L.G[o];
    T aS = face(gc, L.G[oS], hS), aN = face(gc, L.G[oN], hN);
    T aE = face(gc, L.G[oE], hE), aW = face(gc, L.G[oW], hW);
    L.u[o] = point_relax(L.cdiff, L.inv_tau, aS, aN, aE, aW, L.u[oS], L.u[oN], L.u[oE], L.u[oW], L.f[o]);
}

// One warp per (line, 32-cell piece); groups are read from upre (the values at the start of
// the phase) and written to u.
template <typename T>
__global__ void __launch_bounds__(256) k_seg(LevelView<T> L, int sweep, int parity) {
    const int n = L.n, m = L.m, p = L.pitch;
    const bool rowwise = sweep < 2;
    const int nlines = rowwise ? n : m, llen = rowwise ? m : n;
    const int npieces = (llen + 31) / 32;
    const int nl = (nlines - parity + 1) / 2;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x % 32;
    if (wid >= nl * npieces) return;
    const int line = parity + 2 * (wid / npieces), piece = wid % npieces;
    const int t0 = piece * 32, len = min(32, llen - t0);
    auto cell = [&](int t) -> size_t {
        return rowwise ? (size_t)line * p + (t0 + t) : (size_t)(t0 + t) * p + line;
    };
    bool mbit = lane < len && ((L.cls[lane < len ? cell(lane) : cell(0)] >> sweep) & 1u);
    uint32_t mask = __ballot_sync(0xffffffffu, mbit);
    uint32_t starts = mask & ~(mask << 1);
    if (!((starts >> lane) & 1u)) return;
    uint32_t rest = ~(mask >> lane);
    int rl = rest ? __ffs(rest) - 1 : 32 - lane;
    const T *up = L.upre;
    auto at = [&](int s) -> RunCell<T> {
        int t = lane + s;
        int i = rowwise ? line : t0 + t, j = rowwise ? t0 + t : line;
        size_t o = cell(t);
        bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
        size_t oS = hS ? o + p : o, oN = hN ? o - p : o, oE = hE ? o + 1 : o, oW = hW ? o - 1 : o;
        T gc = L.G[o];
        T aS = face(gc, L.G[oS], hS), aN = face(gc, L.G[oN], hN);
        T aE = face(gc, L.G[oE], hE), aW = face(gc, L.G[oW], hW);
        RunCell<T> c;
        if (rowwise) { c.ap = aW; c.an = aE; c.ax1 = aS; c.ax2 = aN; c.ux1 = up[oS]; c.ux2 = up[oN]; }
        else         { c.ap = aN; c.an = aS; c.ax1 = aE; c.ax2 = aW; c.ux1 = up[oE]; c.ux2 = up[oW]; }
        c.f = L.f[o];
        return c;
    };
    int ta = t0 + lane, tb = t0 + lane + rl - 1;      // first / last position along the line
    T endp = T(0), endn = T(0);
    if (ta > 0) endp = up[rowwise ? (size_t)line * p + ta - 1 : (size_t)(ta - 1) * p + line];
    if (tb + 1 < llen) endn = up[rowwise ? (size_t)line * p + tb + 1 : (size_t)(tb + 1) * p + line];
    thomas_run<T>(rl, L.cdiff, L.inv_tau, endp, endn, at, [&](int s, T x) { L.u[cell(lane + s)] = x; });
}

// ---------------------------------------------------------------------------------------
// Fused path: one kernel per sweep.  A block owns a 32 x 64 output tile (aligned to the
// 32-cell pieces of rows and columns) and loads it with a 4-cell halo: two checkerboard phases
// and two zebra phases each consume one cell of halo across the line direction, and the
// checkerboard phases one cell each along it.  Shared memory holds each field split by
// checkerboard colour (cell (a, b) of the region at [(a + b) & 1][a][b >> 1]), so the cells a
// warp updates in one colour phase, and their neighbours, are consecutive words.
// ---------------------------------------------------------------------------------------
constexpr int kOH = 32, kOW = 64, kH = 4, kRH = kOH + 2 * kH, kRW = kOW + 2 * kH, kHW = kRW / 2;
constexpr int kMaxTasks = 72;

template <typename T> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int n = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
struct FusedSmem {
    T u[2][kRH][kHW];
    T G[2][kRH][kHW];
    T f[2][kRH][kHW];
    uint8_t c[2][kRH][kHW + 4];
    T endv[kMaxTasks][2];
    uint32_t mask[kMaxTasks];
};

#define SW_AT(arr, a, b) S.arr[((a) + (b)) & 1][a][(b) >> 1]

template <typename T, int SWEEP>
__global__ void __launch_bounds__(256) k_sweep(LevelView<T> L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<T> &S = *reinterpret_cast<FusedSmem<T> *>(smem_raw);
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n, NV = kRW / VN, NVO = kOW / VN;
    constexpr bool rowwise = SWEEP < 2, rev = (SWEEP & 1) != 0;
    const int i0 = blockIdx.y * kOH, j0 = blockIdx.x * kOW;
    const int n = L.n, m = L.m, p = L.pitch;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // ---- load u, G, f (vectors; the region starts 16-byte aligned) and the cls bytes
    for (int q = tid; q < kRH * NV; q += 256) {
        const int a = q / NV, b0 = (q % NV) * VN;
        const int gi = i0 - kH + a, gj = j0 - kH + b0;
        T uu[VN], gg[VN], ff[VN];
        if (gi >= 0 && gi < n && gj >= 0 && gj < p) {
            const size_t o = (size_t)gi * p + gj;
            V x = *reinterpret_cast<const V *>(L.u + o);
            V y = *reinterpret_cast<const V *>(L.G + o);
            V z = *reinterpret_cast<const V *>(L.f + o);
            memcpy(uu, &x, sizeof(V)); memcpy(gg, &y, sizeof(V)); memcpy(ff, &z, sizeof(V));
        } else {
            for (int e = 0; e < VN; ++e) uu[e] = gg[e] = ff[e] = T(0);
        }
        for (int e = 0; e < VN; ++e) {
            SW_AT(u, a, b0 + e) = uu[e];
            SW_AT(G, a, b0 + e) = gg[e];
            SW_AT(f, a, b0 + e) = ff[e];
        }
    }
    for (int q = tid; q < kRH * (kRW / 4); q += 256) {
        const int a = q / (kRW / 4), b0 = (q % (kRW / 4)) * 4;
        const int gi = i0 - kH + a, gj = j0 - kH + b0;
        uint32_t w4 = 0xffffffffu;
        if (gi >= 0 && gi < n && gj >= 0 && gj < p) w4 = *reinterpret_cast<const uint32_t *>(L.cls + (size_t)gi * p + gj);
        for (int e = 0; e < 4; ++e) SW_AT(c, a, b0 + e) = (uint8_t)(w4 >> (8 * e));
    }
    __syncthreads();
    // ---- checkerboard phases (distance 3 then 2 from the output tile)
#pragma unroll
    for (int ph = 0; ph < 2; ++ph) {
        const int colour = rev ? 1 - ph : ph, lo = 1 + ph, other = 1 - colour;
        const int R = kRH - 2 * lo;
        for (int q = tid; q < R * kHW; q += 256) {
            const int a = lo + q / kHW, k = q % kHW;
            const int x = (a + colour) & 1, b = 2 * k + x;
            if (b < lo || b >= kRW - lo) continue;
            const int gi = i0 - kH + a, gj = j0 - kH + b;
            if (gi < 0 || gi >= n || gj < 0 || gj >= m) continue;
            if ((S.c[colour][a][k] >> SWEEP) & 1u) continue;
            const bool hS = gi + 1 < n, hN = gi > 0, hE = gj + 1 < m, hW = gj > 0;
            const T gc = S.G[colour][a][k];
            const T aS = face(gc, S.G[other][a + 1][k], hS), aN = face(gc, S.G[other][a - 1][k], hN);
            const T aE = face(gc, S.G[other][a][k + x], hE), aW = face(gc, S.G[other][a][k + x - 1], hW);
            S.u[colour][a][k] = point_relax(L.cdiff, L.inv_tau, aS, aN, aE, aW, S.u[other][a + 1][k],
                                            S.u[other][a - 1][k], S.u[other][a][k + x],
                                            S.u[other][a][k + x - 1], S.f[colour][a][k]);
        }
        __syncthreads();
    }
    // ---- partial-line phases: lines at distance 1, then 0, one parity each
    constexpr int npc = rowwise ? 2 : 1;
    const int len_lim = rowwise ? m : n, gl_lim = rowwise ? n : m;
#pragma unroll
    for (int ph = 0; ph < 2; ++ph) {
        const int parity = rev ? 1 - ph : ph, dist = 1 - ph;
        const int lfirst = kH - dist;
        const int ntask = ((rowwise ? kOH : kOW) + 2 * dist) * npc;
        // step a: member masks by warp ballots, end values at the piece boundaries (pre-phase)
        for (int t = warp; t < ntask; t += 8) {
            const int li = lfirst + t / npc, pc = t % npc;
            const int gline = rowwise ? i0 - kH + li : j0 - kH + li;
            const int gstart = rowwise ? j0 + 32 * pc : i0;
            const int s0 = kH + 32 * pc;
            const bool ok = gline >= 0 && gline < gl_lim && (gline & 1) == parity && gstart < len_lim;
            const int len = ok ? min(32, len_lim - gstart) : 0;
            bool bit = false;
            if (lane < len) bit = ((rowwise ? SW_AT(c, li, s0 + lane) : SW_AT(c, s0 + lane, li)) >> SWEEP) & 1u;
            const uint32_t mk = __ballot_sync(0xffffffffu, bit);
            if (lane == 0) {
                T e0 = T(0), e1 = T(0);
                if (mk) {
                    if (gstart > 0) e0 = rowwise ? SW_AT(u, li, s0 - 1) : SW_AT(u, s0 - 1, li);
                    if (gstart + len < len_lim) e1 = rowwise ? SW_AT(u, li, s0 + len) : SW_AT(u, s0 + len, li);
                }
                S.mask[t] = mk;
                S.endv[t][0] = e0;
                S.endv[t][1] = e1;
            }
        }
        __syncthreads();
        // step b: every run of every task, one thread per task
        for (int t = tid; t < ntask; t += 256) {
            const uint32_t mk = S.mask[t];
            if (!mk) continue;
            const int li = lfirst + t / npc, pc = t % npc;
            const int s0 = kH + 32 * pc;
            const int gline = rowwise ? i0 - kH + li : j0 - kH + li;
            const int gstart = rowwise ? j0 + 32 * pc : i0;
            const int len = min(32, len_lim - gstart);
            int s = 0;
            while (s < len) {
                if (!((mk >> s) & 1u)) { ++s; continue; }
                const int a0 = s;
                while (s < len && ((mk >> s) & 1u)) ++s;
                const int rl = s - a0;
                const T endp = a0 == 0 ? S.endv[t][0] : (rowwise ? SW_AT(u, li, s0 + a0 - 1) : SW_AT(u, s0 + a0 - 1, li));
                const T endn = (a0 + rl == len) ? S.endv[t][1] : (rowwise ? SW_AT(u, li, s0 + a0 + rl) : SW_AT(u, s0 + a0 + rl, li));
                auto at = [&](int r) -> RunCell<T> {
                    const int pos = s0 + a0 + r;
                    const int a = rowwise ? li : pos, b = rowwise ? pos : li;
                    const int gi = rowwise ? gline : i0 - kH + pos, gj = rowwise ? j0 - kH + pos : gline;
                    const bool hS = gi + 1 < n, hN = gi > 0, hE = gj + 1 < m, hW = gj > 0;
                    const T gc = SW_AT(G, a, b);
                    const T aS = face(gc, SW_AT(G, a + 1, b), hS), aN = face(gc, SW_AT(G, a - 1, b), hN);
                    const T aE = face(gc, SW_AT(G, a, b + 1), hE), aW = face(gc, SW_AT(G, a, b - 1), hW);
                    RunCell<T> c;
                    if (rowwise) {
                        c.ap = aW; c.an = aE; c.ax1 = aS; c.ax2 = aN;
                        c.ux1 = SW_AT(u, a + 1, b); c.ux2 = SW_AT(u, a - 1, b);
                    } else {
                        c.ap = aN; c.an = aS; c.ax1 = aE; c.ax2 = aW;
                        c.ux1 = SW_AT(u, a, b + 1); c.ux2 = SW_AT(u, a, b - 1);
                    }
                    c.f = SW_AT(f, a, b);
                    return c;
                };
                thomas_run<T>(rl, L.cdiff, L.inv_tau, endp, endn, at, [&](int r, T xv) {
                    const int pos = s0 + a0 + r;
                    if (rowwise) SW_AT(u, li, pos) = xv; else SW_AT(u, pos, li) = xv;
                });
            }
        }
        __syncthreads();
    }
    // ---- write the output tile (vectors; padding columns keep their loaded values)
    for (int q = tid; q < kOH * NVO; q += 256) {
        const int a = kH + q / NVO, b0 = kH + (q % NVO) * VN;
        const int gi = i0 + q / NVO, gj = j0 + (q % NVO) * VN;
        if (gi >= n || gj >= p) continue;
        T uu[VN];
        for (int e = 0; e < VN; ++e) uu[e] = SW_AT(u, a, b0 + e);
        V x;
        memcpy(&x, uu, sizeof(V));
        *reinterpret_cast<V *>(L.u + (size_t)gi * p + gj) = x;
    }
}

#undef SW_AT

}  // namespace

template <typename T>
void launch_snapshot(const LevelView<T> &L, const double *area, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32), block(32, 8);
    k_snapshot<T><<<grid, block, 0, st>>>(L, area);
}

template <typename T>
void launch_sweep_phased(const LevelView<T> &L, int sweep, cudaStream_t st) {
    const bool rev = sweep & 1;
    dim3 grid((L.m + 31) / 32, (L.n + 7) / 8), block(32, 8);
    for (int ph = 0; ph < 2; ++ph) k_rb<T><<<grid, block, 0, st>>>(L, rev ? 1 - ph : ph, sweep);
    const bool rowwise = sweep < 2;
    const int nlines = rowwise ? L.n : L.m, llen = rowwise ? L.m : L.n;
    const int npieces = (llen + 31) / 32;
    for (int ph = 0; ph < 2; ++ph) {
        int parity = rev ? 1 - ph : ph;
        int nl = (nlines - parity + 1) / 2;
        if (nl <= 0) continue;
        cudaMemcpy2DAsync(L.upre, (size_t)L.pitch * sizeof(T), L.u, (size_t)L.pitch * sizeof(T),
                          (size_t)L.m * sizeof(T), L.n, cudaMemcpyDeviceToDevice, st);
        long warps = (long)nl * npieces;
        int blocks = (int)((warps * 32 + 255) / 256);
        k_seg<T><<<blocks, 256, 0, st>>>(L, sweep, parity);
    }
}

template <typename T, int SW>
static void set_fused_attr() {
    cudaFuncSetAttribute(k_sweep<T, SW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(FusedSmem<T>));
}

// Raises the dynamic shared-memory limit of the fused sweep kernels on the current device
// (called once per set-up, before any stream capture).
void prepare_smoother_kernels() {
    set_fused_attr<float, 0>(); set_fused_attr<float, 1>(); set_fused_attr<float, 2>(); set_fused_attr<float, 3>();
    set_fused_attr<double, 0>(); set_fused_attr<double, 1>(); set_fused_attr<double, 2>(); set_fused_attr<double, 3>();
}

template <typename T, int SW>
static void launch_fused_one(const LevelView<T> &L, cudaStream_t st) {
    size_t smem = sizeof(FusedSmem<T>);
    dim3 grid((L.m + kOW - 1) / kOW, (L.n + kOH - 1) / kOH);
    k_sweep<T, SW><<<grid, 256, smem, st>>>(L);
}

template <typename T>
void launch_sweep_fused(const LevelView<T> &L, int sweep, cudaStream_t st) {
    switch (sweep) {
        case 0: launch_fused_one<T, 0>(L, st); break;
        case 1: launch_fused_one<T, 1>(L, st); break;
        case 2: launch_fused_one<T, 2>(L, st); break;
        default: launch_fused_one<T, 3>(L, st); break;
    }
}

template void launch_snapshot<float>(const LevelView<float> &, const double *, cudaStream_t);
template void launch_snapshot<double>(const LevelView<double> &, const double *, cudaStream_t);
template void launch_sweep_phased<float>(const LevelView<float> &, int, cudaStream_t);
template void launch_sweep_phased<double>(const LevelView<double> &, int, cudaStream_t);
template void launch_sweep_fused<float>(const LevelView<float> &, int, cudaStream_t);
template void launch_sweep_fused<double>(const LevelView<double> &, int, cudaStream_t);

}  // namespace segmg
