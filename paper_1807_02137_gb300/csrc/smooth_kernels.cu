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
//   - the fused path runs one kernel per sweep on output tiles (32 x 64 by default; the shape
//     is chosen per grid) with a 4-cell halo, recomputing the halo redundantly so that no tile
//     depends on another within a sweep.
#include "arith.cuh"
#include "line_phase.cuh"

namespace segmg {

namespace {

// ---------------------------------------------------------------------------------------
// Snapshot: G and f of every cell and the member mask of every 32-cell piece of every row and
// column (32 x 32 tiles aligned to the pieces, so each piece lies inside exactly one tile).
// ---------------------------------------------------------------------------------------
// WARPS warps per tile (8, 16 or 32): more threads per tile shorten each thread's chain of work
// on small grids, where a launch is latency-bound; large grids use 8 (more tiles per SM).
// MINB > 1 asks the compiler for that many resident blocks per SM (fewer registers): used when
// it lets every tile of the grid be resident at once (a 1024^2 grid with 8 warps per tile)
template <typename T, int WARPS, int MINB = 1>
__global__ void __launch_bounds__(32 * WARPS, MINB) k_snapshot(LevelView<T> L, const double *area) {
    constexpr int R = 36, NT = 32 * WARPS, RPW = 32 / WARPS;   // threads; tile rows per warp
    __shared__ T sP[R][R + 1];
    __shared__ T sU[R][R + 1];
    __shared__ T sG[R][R + 1];
    // FP32 stages w, F and rhs in shared memory too; FP64 reads them from global memory (its
    // static shared memory would otherwise exceed 48 KB)
    constexpr bool kStage = sizeof(T) == 4;
    constexpr int RW = kStage ? R : 1, FW = kStage ? 32 : 1;
    __shared__ T sW[RW][RW + 1];
    __shared__ T sF[FW][FW + 1];
    __shared__ T sR[FW][FW + 1];
    __shared__ uint8_t sStar[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int n = L.n, m = L.m, p = L.pitch;
    // stage pn, u (mirror-clamped, 36 x 36), w and F, rhs (FP32 only) with vector loads
    load_halo2<T, NT>(sP, L.pn, sU, L.u, i0, j0, n, m, p, tid);
    if (kStage) {
        if (!L.wb) load_halo2<T, NT>(reinterpret_cast<T (*)[37]>(sW), L.w, nullptr, nullptr, i0, j0, n, m, p, tid);
        load_tile32<T, NT>(reinterpret_cast<T (*)[33]>(sF), L.F, reinterpret_cast<T (*)[33]>(sR),
                           L.has_rhs ? L.rhs : nullptr, i0, j0, n, m, p, tid);
    }
    __syncthreads();
    // Lane = tile column, warp row wy handles tile rows wy, wy + WARPS, ....  Interior
    // tiles (every cell with four faces, the G ring inside the grid) skip the bounds tests.
    const int lane = threadIdx.x, wy = threadIdx.y;
    const bool interior = i0 >= 1 && j0 >= 1 && i0 + 33 <= n && j0 + 33 <= m;
    auto g_at = [&](int a, int b, bool check) {   // G of box cell (a, b), 1 <= a, b <= 34
        const int gi = i0 - 2 + a, gj = j0 - 2 + b;
        T g = T(0);
        if (!check || (gi >= 0 && gi < n && gj >= 0 && gj < m))
            g = cell_G((L.wb || !kStage) ? weight_at(L, (size_t)gi * p + gj) : sW[kStage ? a : 0][kStage ? b : 0],
                       sP[a + 1][b], sP[a - 1][b], sP[a][b + 1], sP[a][b - 1], sU[a + 1][b], sU[a - 1][b],
                       sU[a][b + 1], sU[a][b - 1], L.inv_2h, L.beta);
        sG[a][b] = g;
    };
    // G on the 34 x 34 box rows / columns 1..34: the 32 tile columns by lane, then the two ring
    // columns (68 cells) packed into whole warps
    if (interior) {
        for (int a = 1 + wy; a <= 34; a += WARPS) g_at(a, lane + 2, false);
        if (tid < 68) g_at(1 + (tid >> 1), (tid & 1) ? 34 : 1, false);
    } else {
        for (int a = 1 + wy; a <= 34; a += WARPS) g_at(a, lane + 2, true);
        if (tid < 68) g_at(1 + (tid >> 1), (tid & 1) ? 34 : 1, true);
    }
    __syncthreads();
    const T ar = area ? T(area[L.level]) : T(0);
    const int gj = j0 + lane, b = lane + 2;
    const int lenr = min(32, m - j0), lenc = min(32, n - i0);
    // The 4 RPW pieces of this warp (rows wy + WARPS k: sweeps A, B; columns wy + WARPS k:
    // sweeps C, D) are collected as ballots into lanes 0 .. 4 RPW - 1 and finished by one
    // members_of: lane 2k + s holds row wy + WARPS k, sweep A (s = 0) or B (s = 1); lane
    // 2 RPW + 2k + s column wy + WARPS k, sweep C or D.
    uint32_t bits = 0;
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const int ti = wy + WARPS * k, a = ti + 2, gi = i0 + ti;
        uint8_t star = 0;
        if (interior || (gi < n && gj < m)) {
            const bool hS = interior || gi + 1 < n, hN = interior || gi > 0;
            const bool hE = interior || gj + 1 < m, hW = interior || gj > 0;
            T gc = sG[a][b];
            T aS = face(gc, sG[a + 1][b], hS), aN = face(gc, sG[a - 1][b], hN);
            T aE = face(gc, sG[a][b + 1], hE), aW = face(gc, sG[a][b - 1], hW);
            T pc = sP[a][b];
            T ds = mul_rn(aS, sub_rn(sP[a + 1][b], pc));
            ds = fma_rn(aN, sub_rn(sP[a - 1][b], pc), ds);
            ds = fma_rn(aE, sub_rn(sP[a][b + 1], pc), ds);
            ds = fma_rn(aW, sub_rn(sP[a][b - 1], pc), ds);
            size_t o = (size_t)gi * p + gj;
            const size_t lim = (size_t)n * p;
            T base = add_rn(kStage ? sF[kStage ? ti : 0][kStage ? lane : 0] : ldc(L.F, o, lim, kDbgSnapshot), ar);
            if (L.has_rhs)
                base = add_rn(base, kStage ? sR[kStage ? ti : 0][kStage ? lane : 0] : ldc(L.rhs, o, lim, kDbgSnapshot));
            stc(L.f, o, lim, kDbgSnapshot, fma_rn(-L.cdiff, ds, base));
            stc(L.G, o, lim, kDbgSnapshot, gc);
            // jump set D (Sec. 4.1): max > Sigma * min over the faces inside the domain;
            // smallest coefficient with ties to the earlier of A, B, C, D (Sec. 4.1.3).
            const T big = T(3.0e38);
            const T vS = hS ? aS : big, vN = hN ? aN : big, vE = hE ? aE : big, vW = hW ? aW : big;
            const T mn = fmin(fmin(vS, vN), fmin(vE, vW));
            const T mx = fmax(fmax(hS ? aS : T(-1), hN ? aN : T(-1)), fmax(hE ? aE : T(-1), hW ? aW : T(-1)));
            const int am = vS == mn ? 0 : (vN == mn ? 1 : (vE == mn ? 2 : 3));
            const int cnt = (int)hS + (int)hN + (int)hE + (int)hW;
            if (cnt >= 2 && mx > mul_rn(L.Sigma, mn)) star = (uint8_t)(1u << am);
            if (L.cls) stc(L.cls, o, lim, kDbgSnapshot, star);
        }
        sStar[ti][lane] = star;
        const uint32_t bA = __ballot_sync(0xffffffffu, star & 1u), bB = __ballot_sync(0xffffffffu, star & 2u);
        if (lane == 2 * k) bits = bA;
        if (lane == 2 * k + 1) bits = bB;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < RPW; ++k) {
        const uint8_t sc = sStar[lane][wy + WARPS * k];
        const uint32_t bC = __ballot_sync(0xffffffffu, sc & 4u), bD = __ballot_sync(0xffffffffu, sc & 8u);
        if (lane == 2 * RPW + 2 * k) bits = bC;
        if (lane == 2 * RPW + 2 * k + 1) bits = bD;
    }
    if (lane < 4 * RPW) {
        const bool row = lane < 2 * RPW;
        const int line = wy + WARPS * ((lane >> 1) % RPW), s = lane & 1;
        const uint32_t mk = members_of(bits, row ? lenr : lenc);
        if (row) {
            if (i0 + line < n)
                stc(L.mrow, ((size_t)s * n + i0 + line) * L.npm + (j0 >> 5), (size_t)2 * n * L.npm, kDbgMaskStore, mk);
        } else if (j0 + line < m) {
            stc(L.mcol, ((size_t)s * m + j0 + line) * L.npn + (i0 >> 5), (size_t)2 * m * L.npn, kDbgMaskStore, mk);
        }
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
    if (member_bit(L, sweep, i, j)) return;
    bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
    size_t oS = hS ? o + p : o, oN = hN ? o - p : o, oE = hE ? o + 1 : o, oW = hW ? o - 1 : o;
    T gc = L.G[o];
    T aS = face(gc, L.G[oS], hS), aN = face(gc, L.G[oN], hN);
    T aE = face(gc, L.G[oE], hE), aW = face(gc, L.G[oW], hW);
    T v = point_relax(L.cdiff, L.inv_tau, aS, aN, aE, aW, L.u[oS], L.u[oN], L.u[oE], L.u[oW], L.f[o]);
    if (L.omega) v = relax_weighted(L.omega[o], v, L.u[o]);
    stc(L.u, o, (size_t)n * p, kDbgSweep, v);
}

// One warp per (line, 32-cell piece), solved together by pcr_piece; groups are read from upre
// (the values at the start of the phase) and written to u.
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
    const uint32_t mask = rowwise ? ldc(L.mrow, ((size_t)sweep * n + line) * L.npm + piece, (size_t)2 * n * L.npm, kDbgMaskLoad)
                                  : ldc(L.mcol, ((size_t)(sweep - 2) * m + line) * L.npn + piece, (size_t)2 * m * L.npn, kDbgMaskLoad);
    if (!mask) return;   // the whole warp
    const T *up = L.upre;
    auto at = [&](int t) -> RunCell<T> {
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
    const T own = lane < len ? up[cell(lane)] : T(0);
    T endp = T(0), endn = T(0);
    if (t0 > 0) endp = up[rowwise ? (size_t)line * p + t0 - 1 : (size_t)(t0 - 1) * p + line];
    if (t0 + len < llen) endn = up[rowwise ? (size_t)line * p + t0 + len : (size_t)(t0 + len) * p + line];
    T x;
    if (pcr_piece<T>(mask, len, L.cdiff, L.inv_tau, own, endp, endn, at, x)) stc(L.u, cell(lane), (size_t)n * p, kDbgSweep, x);
}

// ---------------------------------------------------------------------------------------
// Fused path: one kernel per sweep, reading u from one buffer and writing the other (sweeps A
// and C: u -> t, B and D: t -> u).  A block owns a 32 x 64 output tile (aligned to the
// 32-cell pieces of rows and columns) and loads it with a 4-cell halo: two checkerboard phases
// and two zebra phases each consume one cell of halo across the line direction, and the
// checkerboard phases one cell each along it.  Shared memory holds each field split by
// checkerboard colour (cell (a, b) of the region at [(a + b) & 1][a][b >> 1]), so the cells a
// warp updates in one colour phase, and their neighbours, are consecutive words.
// ---------------------------------------------------------------------------------------
constexpr int kH = 4;

// Tile shapes of the fused sweep (output rows x columns, threads): both sides multiples of 32 so
// that every 32-cell piece of a row or column lies wholly inside one tile.  The shape changes
// only the memory traffic, never the results (tested); the autotuner picks one per grid.
template <int OH_, int OW_, int NT_>
struct TileShape {
    static constexpr int OH = OH_, OW = OW_, NT = NT_;
    static constexpr int RH = OH + 2 * kH, RW = OW + 2 * kH, HW = RW / 2;
    // member-mask words per region line: OW/32 + 2 pieces along a row, OH/32 + 2 along a column
    static constexpr int RowPieces = OW / 32 + 2, ColPieces = OH / 32 + 2;
    static constexpr int MkLines = RH > RW ? RH : RW, MkPieces = RowPieces > ColPieces ? RowPieces : ColPieces;
};
using Tile0 = TileShape<32, 64, 256>;
using Tile1 = TileShape<32, 32, 128>;
using Tile2 = TileShape<64, 64, 512>;
using Tile3 = TileShape<32, 64, 512>;   // more threads per tile: fewer cells per thread per phase
using Tile4 = TileShape<32, 32, 256>;
using Tile5 = TileShape<32, 32, 512>;   // one cell per thread per checkerboard phase

template <typename T, typename TS>
struct FusedSmem {
    T u[2][TS::RH][TS::HW];
    T G[2][TS::RH][TS::HW];
    T f[2][TS::RH][TS::HW];
    uint32_t mk[TS::MkLines][TS::MkPieces];   // rowwise: [region row][piece]; colwise: [region column][piece]
};

#define SW_AT(arr, a, b) S.arr[((a) + (b)) & 1][a][(b) >> 1]

// Member bit of region cell (a, b) in the tile's sweep (masks staged in S.mk).
template <typename T, typename TS, bool ROWWISE>
__device__ __forceinline__ bool tile_member(const FusedSmem<T, TS> &S, int a, int b) {
    if (ROWWISE) return (S.mk[a][(b + 28) >> 5] >> ((b - kH) & 31)) & 1u;
    return (S.mk[b][(a + 28) >> 5] >> ((a - kH) & 31)) & 1u;
}

// One checkerboard phase over the region cells within distance 3 - ph of the output tile.
// INTERIOR: the whole region lies inside the domain, so every updated cell has four faces.
template <typename T, typename TS, int SWEEP, bool INTERIOR, bool WEIGHTED>
__device__ __forceinline__ void rb_phase(FusedSmem<T, TS> &S, const LevelView<T> &L, int ph, int i0, int j0) {
    constexpr int kRH = TS::RH, kRW = TS::RW, kHW = TS::HW, kThreads = TS::NT;
    constexpr bool rev = (SWEEP & 1) != 0;
    const int colour = rev ? 1 - ph : ph, lo = 1 + ph, other = 1 - colour;
    const int R = kRH - 2 * lo;
    const int n = L.n, m = L.m;
    for (int q = threadIdx.x; q < R * kHW; q += kThreads) {
        const int a = lo + q / kHW, k = q % kHW;
        const int x = (a + colour) & 1, b = 2 * k + x;
        if (b < lo || b >= kRW - lo) continue;
        bool hS = true, hN = true, hE = true, hW = true;
        if (!INTERIOR) {
            const int gi = i0 - kH + a, gj = j0 - kH + b;
            if (gi < 0 || gi >= n || gj < 0 || gj >= m) continue;
            hS = gi + 1 < n; hN = gi > 0; hE = gj + 1 < m; hW = gj > 0;
        }
        if (tile_member<T, TS, (SWEEP < 2)>(S, a, b)) continue;
        const T gc = S.G[colour][a][k];
        const T aS = face(gc, S.G[other][a + 1][k], hS), aN = face(gc, S.G[other][a - 1][k], hN);
        const T aE = face(gc, S.G[other][a][k + x], hE), aW = face(gc, S.G[other][a][k + x - 1], hW);
        T v = point_relax(L.cdiff, L.inv_tau, aS, aN, aE, aW, S.u[other][a + 1][k], S.u[other][a - 1][k],
                          S.u[other][a][k + x], S.u[other][a][k + x - 1], S.f[colour][a][k]);
        if (WEIGHTED) {
            const size_t o = (size_t)(i0 - kH + a) * L.pitch + (j0 - kH + b);
            v = relax_weighted(__ldg(L.omega + o), v, S.u[colour][a][k]);
        }
        S.u[colour][a][k] = v;
    }
}

template <typename T, int SWEEP, typename TS>
__global__ void __launch_bounds__(TS::NT) k_sweep(LevelView<T> L) {
    constexpr int kOH = TS::OH, kOW = TS::OW, kRH = TS::RH, kRW = TS::RW, kThreads = TS::NT;
    constexpr int kRowPieces = TS::RowPieces, kColPieces = TS::ColPieces;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FusedSmem<T, TS> &S = *reinterpret_cast<FusedSmem<T, TS> *>(smem_raw);
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n, NV = kRW / VN, NVO = kOW / VN;
    constexpr bool rowwise = SWEEP < 2, rev = (SWEEP & 1) != 0;
    const int i0 = blockIdx.y * kOH, j0 = blockIdx.x * kOW;
    const int n = L.n, m = L.m, p = L.pitch;
    const int tid = threadIdx.x;
    // ping-pong: tiles read their halo from one buffer and write their output to the other, so
    // no tile can read a neighbour's already updated cells
    const T *uin = (SWEEP & 1) ? L.t : L.u;
    T *uout = (SWEEP & 1) ? L.u : L.t;
    // ---- load u, G, f as vectors (the region starts 16-byte aligned): all loads of a batch are
    // issued before any shared-memory store, so they are in flight together
    constexpr int NVEC = kRH * NV, PER = (NVEC + kThreads - 1) / kThreads, BATCH = VN == 4 ? PER : 3;
#pragma unroll
    for (int k0 = 0; k0 < PER; k0 += BATCH) {
        V x[BATCH][3];
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int q = tid + (k0 + k) * kThreads;
            const int a = q / NV, b0 = (q % NV) * VN;
            const int gi = i0 - kH + a, gj = j0 - kH + b0;
            if (k0 + k < PER && q < NVEC && gi >= 0 && gi < n && gj >= 0 && gj < p &&
                MG_DBG_OK((size_t)gi * p + gj + VN - 1, (size_t)n * p, kDbgSweep)) {
                const size_t o = (size_t)gi * p + gj;
                x[k][0] = __ldg(reinterpret_cast<const V *>(uin + o));
                x[k][1] = __ldg(reinterpret_cast<const V *>(L.G + o));
                x[k][2] = __ldg(reinterpret_cast<const V *>(L.f + o));
            } else {
                memset(&x[k][0], 0, 3 * sizeof(V));
            }
        }
#pragma unroll
        for (int k = 0; k < BATCH; ++k) {
            const int q = tid + (k0 + k) * kThreads;
            if (k0 + k >= PER || q >= NVEC) continue;
            const int a = q / NV, b0 = (q % NV) * VN;
            T e3[3][VN];
            memcpy(e3, x[k], sizeof(e3));
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                SW_AT(u, a, b0 + e) = e3[0][e];
                SW_AT(G, a, b0 + e) = e3[1][e];
                SW_AT(f, a, b0 + e) = e3[2][e];
            }
        }
    }
    // ---- member masks of every line piece that touches the region (zero outside the domain)
    bool lm = false;   // a piece the line phases solve has a member
    if (rowwise) {
        for (int q = tid; q < kRH * kRowPieces; q += kThreads) {
            const int a = q / kRowPieces, pc = q % kRowPieces;
            const int gi = i0 - kH + a, piece = (j0 >> 5) - 1 + pc;
            uint32_t w = 0;
            if (gi >= 0 && gi < n && piece >= 0 && piece < L.npm &&
                MG_DBG_OK(((size_t)SWEEP * n + gi) * L.npm + piece, (size_t)2 * n * L.npm, kDbgMaskLoad))
                w = __ldg(L.mrow + ((size_t)SWEEP * n + gi) * L.npm + piece);
            S.mk[a][pc] = w;
            lm |= solves_word<kH, kOH, kOW, true>(a, pc, w);
        }
    } else {
        for (int q = tid; q < kRW * kColPieces; q += kThreads) {
            const int b = q / kColPieces, pc = q % kColPieces;
            const int gj = j0 - kH + b, piece = (i0 >> 5) - 1 + pc;
            uint32_t w = 0;
            if (gj >= 0 && gj < m && piece >= 0 && piece < L.npn &&
                MG_DBG_OK(((size_t)(SWEEP - 2) * m + gj) * L.npn + piece, (size_t)2 * m * L.npn, kDbgMaskLoad))
                w = __ldg(L.mcol + ((size_t)(SWEEP - 2) * m + gj) * L.npn + piece);
            S.mk[b][pc] = w;
            lm |= solves_word<kH, kOH, kOW, false>(b, pc, w);
        }
    }
    const bool lines = __syncthreads_or(lm);
    // ---- checkerboard phases (distance 3 then 2 from the output tile)
    const bool interior = i0 - kH >= 0 && i0 - kH + kRH <= n && j0 - kH >= 0 && j0 - kH + kRW <= m;
#pragma unroll
    for (int ph = 0; ph < 2; ++ph) {
        if (L.omega) {
            if (interior) rb_phase<T, TS, SWEEP, true, true>(S, L, ph, i0, j0);
            else rb_phase<T, TS, SWEEP, false, true>(S, L, ph, i0, j0);
        } else {
            if (interior) rb_phase<T, TS, SWEEP, true, false>(S, L, ph, i0, j0);
            else rb_phase<T, TS, SWEEP, false, false>(S, L, ph, i0, j0);
        }
        __syncthreads();
    }
    // ---- partial-line phases (line_phase.cuh), skipped when no piece of the tile has a member
    if (lines)
        tile_line_phases<T, kH, kOH, kOW, kThreads, rowwise, rev>(
            [&](int a, int b) -> T & { return SW_AT(u, a, b); }, [&](int a, int b) { return SW_AT(G, a, b); },
            [&](int a, int b) { return SW_AT(f, a, b); }, [&](int li, int pc) { return S.mk[li][1 + pc]; }, i0, j0,
            n, m, L.cdiff, L.inv_tau);
    // ---- write the output tile (vectors; padding columns keep their loaded values)
    for (int q = tid; q < kOH * NVO; q += kThreads) {
        const int a = kH + q / NVO, b0 = kH + (q % NVO) * VN;
        const int gi = i0 + q / NVO, gj = j0 + (q % NVO) * VN;
        if (gi >= n || gj >= p) continue;
        if (!MG_DBG_OK((size_t)gi * p + gj + VN - 1, (size_t)n * p, kDbgSweep)) continue;
        T uu[VN];
        for (int e = 0; e < VN; ++e) uu[e] = SW_AT(u, a, b0 + e);
        V xv;
        memcpy(&xv, uu, sizeof(V));
        *reinterpret_cast<V *>(uout + (size_t)gi * p + gj) = xv;
    }
}

#undef SW_AT

}  // namespace

// Resident snapshot blocks per SM for 8, 16, 32 warps per tile and for 8 warps held to 7
// blocks per SM (FP32) (measured once, outside any capture), and the SM count.
template <typename T>
struct SnapOcc {
    int per_sm[4] = {1, 1, 1, 0}, sms = 1;
    SnapOcc() {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_snapshot<T, 8>, 256, 0) == cudaSuccess && v > 0) per_sm[0] = v;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_snapshot<T, 16>, 512, 0) == cudaSuccess && v > 0) per_sm[1] = v;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_snapshot<T, 32>, 1024, 0) == cudaSuccess && v > 0) per_sm[2] = v;
        if constexpr (sizeof(T) == 4)
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_snapshot<T, 8, 7>, 256, 0) == cudaSuccess) per_sm[3] = v;
    }
};

template <typename T>
const SnapOcc<T> &snap_occ() {
    static const SnapOcc<T> o;
    return o;
}

// The most threads per tile with which every tile of the grid still gets a resident block.
template <typename T>
void launch_snapshot(const LevelView<T> &L, const double *area, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32);
    const long tiles = (long)grid.x * grid.y;
    const SnapOcc<T> &o = snap_occ<T>();
    if (tiles <= (long)o.sms * o.per_sm[2])
        k_snapshot<T, 32><<<grid, dim3(32, 32), 0, st>>>(L, area);
    else if (tiles <= (long)o.sms * o.per_sm[1])
        k_snapshot<T, 16><<<grid, dim3(32, 16), 0, st>>>(L, area);
    else if (sizeof(T) == 4 && tiles <= (long)o.sms * o.per_sm[3])
        k_snapshot<T, 8, sizeof(T) == 4 ? 7 : 1><<<grid, dim3(32, 8), 0, st>>>(L, area);
    else
        k_snapshot<T, 8><<<grid, dim3(32, 8), 0, st>>>(L, area);
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

template <typename T, int SW, typename TS>
static void set_fused_attr() {
    cudaFuncSetAttribute(k_sweep<T, SW, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(FusedSmem<T, TS>));
}

template <typename T, typename TS>
static void set_fused_attrs() {
    set_fused_attr<T, 0, TS>(); set_fused_attr<T, 1, TS>(); set_fused_attr<T, 2, TS>(); set_fused_attr<T, 3, TS>();
}

// Raises the dynamic shared-memory limit of the fused sweep kernels on the current device and
// measures the snapshot's occupancy (called once per set-up, before any stream capture).
void prepare_smoother_kernels() {
    set_fused_attrs<float, Tile0>(); set_fused_attrs<float, Tile1>(); set_fused_attrs<float, Tile2>();
    set_fused_attrs<float, Tile3>(); set_fused_attrs<float, Tile4>(); set_fused_attrs<float, Tile5>();
    set_fused_attrs<double, Tile0>(); set_fused_attrs<double, Tile1>(); set_fused_attrs<double, Tile2>();
    set_fused_attrs<double, Tile3>(); set_fused_attrs<double, Tile4>(); set_fused_attrs<double, Tile5>();
    (void)snap_occ<double>();   // snapshot occupancy, measured here rather than inside a capture
}

template <typename T, int SW, typename TS>
static void launch_fused_one(const LevelView<T> &L, cudaStream_t st) {
    size_t smem = sizeof(FusedSmem<T, TS>);
    dim3 grid((L.m + TS::OW - 1) / TS::OW, (L.n + TS::OH - 1) / TS::OH);
    k_sweep<T, SW, TS><<<grid, TS::NT, smem, st>>>(L);
}

template <typename T, typename TS>
static void launch_fused_shape(const LevelView<T> &L, int sweep, cudaStream_t st) {
    switch (sweep) {
        case 0: launch_fused_one<T, 0, TS>(L, st); break;
        case 1: launch_fused_one<T, 1, TS>(L, st); break;
        case 2: launch_fused_one<T, 2, TS>(L, st); break;
        default: launch_fused_one<T, 3, TS>(L, st); break;
    }
}

template <typename T>
void launch_sweep_fused(const LevelView<T> &L, int sweep, int shape, cudaStream_t st) {
    if (shape == 1) launch_fused_shape<T, Tile1>(L, sweep, st);
    else if (shape == 2) launch_fused_shape<T, Tile2>(L, sweep, st);
    else if (shape == 3) launch_fused_shape<T, Tile3>(L, sweep, st);
    else if (shape == 4) launch_fused_shape<T, Tile4>(L, sweep, st);
    else if (shape == 5) launch_fused_shape<T, Tile5>(L, sweep, st);
    else launch_fused_shape<T, Tile0>(L, sweep, st);
}

template void launch_snapshot<double>(const LevelView<double> &, const double *, cudaStream_t);
template void launch_sweep_phased<float>(const LevelView<float> &, int, cudaStream_t);
template void launch_sweep_phased<double>(const LevelView<double> &, int, cudaStream_t);
template void launch_sweep_fused<float>(const LevelView<float> &, int, int, cudaStream_t);
template void launch_sweep_fused<double>(const LevelView<double> &, int, int, cudaStream_t);

}  // namespace segmg
