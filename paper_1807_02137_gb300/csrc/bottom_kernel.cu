// bottom_kernel.cu -- the bottom of the FAS V-cycle (the small grids and the coarsest solve) in
// one block.
//
// On the small grids (here at most 64 x 64 cells) every kernel of the V-cycle is latency-bound:
// a launch costs far more than its few thousand cells of work.  This kernel runs the whole
// sub-cycle from grid `lb` down to the coarsest and back in a single 1024-thread block, with
// every grid resident in shared memory.  It executes, cell by cell, exactly the arithmetic of
// the per-grid kernels (the snapshot, the per-phase smoother, the residual, the transfers and the
// coarsest solve share their device functions), so the V-cycle's results do not change.
// Used for the FP32 / mixed storage and the Spencer-Chen model when the grids fit in shared
// memory; the host falls back to the per-grid kernels otherwise.
#include <cooperative_groups.h>

#include "arith.cuh"
#include "coarse_body.cuh"
#include "reduce.cuh"

#include <algorithm>

namespace segmg {

namespace {

constexpr int kBT = kCoarseThreads;   // threads of the block (the coarsest solve uses them all)
static_assert(kBT == kBottomThreads, "the host's default first grid assumes this block size");

// One grid in shared memory (row pitch m).
struct BGrid {
    int n, m, npm, npn;
    float cdiff, inv_tau, Sigma, inv_2h, beta;
    float *pn, *u, *w, *F, *rhs, *G, *f, *u0;
    uint32_t *mrow, *mcol;   // [2][n][npm], [2][m][npn]
    int has_rhs;
};


// Thread layout over an array with `cols` columns: TX = the power of two >= cols (at most the
// block size) threads along a row, kBT / TX rows at a time; no integer division per cell.
struct Map2 {
    int tx, ty, TX, TY;
};
__device__ __forceinline__ Map2 map_for(int cols) {
    int lg = cols <= 1 ? 0 : 32 - __clz(cols - 1);
    lg = min(lg, 10);
    Map2 r;
    r.TX = 1 << lg;
    r.TY = kBT >> lg;
    r.tx = threadIdx.x & (r.TX - 1);
    r.ty = threadIdx.x >> lg;
    return r;
}
#define FOR_CELLS(M, n, m, i, j)                                                              \
    for (int i = (M).ty; i < (n); i += (M).TY)                                                \
        for (int j = (M).tx; j < (m); j += (M).TX)

// G = w / |grad phi|_beta of every cell at phi = pn + uu (mirror-clamped neighbours), as the
// tile kernels form it.
__device__ void b_G(const BGrid &B, const float *uu) {
    const int n = B.n, m = B.m;
    const Map2 M = map_for(m);
    FOR_CELLS(M, n, m, i, j) {
        const int q = i * m + j;
        const int s = (i + 1 < n ? i + 1 : n - 1) * m + j, nn = (i > 0 ? i - 1 : 0) * m + j;
        const int e = q + (j + 1 < m ? 1 : 0), w = q - (j > 0 ? 1 : 0);
        stc(B.G, q, (size_t)n * m, kDbgBottom,
            cell_G(B.w[q], B.pn[s], B.pn[nn], B.pn[e], B.pn[w], uu[s], uu[nn], uu[e], uu[w], B.inv_2h, B.beta));
    }
    __syncthreads();
}

// Snapshot (as k_snapshot): G, f, jump class and the member masks of every piece.
__device__ void b_snapshot(const BGrid &B, uint8_t *star) {
    const int n = B.n, m = B.m;
    b_G(B, B.u);
    const Map2 M = map_for(m);
    FOR_CELLS(M, n, m, i, j) {
        const int q = i * m + j;
        const bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
        const int oS = hS ? q + m : q, oN = hN ? q - m : q, oE = hE ? q + 1 : q, oW = hW ? q - 1 : q;
        const float gc = B.G[q];
        const float aS = face(gc, B.G[oS], hS), aN = face(gc, B.G[oN], hN);
        const float aE = face(gc, B.G[oE], hE), aW = face(gc, B.G[oW], hW);
        const float pc = B.pn[q];
        float ds = mul_rn(aS, sub_rn(B.pn[oS], pc));
        ds = fma_rn(aN, sub_rn(B.pn[oN], pc), ds);
        ds = fma_rn(aE, sub_rn(B.pn[oE], pc), ds);
        ds = fma_rn(aW, sub_rn(B.pn[oW], pc), ds);
        float base = add_rn(B.F[q], 0.0f);
        if (B.has_rhs) base = add_rn(base, B.rhs[q]);
        stc(B.f, q, (size_t)n * m, kDbgBottom, fma_rn(-B.cdiff, ds, base));
        const float big = 3.0e38f;
        const float vS = hS ? aS : big, vN = hN ? aN : big, vE = hE ? aE : big, vW = hW ? aW : big;
        const float mn = fminf(fminf(vS, vN), fminf(vE, vW));
        const float mx = fmaxf(fmaxf(hS ? aS : -1.f, hN ? aN : -1.f), fmaxf(hE ? aE : -1.f, hW ? aW : -1.f));
        const int am = vS == mn ? 0 : (vN == mn ? 1 : (vE == mn ? 2 : 3));
        const int cnt = (int)hS + (int)hN + (int)hE + (int)hW;
        stc(star, q, (size_t)n * m, kDbgBottom, (cnt >= 2 && mx > mul_rn(B.Sigma, mn)) ? (uint8_t)(1u << am) : (uint8_t)0);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < n; i += kBT / 32)                  // row pieces: sweeps A, B
        for (int pc = 0; pc < B.npm; ++pc) {
            const int j = pc * 32 + lane, len = min(32, m - pc * 32);
            const uint8_t s = lane < len ? star[i * m + j] : 0;
            const uint32_t mA = members_of(__ballot_sync(0xffffffffu, s & 1u), len);
            const uint32_t mB = members_of(__ballot_sync(0xffffffffu, s & 2u), len);
            if (lane == 0) {
                stc(B.mrow, (size_t)(0 * n + i) * B.npm + pc, (size_t)2 * n * B.npm, kDbgBottom, mA);
                stc(B.mrow, (size_t)(1 * n + i) * B.npm + pc, (size_t)2 * n * B.npm, kDbgBottom, mB);
            }
        }
    for (int j = warp; j < m; j += kBT / 32)                  // column pieces: sweeps C, D
        for (int pc = 0; pc < B.npn; ++pc) {
            const int i = pc * 32 + lane, len = min(32, n - pc * 32);
            const uint8_t s = lane < len ? star[i * m + j] : 0;
            const uint32_t mC = members_of(__ballot_sync(0xffffffffu, s & 4u), len);
            const uint32_t mD = members_of(__ballot_sync(0xffffffffu, s & 8u), len);
            if (lane == 0) {
                stc(B.mcol, (size_t)(0 * m + j) * B.npn + pc, (size_t)2 * m * B.npn, kDbgBottom, mC);
                stc(B.mcol, (size_t)(1 * m + j) * B.npn + pc, (size_t)2 * m * B.npn, kDbgBottom, mD);
            }
        }
    __syncthreads();
}

__device__ __forceinline__ bool b_member(const BGrid &B, int sweep, int i, int j) {
    if (sweep < 2) return (B.mrow[(sweep * B.n + i) * B.npm + (j >> 5)] >> (j & 31)) & 1u;
    return (B.mcol[((sweep - 2) * B.m + j) * B.npn + (i >> 5)] >> (i & 31)) & 1u;
}

// The two partial-line phases of one directional sweep (as k_seg): one warp per line of the
// phase's parity.  Lines of one parity do not interact, and the cells just outside a piece lie
// on the same line, so a warp reads the end values of all its pieces before it solves any run:
// no block-wide barrier is needed within a phase.
__device__ void b_lines(const BGrid &B, int sweep, float *endv) {
    const int n = B.n, m = B.m;
    const bool rev = sweep & 1, rowwise = sweep < 2;
    const int nlines = rowwise ? n : m, llen = rowwise ? m : n, npieces = rowwise ? B.npm : B.npn;
    const int step = rowwise ? 1 : m;                 // stride along a line
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ph = 0; ph < 2; ++ph) {
        const int parity = rev ? 1 - ph : ph;
        const int nl = (nlines - parity + 1) / 2;
        for (int li = warp; li < nl; li += kBT / 32) {
            const int line = parity + 2 * li;
            const int base = rowwise ? line * m : line;   // cell of position 0 on the line
            const uint32_t *mks = rowwise ? B.mrow + (sweep * n + line) * B.npm
                                          : B.mcol + ((sweep - 2) * m + line) * B.npn;
            float *ev = endv + 2 * li * npieces;
            for (int pc = lane; pc < npieces; pc += 32) {
                const int t0 = pc * 32, len = min(32, llen - t0);
                ev[2 * pc] = t0 > 0 ? B.u[base + (t0 - 1) * step] : 0.f;
                ev[2 * pc + 1] = t0 + len < llen ? B.u[base + (t0 + len) * step] : 0.f;
            }
            __syncwarp();
            for (int pc = 0; pc < npieces; ++pc) {
                const uint32_t mk = mks[pc];
                if (!mk) continue;   // the whole warp
                const int t0 = pc * 32, len = min(32, llen - t0), tt = t0 + lane;
                const float own = lane < len ? B.u[base + tt * step] : 0.f;
                auto at = [&](int r) -> RunCell<float> {
                    const int o = base + (t0 + r) * step;
                    const int i = rowwise ? line : t0 + r, j = rowwise ? t0 + r : line;
                    const bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
                    const int oS = hS ? o + m : o, oN = hN ? o - m : o, oE = hE ? o + 1 : o, oW = hW ? o - 1 : o;
                    const float gc = B.G[o];
                    const float aS = face(gc, B.G[oS], hS), aN = face(gc, B.G[oN], hN);
                    const float aE = face(gc, B.G[oE], hE), aW = face(gc, B.G[oW], hW);
                    RunCell<float> c;
                    if (rowwise) { c.ap = aW; c.an = aE; c.ax1 = aS; c.ax2 = aN; c.ux1 = B.u[oS]; c.ux2 = B.u[oN]; }
                    else         { c.ap = aN; c.an = aS; c.ax1 = aE; c.ax2 = aW; c.ux1 = B.u[oE]; c.ux2 = B.u[oW]; }
                    c.f = B.f[o];
                    return c;
                };
                float x;
                if (pcr_piece<float>(mk, len, B.cdiff, B.inv_tau, own, ev[2 * pc], ev[2 * pc + 1], at, x))
                    stc(B.u, (size_t)(base + tt * step), (size_t)n * m, kDbgBottom, x);
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

// One directional sweep of Hybrid Smoother 2 in the parallel ordering (as k_rb + k_seg).
__device__ void b_sweep(const BGrid &B, int sweep, float *endv) {
    const int n = B.n, m = B.m;
    const bool rev = sweep & 1;
    // checkerboard phases: the cells of one colour, two per row pair of threads' columns
    const int mh = (m + 1) >> 1;
    const Map2 MH = map_for(mh);
    for (int ph = 0; ph < 2; ++ph) {
        const int colour = rev ? 1 - ph : ph;
        FOR_CELLS(MH, n, mh, i, k) {
            const int j = 2 * k + ((i + colour) & 1);
            if (j >= m || b_member(B, sweep, i, j)) continue;
            const int q = i * m + j;
            const bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
            const int oS = hS ? q + m : q, oN = hN ? q - m : q, oE = hE ? q + 1 : q, oW = hW ? q - 1 : q;
            const float gc = B.G[q];
            const float aS = face(gc, B.G[oS], hS), aN = face(gc, B.G[oN], hN);
            const float aE = face(gc, B.G[oE], hE), aW = face(gc, B.G[oW], hW);
            stc(B.u, q, (size_t)n * m, kDbgBottom,
                point_relax(B.cdiff, B.inv_tau, aS, aN, aE, aW, B.u[oS], B.u[oN], B.u[oE], B.u[oW], B.f[q]));
        }
        __syncthreads();
    }
    b_lines(B, sweep, endv);
}

// One outer smoothing iteration (snapshot and four sweeps) of a grid with at most one cell per
// thread.  The cell's four face values, the denominator of its point update, f and its member
// bits are formed once after the snapshot and kept in registers, so a checkerboard phase reads
// only the four neighbouring values of u from shared memory.  The update is point_relax's
// sequence of operations, so the results equal those of b_snapshot and four b_sweep calls; a
// sweep with no member cell on the grid skips its (empty) line phases.
__device__ void b_smooth_small(const BGrid &B, uint8_t *star, float *endv) {
    __shared__ unsigned s_any;   // bit k: sweep k has a member cell somewhere on the grid
    if (threadIdx.x == 0) s_any = 0;
    b_snapshot(B, star);         // ends with a barrier
    const int n = B.n, m = B.m, q = threadIdx.x;
    const bool own = q < n * m;
    float aS = 0.f, aN = 0.f, aE = 0.f, aW = 0.f, dv = 1.f, fq = 0.f;
    int oS = q, oN = q, oE = q, oW = q, colour = 0;
    unsigned mem = 0;
    if (own) {
        const int i = q / m, j = q - i * m;
        const bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
        oS = hS ? q + m : q; oN = hN ? q - m : q; oE = hE ? q + 1 : q; oW = hW ? q - 1 : q;
        const float gc = B.G[q];
        aS = face(gc, B.G[oS], hS); aN = face(gc, B.G[oN], hN);
        aE = face(gc, B.G[oE], hE); aW = face(gc, B.G[oW], hW);
        dv = fma_rn(B.cdiff, add_rn(add_rn(aS, aN), add_rn(aE, aW)), B.inv_tau);
        fq = B.f[q];
        colour = (i + j) & 1;
        for (int k = 0; k < 4; ++k) mem |= (unsigned)b_member(B, k, i, j) << k;
    }
    const unsigned wm = __reduce_or_sync(0xffffffffu, mem);
    if ((threadIdx.x & 31) == 0 && wm) atomicOr(&s_any, wm);
    __syncthreads();
    const unsigned any = s_any;
    for (int k = 0; k < 4; ++k) {
        const bool rev = k & 1;
        for (int ph = 0; ph < 2; ++ph) {
            if (own && colour == (rev ? 1 - ph : ph) && !((mem >> k) & 1u)) {
                float num = mul_rn(aS, B.u[oS]);
                num = fma_rn(aN, B.u[oN], num);
                num = fma_rn(aE, B.u[oE], num);
                num = fma_rn(aW, B.u[oW], num);
                stc(B.u, q, (size_t)n * m, kDbgBottom, div_relax(fma_rn(B.cdiff, num, -fq), dv));
            }
            __syncthreads();
        }
        if ((any >> k) & 1u) b_lines(B, k, endv);
    }
}

// out = rhs - L(pn + uu) (mode 0) or out += L(pn + uu) (mode 1), as k_residual.
__device__ void b_residual(const BGrid &B, const float *uu, float *out, int mode) {
    const int n = B.n, m = B.m;
    b_G(B, uu);
    const Map2 M = map_for(m);
    FOR_CELLS(M, n, m, i, j) {
        const int q = i * m + j;
        const bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
        const int oS = hS ? q + m : q, oN = hN ? q - m : q, oE = hE ? q + 1 : q, oW = hW ? q - 1 : q;
        const float gc = B.G[q];
        const float aS = face(gc, B.G[oS], hS), aN = face(gc, B.G[oN], hN);
        const float aE = face(gc, B.G[oE], hE), aW = face(gc, B.G[oW], hW);
        const float pc = B.pn[q], uc = uu[q];
        float fl = mul_rn(aS, add_rn(sub_rn(B.pn[oS], pc), sub_rn(uu[oS], uc)));
        fl = fma_rn(aN, add_rn(sub_rn(B.pn[oN], pc), sub_rn(uu[oN], uc)), fl);
        fl = fma_rn(aE, add_rn(sub_rn(B.pn[oE], pc), sub_rn(uu[oE], uc)), fl);
        fl = fma_rn(aW, add_rn(sub_rn(B.pn[oW], pc), sub_rn(uu[oW], uc)), fl);
        const float Lv = sub_rn(fma_rn(B.cdiff, fl, -add_rn(B.F[q], 0.0f)), mul_rn(B.inv_tau, uc));
        if (mode == 0) stc(out, q, (size_t)n * m, kDbgBottom, B.has_rhs ? sub_rn(B.rhs[q], Lv) : -Lv);
        else stc(out, q, (size_t)n * m, kDbgBottom, add_rn(out[q], Lv));
    }
    __syncthreads();
}

__device__ __forceinline__ int fw(int I, int n, int *idx, float *wt) {
    const int q = 2 * I + 1;
    if (q + 1 < n) { idx[0] = q - 1; idx[1] = q; idx[2] = q + 1; wt[0] = 0.25f; wt[1] = 0.5f; wt[2] = 0.25f; return 3; }
    idx[0] = q - 1; idx[1] = q; wt[0] = 0.5f; wt[1] = 0.5f;
    return 2;
}

__device__ __forceinline__ int bl(int p, int nc, int *idx, float *wt) {
    if (p & 1) { idx[0] = (p - 1) / 2; wt[0] = 1.0f; return 1; }
    if (p == 0) { idx[0] = 0; wt[0] = 1.0f; return 1; }
    const int I = p / 2 - 1;
    if (I + 1 < nc) { idx[0] = I; idx[1] = I + 1; wt[0] = 0.5f; wt[1] = 0.5f; return 2; }
    idx[0] = I; wt[0] = 1.0f;
    return 1;
}

// Full weighting of `src` (fine grid F) into dst (and dst2) on the coarse grid C, as k_restrict.
__device__ void b_restrict(const BGrid &F, const float *src, const BGrid &C, float *dst, float *dst2) {
    const Map2 M = map_for(C.m);
    FOR_CELLS(M, C.n, C.m, I, J) {
        int ri[3], ci[3];
        float rw[3], cw[3];
        const int nr = fw(I, F.n, ri, rw), nk = fw(J, F.m, ci, cw);
        float s = 0.f;
        for (int a = 0; a < nr; ++a) {
            float row = 0.f;
            for (int b = 0; b < nk; ++b)
                row = fma_rn((float)cw[b], ldc(src, (size_t)ri[a] * F.m + ci[b], (size_t)F.n * F.m, kDbgBottom), row);
            s = fma_rn((float)rw[a], row, s);
        }
        const int q = I * C.m + J;
        stc(dst, q, (size_t)C.n * C.m, kDbgBottom, s);
        if (dst2) stc(dst2, q, (size_t)C.n * C.m, kDbgBottom, s);
    }
    __syncthreads();
}

// fine.u += P (coarse.u - coarse.u0), as k_interp_add.
__device__ void b_interp_add(const BGrid &F, const BGrid &C) {
    const Map2 M = map_for(F.m);
    FOR_CELLS(M, F.n, F.m, i, j) {
        int ri[2], ci[2];
        float rw[2], cw[2];
        const int nr = bl(i, C.n, ri, rw), nk = bl(j, C.m, ci, cw);
        float s = 0.f;
        for (int a = 0; a < nr; ++a)
            for (int b = 0; b < nk; ++b) {
                const int o = ri[a] * C.m + ci[b];
                const size_t lc = (size_t)C.n * C.m;
                s = fma_rn((float)(rw[a] * cw[b]), sub_rn(ldc(C.u, o, lc, kDbgBottom), ldc(C.u0, o, lc, kDbgBottom)), s);
            }
        const int q = i * F.m + j;
        stc(F.u, q, (size_t)F.n * F.m, kDbgBottom, add_rn(F.u[q], s));
    }
    __syncthreads();
}

}  // namespace

// Shared-memory bytes the bottom kernel needs for grids lb .. L-1.
size_t bottom_smem_bytes(const int *n, const int *m, int lb, int L, int coarse_fp64) {
    size_t b = 0;
    int maxN = 0, maxTask = 0;
    for (int l = lb; l < L; ++l) {
        const size_t N = (size_t)n[l] * m[l];
        const int npm = (m[l] + 31) / 32, npn = (n[l] + 31) / 32;
        b += 8 * N * sizeof(float);
        b += sizeof(uint32_t) * (2 * (size_t)n[l] * npm + 2 * (size_t)m[l] * npn);
        maxN = std::max(maxN, (int)N);
        maxTask = std::max(maxTask, std::max((n[l] + 1) / 2 * npm, (m[l] + 1) / 2 * npn));
    }
    b += (size_t)maxN;                                   // star bytes
    b = (b + 15) / 16 * 16;
    b += sizeof(float) * 2 * (size_t)maxTask;           // end values
    b = (b + 15) / 16 * 16;
    b += (coarse_fp64 ? sizeof(double) : sizeof(float)) * coarse_scratch_elems(n[L - 1], m[L - 1]);
    return b;
}

// The sub-cycle from grid lb (its u and rhs already in shared memory) down to the coarsest and
// back, run by the whole block: smoothing, residual, restriction, coarse right-hand side, the
// coarsest solve, interpolation, post-smoothing (Algorithm 1).
__device__ void bottom_subcycle(const BottomArgs &A, BGrid *Bs, int lb, uint8_t *star, float *endv,
                                unsigned char *scratch, double *red, int *s_err) {
    auto smooth = [&](int l) {
        if (Bs[l].n * Bs[l].m <= kBT) {
            b_smooth_small(Bs[l], star, endv);
        } else {
            b_snapshot(Bs[l], star);
            for (int k = 0; k < 4; ++k) b_sweep(Bs[l], k, endv);
        }
    };
    // ---- down: smoothing, residual, restriction, coarse right-hand side (Algorithm 1)
    for (int l = lb; l < A.L - 1; ++l) {
        for (int t = 0; t < A.nu1; ++t) smooth(l);
        b_residual(Bs[l], Bs[l].u, Bs[l].f, 0);
        b_restrict(Bs[l], Bs[l].f, Bs[l + 1], Bs[l + 1].rhs, nullptr);
        b_restrict(Bs[l], Bs[l].u, Bs[l + 1], Bs[l + 1].u, Bs[l + 1].u0);
        b_residual(Bs[l + 1], Bs[l + 1].u0, Bs[l + 1].rhs, 1);
    }
    // ---- the coarsest solve
    {
        const BGrid &C = Bs[A.L - 1];
        CoarseGrid<float> cg{C.n, C.m, C.m, C.pn, C.u, C.w, nullptr, C.F, C.rhs, C.has_rhs, C.inv_2h, C.inv_tau, C.beta};
        int it;
        double res;
        if (A.coarse_fp64)
            coarse_solve_block<float, double>(cg, A.mp, A.sc->A1frac, A.h2nm_coarse, A.coarse_maxit, A.coarse_tol,
                                              reinterpret_cast<double *>(scratch), red, s_err, &it, &res,
                                              A.coarse_aos, A.aos_dt);
        else
            coarse_solve_block<float, float>(cg, A.mp, A.sc->A1frac, A.h2nm_coarse, A.coarse_maxit, A.coarse_tol,
                                             reinterpret_cast<float *>(scratch), red, s_err, &it, &res,
                                             A.coarse_aos, A.aos_dt);
        if (threadIdx.x == 0) {
            A.sc->picard = it;
            A.sc->coarse_res = res;
            if (*s_err) A.sc->err = 1;
        }
    }
    // ---- up: interpolation and post-smoothing
    for (int l = A.L - 2; l >= lb; --l) {
        b_interp_add(Bs[l], Bs[l + 1]);
        for (int t = 0; t < A.nu2; ++t) smooth(l);
    }
}

// Carves the shared memory of grids lb .. L-1 (thread 0) and loads pn, w and F of every grid and,
// when load_first, u and rhs of grid lb.  s_off: star bytes, end values, coarsest-solve scratch.
__device__ void bottom_setup(const BottomArgs &A, BGrid *Bs, int lb, bool load_first, unsigned char *sm,
                             size_t *s_off) {
    if (threadIdx.x == 0) {
        size_t off = 0;
        int maxN = 0, maxTask = 0;
        for (int l = lb; l < A.L; ++l) {
            const LevelView<float> &G = A.g[l];
            BGrid &B = Bs[l];
            B.n = G.n; B.m = G.m; B.npm = (G.m + 31) / 32; B.npn = (G.n + 31) / 32;
            B.cdiff = G.cdiff; B.inv_tau = G.inv_tau; B.Sigma = G.Sigma; B.inv_2h = G.inv_2h; B.beta = G.beta;
            B.has_rhs = G.has_rhs;
            const int N = G.n * G.m;
            float **arr[] = {&B.pn, &B.u, &B.w, &B.F, &B.rhs, &B.G, &B.f, &B.u0};
            for (float **a : arr) { *a = reinterpret_cast<float *>(sm + off); off += sizeof(float) * N; }
            B.mrow = reinterpret_cast<uint32_t *>(sm + off); off += sizeof(uint32_t) * 2 * (size_t)G.n * B.npm;
            B.mcol = reinterpret_cast<uint32_t *>(sm + off); off += sizeof(uint32_t) * 2 * (size_t)G.m * B.npn;
            maxN = max(maxN, N);
            maxTask = max(maxTask, max((G.n + 1) / 2 * B.npm, (G.m + 1) / 2 * B.npn));
        }
        s_off[0] = off;                                 // star bytes
        off += maxN;
        off = (off + 15) / 16 * 16;
        s_off[1] = off;                                 // end values
        off += sizeof(float) * 2 * maxTask;
        off = (off + 15) / 16 * 16;
        s_off[2] = off;                                 // coarsest-solve scratch
    }
    __syncthreads();
    for (int l = lb; l < A.L; ++l) {
        const LevelView<float> &G = A.g[l];
        const BGrid &B = Bs[l];
        const Map2 M = map_for(B.m);
        FOR_CELLS(M, B.n, B.m, i, j) {
            const int q = i * B.m + j;
            const size_t o = (size_t)i * G.pitch + j, lim = (size_t)G.n * G.pitch;
            B.pn[q] = ldc(G.pn, o, lim, kDbgBottom);
            B.w[q] = weight_at(G, o);
            B.F[q] = ldc(G.F, o, lim, kDbgBottom);
            if (load_first && l == lb) {
                B.u[q] = ldc(G.u, o, lim, kDbgBottom);
                B.rhs[q] = G.has_rhs ? ldc(G.rhs, o, lim, kDbgBottom) : 0.f;
            }
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBT) k_bottom(BottomArgs A) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red[33];
    __shared__ int s_err;
    __shared__ BGrid Bs[kMaxLevels];
    __shared__ size_t s_off[3];
    bottom_setup(A, Bs, A.lb, true, sm, s_off);
    uint8_t *star = sm + s_off[0];
    float *endv = reinterpret_cast<float *>(sm + s_off[1]);
    __syncthreads();
    bottom_subcycle(A, Bs, A.lb, star, endv, sm + s_off[2], red, &s_err);
    // ---- grid lb's increment back to global memory
    {
        const LevelView<float> &G = A.g[A.lb];
        const BGrid &B = Bs[A.lb];
        const Map2 M = map_for(B.m);
        FOR_CELLS(M, B.n, B.m, i, j) stc(G.u, (size_t)i * G.pitch + j, (size_t)G.n * G.pitch, kDbgBottom, B.u[i * B.m + j]);
    }
}

// ---------------------------------------------------------------------------------------
// The bottom of the V-cycle from a grid spread over a thread-block cluster.  On grids of about
// 64^2 every per-grid launch is latency-bound (a V-cycle spends about 23 launches per grid) while
// one block is too little for the grid.  Here one 1024-thread CTA owns each 32 x 32 tile of grid
// lc (one cell per thread, at most 16 tiles: one cluster) in its shared memory, pn, u and G with
// a ring of the neighbouring tiles' edge cells, so every phase computes from local shared
// memory.  A thread that changes an edge cell also stores the value into the rings of the
// neighbouring tiles (distributed shared memory); the cluster barrier after the phase publishes
// it.  The store may land while a neighbour is still in the same phase: a checkerboard phase's
// neighbours read only cells of the other colour, and a partial-line phase's neighbours read
// only lines of the other parity, except for the end values of their own pieces, which every CTA
// reads before a barrier at the start of the phase.  CTA 0 also holds grids
// lc+1 .. L-1 and runs their sub-cycle (bottom_subcycle) between the restriction and the
// interpolation.  Every cell performs the per-grid kernels' operations, so the results are the
// same.
// ---------------------------------------------------------------------------------------
constexpr int kHP = 34;   // the 32 x 32 tile and its ring

struct CTile {
    float P[kHP][kHP], U[kHP][kHP], G[kHP][kHP];            // pn, u, G; tile cell (a, b) at [a + 1][b + 1]
    float W[32][32], F[32][32], R[32][32], Fv[32][32], Res[32][32];   // w, F, rhs, f, residual
    uint32_t mrow[2][32];   // sweeps A, B: the piece of tile row r
    uint32_t mcol[2][32];   // sweeps C, D: the piece of tile column c
    uint8_t star[32][33];
    unsigned any;           // bit k: a member cell of sweep k in this tile
};
constexpr size_t kTileBytes = (sizeof(CTile) + 127) / 128 * 128;

__global__ void __launch_bounds__(kBT) k_cluster(BottomArgs A) {
    namespace cgc = cooperative_groups;
    cgc::cluster_group cl = cgc::this_cluster();
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red[33];
    __shared__ int s_err;
    __shared__ BGrid Bs[kMaxLevels];
    __shared__ size_t s_off[3];
    __shared__ CTile *tp[16];
    CTile &T = *reinterpret_cast<CTile *>(sm);
    const int lc = A.lb;
    const LevelView<float> &Lg = A.g[lc];
    const int n = Lg.n, m = Lg.m, TX = (m + 31) / 32;
    const float cdiff = Lg.cdiff, inv_tau = Lg.inv_tau, Sigma = Lg.Sigma, inv_2h = Lg.inv_2h, beta = Lg.beta;
    const bool has_rhs = Lg.has_rhs != 0;
    const int rank = (int)cl.block_rank();
    const int ty = rank / TX, tx = rank - ty * TX, i0 = ty * 32, j0 = tx * 32;
    const int q = threadIdx.x, ti = q >> 5, lane = q & 31;
    const int i = i0 + ti, j = j0 + lane;
    const bool own = i < n && j < m;
    if (q < (int)cl.num_blocks()) tp[q] = cl.map_shared_rank(&T, q);
    // padded row / column of grid row / column a, clamped into the grid (the mirror ghosts)
    auto pr = [&](int a) { return min(max(a, 0), n - 1) - i0 + 1; };
    auto pc = [&](int b) { return min(max(b, 0), m - 1) - j0 + 1; };
    const int r0 = ti + 1, c0 = lane + 1, rS = pr(i + 1), rN = pr(i - 1), cE = pc(j + 1), cW = pc(j - 1);
    // field f (0: pn, 1: u, 2: G) of a tile
    auto field = [&](CTile *t, int f) -> float (*)[kHP] { return f == 0 ? t->P : (f == 1 ? t->U : t->G); };
    // value v of tile cell (a, b) of field f into the rings of the neighbouring tiles that hold it
    // (a cell on the tile's edge; a remote store: the cluster barrier that follows publishes it)
    auto push = [&](int f, int a, int b, float v) {
        if (a == 0 && i0 > 0) field(tp[rank - TX], f)[33][b + 1] = v;
        if (a == 31 && i0 + 32 < n) field(tp[rank + TX], f)[0][b + 1] = v;
        if (b == 0 && j0 > 0) field(tp[rank - 1], f)[a + 1][33] = v;
        if (b == 31 && j0 + 32 < m) field(tp[rank + 1], f)[a + 1][0] = v;
    };
    if (own) {
        const size_t o = (size_t)i * Lg.pitch + j, lim = (size_t)n * Lg.pitch;
        T.P[r0][c0] = ldc(Lg.pn, o, lim, kDbgBottom);
        T.U[r0][c0] = ldc(Lg.u, o, lim, kDbgBottom);
        T.W[ti][lane] = weight_at(Lg, o);
        T.F[ti][lane] = ldc(Lg.F, o, lim, kDbgBottom);
        T.R[ti][lane] = has_rhs ? ldc(Lg.rhs, o, lim, kDbgBottom) : 0.f;
    }
    // grids lc+1 .. L-1: every CTA carves the same offsets (CTA 0's arrays are then reached by
    // mapping this CTA's addresses); their pn, w, F are loaded
    bottom_setup(A, Bs, lc + 1, false, sm + kTileBytes, s_off);
    cl.sync();   // every CTA of the cluster runs: its shared memory may be written
    if (own) {
        push(0, ti, lane, T.P[r0][c0]);
        push(1, ti, lane, T.U[r0][c0]);
    }
    cl.sync();
    auto g_phase = [&]() {   // G at pn + u of the own cell, into the neighbours' rings
        if (own) {
            const float g = cell_G(T.W[ti][lane], T.P[rS][c0], T.P[rN][c0], T.P[r0][cE], T.P[r0][cW], T.U[rS][c0],
                                   T.U[rN][c0], T.U[r0][cE], T.U[r0][cW], inv_2h, beta);
            T.G[r0][c0] = g;
            push(2, ti, lane, g);
        }
        cl.sync();
    };
    const bool hS = i + 1 < n, hN = i > 0, hE = j + 1 < m, hW = j > 0;
    const int colour = (i + j) & 1;
    // ---- one outer smoothing iteration (snapshot and four sweeps)
    auto smooth = [&]() {
        g_phase();
        float aS = 0.f, aN = 0.f, aE = 0.f, aW = 0.f, dv = 1.f, fq = 0.f;
        uint32_t star = 0;
        if (own) {
            const float gc = T.G[r0][c0];
            aS = face(gc, T.G[rS][c0], hS); aN = face(gc, T.G[rN][c0], hN);
            aE = face(gc, T.G[r0][cE], hE); aW = face(gc, T.G[r0][cW], hW);
            const float pcv = T.P[r0][c0];
            float ds = mul_rn(aS, sub_rn(T.P[rS][c0], pcv));
            ds = fma_rn(aN, sub_rn(T.P[rN][c0], pcv), ds);
            ds = fma_rn(aE, sub_rn(T.P[r0][cE], pcv), ds);
            ds = fma_rn(aW, sub_rn(T.P[r0][cW], pcv), ds);
            float base = add_rn(T.F[ti][lane], 0.0f);
            if (has_rhs) base = add_rn(base, T.R[ti][lane]);
            fq = fma_rn(-cdiff, ds, base);
            T.Fv[ti][lane] = fq;
            const float big = 3.0e38f;
            const float vS = hS ? aS : big, vN = hN ? aN : big, vE = hE ? aE : big, vW = hW ? aW : big;
            const float mn = fminf(fminf(vS, vN), fminf(vE, vW));
            const float mx = fmaxf(fmaxf(hS ? aS : -1.f, hN ? aN : -1.f), fmaxf(hE ? aE : -1.f, hW ? aW : -1.f));
            const int am = vS == mn ? 0 : (vN == mn ? 1 : (vE == mn ? 2 : 3));
            const int cnt = (int)hS + (int)hN + (int)hE + (int)hW;
            star = (cnt >= 2 && mx > mul_rn(Sigma, mn)) ? (1u << am) : 0u;
            dv = fma_rn(cdiff, add_rn(add_rn(aS, aN), add_rn(aE, aW)), inv_tau);
        }
        // member masks of the tile's pieces: row ti (this warp) and column ti
        T.star[ti][lane] = (uint8_t)star;
        const int lenr = min(32, m - j0), lenc = min(32, n - i0);
        const uint32_t mA = members_of(__ballot_sync(0xffffffffu, star & 1u), lenr);
        const uint32_t mB = members_of(__ballot_sync(0xffffffffu, star & 2u), lenr);
        if (lane == 0) { T.mrow[0][ti] = mA; T.mrow[1][ti] = mB; }
        __syncthreads();
        const uint8_t sc = T.star[lane][ti];
        const uint32_t mC = members_of(__ballot_sync(0xffffffffu, sc & 4u), lenc);
        const uint32_t mD = members_of(__ballot_sync(0xffffffffu, sc & 8u), lenc);
        if (lane == 0) { T.mcol[0][ti] = mC; T.mcol[1][ti] = mD; }
        __syncthreads();
        unsigned mem = 0;
        if (own) {
            mem |= (T.mrow[0][ti] >> lane) & 1u;
            mem |= ((T.mrow[1][ti] >> lane) & 1u) << 1;
            mem |= ((T.mcol[0][lane] >> ti) & 1u) << 2;
            mem |= ((T.mcol[1][lane] >> ti) & 1u) << 3;
        }
        if (q < 32) {
            const unsigned a = (T.mrow[0][q] ? 1u : 0u) | (T.mrow[1][q] ? 2u : 0u) | (T.mcol[0][q] ? 4u : 0u) |
                               (T.mcol[1][q] ? 8u : 0u);
            const unsigned r = __reduce_or_sync(0xffffffffu, a);
            if (q == 0) T.any = r;
        }
        unsigned any = 0;   // every tile's bits, read after the first checkerboard phase's barrier
        for (int k = 0; k < 4; ++k) {
            const bool rev = k & 1, rowwise = k < 2;
            for (int ph = 0; ph < 2; ++ph) {
                if (own && colour == (rev ? 1 - ph : ph) && !((mem >> k) & 1u)) {
                    float num = mul_rn(aS, T.U[rS][c0]);
                    num = fma_rn(aN, T.U[rN][c0], num);
                    num = fma_rn(aE, T.U[r0][cE], num);
                    num = fma_rn(aW, T.U[r0][cW], num);
                    const float v = div_relax(fma_rn(cdiff, num, -fq), dv);
                    T.U[r0][c0] = v;
                    // the neighbours read only the other colour in this phase: the push can go now
                    push(1, ti, lane, v);
                }
                cl.sync();
                if (k == 0 && ph == 0)
                    for (int r = 0; r < (int)cl.num_blocks(); ++r) any |= tp[r]->any;
            }
            if (!((any >> k) & 1u)) continue;
            // partial-line phases: warp ti owns tile row ti (rowwise) or tile column ti
            for (int ph = 0; ph < 2; ++ph) {
                const int parity = rev ? 1 - ph : ph;
                const int gl = (rowwise ? i0 : j0) + ti, llen = rowwise ? m : n, t0 = rowwise ? j0 : i0;
                const int len = min(32, llen - t0);
                const bool ok = gl < (rowwise ? n : m) && (gl & 1) == parity;
                const uint32_t mk = ok ? (rowwise ? T.mrow[k][ti] : T.mcol[k - 2][ti]) : 0u;
                // the end values (the neighbouring tiles' cells of this line) as the phase starts,
                // read before the barrier after which this phase's pushes may overwrite them
                float e0 = 0.f, e1 = 0.f;
                if (mk) {
                    if (t0 > 0) e0 = rowwise ? T.U[r0][0] : T.U[0][r0];
                    if (t0 + len < llen) e1 = rowwise ? T.U[r0][len + 1] : T.U[len + 1][r0];
                }
                cl.sync();
                if (mk) {
                    float ownv = 0.f;
                    if (lane < len) ownv = rowwise ? T.U[r0][lane + 1] : T.U[lane + 1][r0];
                    __syncwarp();
                    auto at = [&](int r) -> RunCell<float> {
                        const int ci = rowwise ? gl : t0 + r, cj = rowwise ? t0 + r : gl;
                        const int a = ci - i0 + 1, b = cj - j0 + 1;
                        const int aS2 = pr(ci + 1), aN2 = pr(ci - 1), bE2 = pc(cj + 1), bW2 = pc(cj - 1);
                        const bool cS = ci + 1 < n, cN = ci > 0, cE2 = cj + 1 < m, cW2 = cj > 0;
                        const float gc = T.G[a][b];
                        const float bS = face(gc, T.G[aS2][b], cS), bN = face(gc, T.G[aN2][b], cN);
                        const float bE = face(gc, T.G[a][bE2], cE2), bW = face(gc, T.G[a][bW2], cW2);
                        RunCell<float> c;
                        if (rowwise) { c.ap = bW; c.an = bE; c.ax1 = bS; c.ax2 = bN; c.ux1 = T.U[aS2][b]; c.ux2 = T.U[aN2][b]; }
                        else         { c.ap = bN; c.an = bS; c.ax1 = bE; c.ax2 = bW; c.ux1 = T.U[a][bE2]; c.ux2 = T.U[a][bW2]; }
                        c.f = T.Fv[a - 1][b - 1];
                        return c;
                    };
                    float x;
                    if (pcr_piece<float>(mk, len, cdiff, inv_tau, ownv, e0, e1, at, x)) {
                        // the neighbours read only lines of the other parity in this phase
                        if (rowwise) {
                            T.U[r0][lane + 1] = x;
                            push(1, ti, lane, x);
                        } else {
                            T.U[lane + 1][r0] = x;
                            push(1, lane, ti, x);
                        }
                    }
                }
                cl.sync();
            }
        }
    };
    for (int t = 0; t < A.nu1; ++t) smooth();
    // ---- residual r = rhs - L(pn + u) of the own cell (as b_residual, mode 0)
    g_phase();
    if (own) {
        const float gc = T.G[r0][c0];
        const float aS = face(gc, T.G[rS][c0], hS), aN = face(gc, T.G[rN][c0], hN);
        const float aE = face(gc, T.G[r0][cE], hE), aW = face(gc, T.G[r0][cW], hW);
        const float pcv = T.P[r0][c0], uc = T.U[r0][c0];
        float fl = mul_rn(aS, add_rn(sub_rn(T.P[rS][c0], pcv), sub_rn(T.U[rS][c0], uc)));
        fl = fma_rn(aN, add_rn(sub_rn(T.P[rN][c0], pcv), sub_rn(T.U[rN][c0], uc)), fl);
        fl = fma_rn(aE, add_rn(sub_rn(T.P[r0][cE], pcv), sub_rn(T.U[r0][cE], uc)), fl);
        fl = fma_rn(aW, add_rn(sub_rn(T.P[r0][cW], pcv), sub_rn(T.U[r0][cW], uc)), fl);
        const float Lv = sub_rn(fma_rn(cdiff, fl, -add_rn(T.F[ti][lane], 0.0f)), mul_rn(inv_tau, uc));
        T.Res[ti][lane] = has_rhs ? sub_rn(T.R[ti][lane], Lv) : -Lv;
    }
    cl.sync();
    // ---- CTA 0: restriction of the residual and of u (as b_restrict), the coarse right-hand
    // side, and the sub-cycle of grids lc+1 .. L-1
    if (rank == 0) {
        const BGrid &C = Bs[lc + 1];
        auto fine = [&](bool res, int a, int b) -> float {   // a fine cell inside the grid
            const CTile *t = tp[(a >> 5) * TX + (b >> 5)];
            return res ? t->Res[a & 31][b & 31] : t->U[(a & 31) + 1][(b & 31) + 1];
        };
        const Map2 M = map_for(C.m);
        FOR_CELLS(M, C.n, C.m, I, J) {
            int ri[3], ci[3];
            float rw[3], cw[3];
            const int nr = fw(I, n, ri, rw), nk = fw(J, m, ci, cw);
            float sr = 0.f, su = 0.f;
            for (int a = 0; a < nr; ++a) {
                float rr = 0.f, ru = 0.f;
                for (int b = 0; b < nk; ++b) {
                    rr = fma_rn((float)cw[b], fine(true, ri[a], ci[b]), rr);
                    ru = fma_rn((float)cw[b], fine(false, ri[a], ci[b]), ru);
                }
                sr = fma_rn((float)rw[a], rr, sr);
                su = fma_rn((float)rw[a], ru, su);
            }
            const int o = I * C.m + J;
            C.rhs[o] = sr;
            C.u[o] = su;
            C.u0[o] = su;
        }
        __syncthreads();
        b_residual(C, C.u0, C.rhs, 1);
        bottom_subcycle(A, Bs, lc + 1, sm + kTileBytes + s_off[0],
                        reinterpret_cast<float *>(sm + kTileBytes + s_off[1]), sm + kTileBytes + s_off[2], red,
                        &s_err);
    }
    cl.sync();
    // ---- interpolation of CTA 0's coarse correction (as b_interp_add)
    {
        const BGrid &C = Bs[lc + 1];
        const float *Cu = cl.map_shared_rank(C.u, 0), *Cu0 = cl.map_shared_rank(C.u0, 0);
        if (own) {
            int ri[2], ci[2];
            float rw[2], cw[2];
            const int nr = bl(i, C.n, ri, rw), nk = bl(j, C.m, ci, cw);
            float sum = 0.f;
            for (int a = 0; a < nr; ++a)
                for (int b = 0; b < nk; ++b) {
                    const int o = ri[a] * C.m + ci[b];
                    sum = fma_rn((float)(rw[a] * cw[b]), sub_rn(Cu[o], Cu0[o]), sum);
                }
            const float v = add_rn(T.U[r0][c0], sum);
            T.U[r0][c0] = v;
            push(1, ti, lane, v);
        }
    }
    cl.sync();
    for (int t = 0; t < A.nu2; ++t) smooth();
    if (own) stc(Lg.u, (size_t)i * Lg.pitch + j, (size_t)n * Lg.pitch, kDbgBottom, T.U[r0][c0]);
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

void prepare_bottom_kernel() {
    cudaFuncSetAttribute(k_bottom, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBottomSmemMax);
    // a refused attribute leaves the cluster kernel unusable: cluster_fits then reports no fit
    if (cudaFuncSetAttribute(k_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmemMax) != cudaSuccess ||
        cudaFuncSetAttribute(k_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        cudaGetLastError();
}

void launch_bottom(const BottomArgs &A, size_t smem, cudaStream_t st) {
    k_bottom<<<1, kBT, smem, st>>>(A);
}

size_t cluster_smem_bytes(size_t bottom_bytes) { return kTileBytes + bottom_bytes; }

int cluster_fits(int tiles, size_t smem) {
    if (tiles < 1 || tiles > kClusterMaxTiles || smem > kClusterSmemMax) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = tiles;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, k_cluster, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();   // the query's error is reported through the return value
        return -(int)e;
    }
    return nc;
}

void launch_cluster(const BottomArgs &A, int tiles, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = tiles;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_cluster, A);
}

}  // namespace segmg
