// line_phase.cuh -- the two partial-line phases of one fused-sweep tile (Sec. 4.3, step III).
//
// A fused sweep smooths a tile held in shared memory: the output tile plus a halo of KH cells.
// After its two checkerboard phases come two zebra phases of partial lines: the lines at
// distance 1 from the output tile, then those at distance 0, one line parity each; each line is
// cut into the tile's 32-cell pieces, and the runs of member cells of a piece are solved exactly
// (pcr_piece).  Pieces of one line are coupled only through their end values at the start of
// the phase, so one warp owns a line: it reads the end values of all the line's pieces, then
// solves the pieces one after another, and no block barrier is needed inside a phase.
#pragma once

#include "arith.cuh"

namespace segmg {

// U(a, b): reference to box cell (row a, column b) of u;  Gc, Fc: values of G and f;
// MK(line, pc): member mask of piece pc (0 .. OW/32 - 1 rowwise, OH/32 - 1 columnwise) of box
// line `line` (a box row rowwise, a box column columnwise).  Ends with a block barrier.
template <typename T, int KH, int OH, int OW, int NT, bool ROWWISE, bool REV, class UA, class GA, class FA, class MA>
__device__ __forceinline__ void tile_line_phases(UA U, GA Gc, FA Fc, MA MK, int i0, int j0, int n, int m, T cdiff,
                                                 T inv_tau) {
    constexpr int npc = ROWWISE ? OW / 32 : OH / 32, NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int len_lim = ROWWISE ? m : n, gl_lim = ROWWISE ? n : m;
    const int pbase = ROWWISE ? j0 : i0;                 // grid position of the first piece
    const int lbase = (ROWWISE ? i0 : j0) - KH;          // grid line of box line 0
#pragma unroll
    for (int ph = 0; ph < 2; ++ph) {
        const int parity = REV ? 1 - ph : ph, dist = 1 - ph;
        const int lfirst = KH - dist, nlines = (ROWWISE ? OH : OW) + 2 * dist;
        // the box lines of this phase's parity: lfirst + off, lfirst + off + 2, ...
        const int off = ((lbase + lfirst) & 1) != parity ? 1 : 0;
        for (int k = warp; off + 2 * k < nlines; k += NW) {
            const int li = lfirst + off + 2 * k, gline = lbase + li;
            if (gline < 0 || gline >= gl_lim) continue;
            T e0 = T(0), e1 = T(0);                      // lane pc: the end values of piece pc
            if (lane < npc) {
                const int gstart = pbase + 32 * lane;
                if (gstart < len_lim && MK(li, lane)) {
                    const int len = min(32, len_lim - gstart), s0 = KH + 32 * lane;
                    if (gstart > 0) e0 = ROWWISE ? U(li, s0 - 1) : U(s0 - 1, li);
                    if (gstart + len < len_lim) e1 = ROWWISE ? U(li, s0 + len) : U(s0 + len, li);
                }
            }
            __syncwarp();
            for (int pc = 0; pc < npc; ++pc) {
                const int gstart = pbase + 32 * pc;
                if (gstart >= len_lim) break;
                const uint32_t mk = MK(li, pc);
                if (!mk) continue;
                const T endp = __shfl_sync(0xffffffffu, e0, pc), endn = __shfl_sync(0xffffffffu, e1, pc);
                const int len = min(32, len_lim - gstart), s0 = KH + 32 * pc, pos = s0 + lane;
                const T own = lane < len ? (ROWWISE ? U(li, pos) : U(pos, li)) : T(0);
                auto at = [&](int t) -> RunCell<T> {
                    const int a = ROWWISE ? li : s0 + t, b = ROWWISE ? s0 + t : li;
                    const int gi = i0 - KH + a, gj = j0 - KH + b;
                    const bool hS = gi + 1 < n, hN = gi > 0, hE = gj + 1 < m, hW = gj > 0;
                    const T gc = Gc(a, b);
                    const T aS = face(gc, Gc(a + 1, b), hS), aN = face(gc, Gc(a - 1, b), hN);
                    const T aE = face(gc, Gc(a, b + 1), hE), aW = face(gc, Gc(a, b - 1), hW);
                    RunCell<T> c;
                    if (ROWWISE) {
                        c.ap = aW; c.an = aE; c.ax1 = aS; c.ax2 = aN;
                        c.ux1 = U(a + 1, b); c.ux2 = U(a - 1, b);
                    } else {
                        c.ap = aN; c.an = aS; c.ax1 = aE; c.ax2 = aW;
                        c.ux1 = U(a, b + 1); c.ux2 = U(a, b - 1);
                    }
                    c.f = Fc(a, b);
                    return c;
                };
                T x;
                if (pcr_piece<T>(mk, len, cdiff, inv_tau, own, endp, endn, at, x)) {
                    if (ROWWISE) U(li, pos) = x; else U(pos, li) = x;
                }
            }
        }
        __syncthreads();
    }
}

// Whether any piece the line phases of a tile solve has a member cell: box line `line`, mask
// word pw of the tile's staged masks (word 0 and the last word belong to the neighbouring tiles'
// pieces).  Threads OR this over the words they stage; the block then skips both line phases
// when no thread saw a member.
template <int KH, int OH, int OW, bool ROWWISE>
__device__ __forceinline__ bool solves_word(int line, int pw, uint32_t w) {
    constexpr int npc = ROWWISE ? OW / 32 : OH / 32, nl = ROWWISE ? OH : OW;
    return w != 0u && line >= KH - 1 && line <= KH + nl && pw >= 1 && pw <= npc;
}

}  // namespace segmg
