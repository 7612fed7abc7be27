// line_smoothers.cu -- the paper's other two smoothers on the GPU: GSLINE-I (Sec. 3.2, the
// smoother of Algorithm 1) and Hybrid Smoother 1 (Sec. 4.2, Algorithm 2), in parallel orderings.
//
// GSLINE-I: every column is one tridiagonal system (eq. system) coupling the column's cells
// through A and B, with C and D terms from the current values.  The columns of one parity are
// not neighbours, so all even columns are solved at once, then all odd ones (zebra); one thread
// solves one whole column by the Thomas algorithm, streaming down the rows, with the eliminated
// diagonal and right-hand side kept in two scratch grids.
//
// Hybrid Smoother 1: after GSLINE-I, every cell P of the set D (from the coefficient snapshot:
// class byte = 1 << index of the smallest coefficient) and its neighbours other than the lagged
// one solve their own equations exactly (the arrow systems of eqs. caseAlagged - caseDlagged).
// Cells are visited in 16 classes (i mod 4, j mod 4): two blocks of one class are 4 or more
// cells apart, so neither reads what the other writes, and one launch does one class.
//
// Rows are in the row-scaled form of the solver (divided by delta): the coefficient of
// neighbour X in the row of a cell is mu/h^2 times the face value of G, S is their sum plus
// 1/tau and f is the snapshot's right-hand side.  A face on the domain boundary is zero.
#include "arith.cuh"

namespace segmg {

namespace {

// ---------------------------------------------------------------------------------------
// GSLINE-I, one parity of columns.  dg / rg: scratch for the eliminated diagonal and
// right-hand side of every cell of the column (pitched like the grid).
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_gsline(LevelView<T> L, int parity, T *__restrict__ dg, T *__restrict__ rg) {
    constexpr int R = 8;   // rows whose inputs are loaded together before their recurrence steps
    const int j = parity + 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int n = L.n, m = L.m, p = L.pitch;
    if (j >= m) return;
    const bool hE = j + 1 < m, hW = j > 0;
    const T *__restrict__ G = L.G;
    const T *__restrict__ U = L.u;   // the neighbouring columns (the other parity) are only read
    const T *__restrict__ F = L.f;
    T cup_prev = T(0), cdi_prev = T(1), crh_prev = T(0);
    T g_next = __ldg(G + j);           // G of the row after the previous chunk's last row
    for (int i0 = 0; i0 < n; i0 += R) {
        T g[R + 1], gE[R], gW[R], uE[R], uW[R], f[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r;
            if (i < n) {
                const size_t o = (size_t)i * p + j;
                gE[r] = __ldg(G + (hE ? o + 1 : o));
                gW[r] = __ldg(G + (hW ? o - 1 : o));
                uE[r] = __ldg(U + (hE ? o + 1 : o));
                uW[r] = __ldg(U + (hW ? o - 1 : o));
                f[r] = __ldg(F + o);
                g[r + 1] = i + 1 < n ? __ldg(G + o + p) : T(0);
            }
        }
        g[0] = g_next;
        T g_up = i0 > 0 ? __ldg(G + (size_t)(i0 - 1) * p + j) : T(0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i0 + r;
            if (i >= n) break;
            const size_t o = (size_t)i * p + j;
            const T gc = g[r];
            const T aS = face(gc, g[r + 1], i + 1 < n), aN = face(gc, g_up, i > 0);
            const T aE = face(gc, gE[r], hE), aW = face(gc, gW[r], hW);
            const T lo = mul_rn(L.cdiff, aN), up = mul_rn(L.cdiff, aS);
            const T sum = add_rn(add_rn(aN, aS), add_rn(aE, aW));
            T di = -fma_rn(L.cdiff, sum, L.inv_tau);
            const T across = fma_rn(aW, uW[r], mul_rn(aE, uE[r]));
            T rhs = fma_rn(-L.cdiff, across, f[r]);
            if (i > 0) {
                const T wgt = div_relax(lo, cdi_prev);
                di = fma_rn(-wgt, cup_prev, di);
                rhs = fma_rn(-wgt, crh_prev, rhs);
            }
            stc(dg, o, (size_t)n * p, kDbgOther, di);
            stc(rg, o, (size_t)n * p, kDbgOther, rhs);
            cup_prev = up;
            cdi_prev = di;
            crh_prev = rhs;
            g_up = gc;
        }
        g_next = g[R < n - i0 ? R : n - i0];
    }
    T x = div_relax(crh_prev, cdi_prev);
    stc(L.u, (size_t)(n - 1) * p + j, (size_t)n * p, kDbgOther, x);
    for (int i1 = n - 2; i1 >= 0; i1 -= R) {
        T gg[R + 1], d[R], rr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i1 - r;
            if (i >= 0) {
                const size_t o = (size_t)i * p + j;
                gg[r] = __ldg(G + o);
                d[r] = dg[o];
                rr[r] = rg[o];
            }
        }
        gg[R] = T(0);
        T g_below = __ldg(G + (size_t)(i1 + 1) * p + j);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = i1 - r;
            if (i < 0) break;
            const T up = mul_rn(L.cdiff, face(gg[r], g_below, true));
            x = div_relax(fma_rn(-up, x, rr[r]), d[r]);
            stc(L.u, (size_t)i * p + j, (size_t)n * p, kDbgOther, x);
            g_below = gg[r];
        }
    }
}

// ---------------------------------------------------------------------------------------
// Hybrid Smoother 1 blocks of one class (ci, cj): cells i = ci + 4I, j = cj + 4J.
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_hs1(LevelView<T> L, int ci, int cj) {
    const int i = ci + 4 * (blockIdx.y * blockDim.y + threadIdx.y);
    const int j = cj + 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int n = L.n, m = L.m, p = L.pitch;
    if (i >= n || j >= m) return;
    const size_t o = (size_t)i * p + j;
    const unsigned cls = L.cls[o];
    if (!cls) return;
    const int lag = __ffs(cls) - 1;                 // 0..3 = A (south), B (north), C (east), D (west)
    const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
    auto inside = [&](int a, int b) { return a >= 0 && a < n && b >= 0 && b < m; };
    // row coefficients of a cell: c[t] = mu/h^2 G_face toward neighbour t (0 if none), S
    auto row = [&](int a, int b, T *c, T &S) {
        const size_t q = (size_t)a * p + b;
        const T gc = L.G[q];
        T s = T(0);
        for (int t = 0; t < 4; ++t) {
            const int a2 = a + di[t], b2 = b + dj[t];
            c[t] = inside(a2, b2) ? L.cdiff * face(gc, L.G[(size_t)a2 * p + b2], true) : T(0);
            s += c[t];
        }
        S = s + L.inv_tau;
    };
    T cP[4], SP;
    row(i, j, cP, SP);
    // P's row: -S_P x_P + sum over leaves c_Pl x_l = f_P - c_P,lag u_lag
    T rP = L.f[o];
    {
        const int a2 = i + di[lag], b2 = j + dj[lag];
        rP -= cP[lag] * L.u[(size_t)a2 * p + b2];
    }
    T num = T(0), den = -SP;
    T rl[4], cl[4], Sl[4];
    bool leaf[4];
    for (int t = 0; t < 4; ++t) {
        const int a = i + di[t], b = j + dj[t];
        leaf[t] = t != lag && inside(a, b);
        if (!leaf[t]) continue;
        T c[4], S;
        row(a, b, c, S);
        const int back = t ^ 1;                     // the direction from the leaf back to P
        T r = L.f[(size_t)a * p + b];
        for (int u = 0; u < 4; ++u) {
            if (u == back || c[u] == T(0)) continue;
            r -= c[u] * L.u[(size_t)(a + di[u]) * p + (b + dj[u])];
        }
        rl[t] = r;
        cl[t] = c[back];
        Sl[t] = S;
        num += cP[t] * r / S;
        den += cP[t] * c[back] / S;
    }
    const T xP = (rP + num) / den;
    stc(L.u, o, (size_t)n * p, kDbgOther, xP);
    for (int t = 0; t < 4; ++t) {
        if (!leaf[t]) continue;
        stc(L.u, (size_t)(i + di[t]) * p + (j + dj[t]), (size_t)n * p, kDbgOther, (cl[t] * xP - rl[t]) / Sl[t]);
    }
}

}  // namespace

template <typename T>
void launch_gsline(const LevelView<T> &L, cudaStream_t st) {
    for (int par = 0; par < 2; ++par) {
        const int cols = (L.m - par + 1) / 2;
        if (cols <= 0) continue;
        k_gsline<T><<<(cols + 127) / 128, 128, 0, st>>>(L, par, L.r, L.t);
    }
}

template <typename T>
void launch_hs1_blocks(const LevelView<T> &L, cudaStream_t st) {
    for (int c = 0; c < 16; ++c) {
        const int ci = c / 4, cj = c % 4;
        const int ni = (L.n - ci + 3) / 4, nj = (L.m - cj + 3) / 4;
        if (ni <= 0 || nj <= 0) continue;
        dim3 block(32, 8), grid((nj + 31) / 32, (ni + 7) / 8);
        k_hs1<T><<<grid, block, 0, st>>>(L, ci, cj);
    }
}

template void launch_gsline<float>(const LevelView<float> &, cudaStream_t);
template void launch_gsline<double>(const LevelView<double> &, cudaStream_t);
template void launch_hs1_blocks<float>(const LevelView<float> &, cudaStream_t);
template void launch_hs1_blocks<double>(const LevelView<double> &, cudaStream_t);

}  // namespace segmg
