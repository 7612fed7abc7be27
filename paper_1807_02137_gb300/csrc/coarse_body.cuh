// coarse_body.cuh -- the coarsest-grid solve as a block-level device function, shared by the
// one-block coarse kernel and the bottom-of-cycle kernel (same arithmetic, same thread count).
#pragma once

#include "internal.h"
#include "reduce.cuh"

namespace segmg {

constexpr int kCoarseThreads = 1024;
constexpr int kWarpCoarseMax = 256;   // grids of at most this many cells are solved by one warp
constexpr int kRegBand = 8;           // one warp keeps the band factor in registers up to this width
                                      // (and at most 32 unknowns: one row per lane)

// The threads that run the coarsest solve: one warp (no block barriers) or the whole block.
template <int NT>
struct Team {
    static __device__ __forceinline__ void sync() {
        if constexpr (NT == 32) __syncwarp();
        else __syncthreads();
    }
    template <typename C>
    static __device__ __forceinline__ C sum(C v, double *red) {
        if constexpr (NT != 32) {
            return block_sum_t<C>(v, red);
        } else {
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            return v;
        }
    }
    template <typename C>
    static __device__ __forceinline__ C max(C v, double *red) {
        if constexpr (NT != 32) {
            return block_max_t<C>(v, red);
        } else {
            for (int o = 16; o > 0; o >>= 1) v = max_t<C>(v, __shfl_xor_sync(0xffffffffu, v, o));
            return v;
        }
    }
};

// A grid the coarsest solve reads (pn, w, F, rhs) and updates (u), row pitch `pitch`.
template <typename T>
struct CoarseGrid {
    int n, m, pitch;
    const T *pn;
    T *u;
    const T *w;
    const __nv_bfloat16 *wb;
    const T *F, *rhs;
    int has_rhs;
    T inv_2h, inv_tau, beta;
};

// ---------------------------------------------------------------------------------------
// Coarsest solve (Algorithm 1, "compute the exact solution"), one block, in the arithmetic
// precision of the path (FP32 for FP32 storage, FP64 for FP64 and mixed storage).  The unknown
// is the increment u of phi = pn + u.  Picard on the frozen
// coefficients G (at phi): each step solves the symmetric positive definite system
//   (mu/h^2 sum_X G_X + 1/tau) u - mu/h^2 sum_X G_X u_X = mu/h^2 sum_X G_X (pn_X - pn) - F - area - rhs
// by banded Cholesky with cells ordered along the shorter side.  It stops when the nonlinear
// residual falls below tol times its initial value, when a step changes no value by more than
// kStat times max(1, max |phi|) (1e-14 in FP64, 1e-6 in FP32: rounding level), when in FP32 a
// step no longer reduces the residual by 10% (it has reached the rounding floor), or after
// maxit steps.
// ---------------------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ C rsqrt_of(C s);
template <>
__device__ __forceinline__ float rsqrt_of<float>(float s) { return rsqrtf(s); }
template <>
__device__ __forceinline__ double rsqrt_of<double>(double s) { return 1.0 / sqrt(s); }

// Banded Cholesky factorisation and solve of A x = b by one warp for N <= 32 unknowns and band
// width bw <= kRegBand: lane r holds row r of the band (Lr[d] = A(r, r - d), then L(r, r - d);
// Lr[0] keeps 1 / L(r, r)).  Column k's pivot and entries reach the other lanes by shuffles;
// every element receives the same updates, in the same order, as in the shared-memory
// factorisation.  The substitutions accumulate column by column.  Returns false (on every lane)
// when a pivot is not positive; else lane r < N holds x(r) in xr.
template <typename C>
__device__ __forceinline__ bool warp_band_solve(const C *band, const C *b, int N, int bw, C &xr) {
    constexpr unsigned kFull = 0xffffffffu;
    const int r = threadIdx.x & 31, bw1 = bw + 1;
    C Lr[kRegBand + 1];
#pragma unroll
    for (int d = 0; d <= kRegBand; ++d) Lr[d] = (r < N && d <= bw && d <= r) ? band[(size_t)r * bw1 + d] : C(0);
    for (int k = 0; k < N; ++k) {
        const C piv = __shfl_sync(kFull, Lr[0], k);
        if (!(piv > C(0))) return false;
        const C rkk = rsqrt_of<C>(piv);
        if (r == k) Lr[0] = rkk;
        const int dk = r - k;
        C lk = C(0);   // L(r, k) once column k is scaled
#pragma unroll
        for (int d = 1; d <= kRegBand; ++d)
            if (d == dk && d <= bw) {
                Lr[d] *= rkk;
                lk = Lr[d];
            }
        // trailing update: L(r, c) -= L(r, k) L(c, k) for k < c <= r <= k + bw
#pragma unroll
        for (int j = 1; j <= kRegBand; ++j) {
            if (j > bw) break;
            const C lck = __shfl_sync(kFull, lk, min(k + j, 31));
            const int idx = dk - j;   // r - c
#pragma unroll
            for (int d = 0; d < kRegBand; ++d)
                if (d == idx && dk <= bw && r < N) Lr[d] -= lk * lck;
        }
    }
    // forward: y = L^-1 b
    const C br = r < N ? b[r] : C(0);
    C acc = C(0), y = C(0);
    for (int c = 0; c < N; ++c) {
        const C yc = __shfl_sync(kFull, (br - acc) * Lr[0], c);
        if (r == c) y = yc;
        const int dc = r - c;
#pragma unroll
        for (int d = 1; d <= kRegBand; ++d)
            if (d == dc && d <= bw) acc += Lr[d] * yc;
    }
    // backward: x = L^-T y
    C acc2 = C(0);
    xr = C(0);
    for (int c = N - 1; c >= 0; --c) {
        const C xc = __shfl_sync(kFull, (y - acc2) * Lr[0], c);
        if (r == c) xr = xc;
#pragma unroll
        for (int d = 1; d <= kRegBand; ++d) {
            if (d > bw) break;
            const C lcd = __shfl_sync(kFull, Lr[d], c);   // L(c, c - d)
            if (r == c - d) acc2 += lcd * xc;
        }
    }
    return true;
}

// Run by the NT threads of a team (NT = 32: warp 0; else the whole block) in the arithmetic
// type C (storage T); scratch holds coarse_scratch_elems(n, m) values of C.
template <typename T, typename C, int NT>
__device__ void coarse_solve_team(const CoarseGrid<T> &L, ModelParams mp, double A1frac, double h2nm,
                                  int maxit, double tol, C *scratch, double *red, int *s_err,
                                  int *it_out, double *res_out) {
    using TM = Team<NT>;
    constexpr bool kF32 = sizeof(C) == 4;
    constexpr C kStat = kF32 ? C(1e-6) : C(1e-14);
    const int n = L.n, m = L.m, p = L.pitch, N = n * m;
    const int tid = threadIdx.x, nt = NT;
    const bool colmajor = m > n;
    const int bw = colmajor ? n : m, bw1 = bw + 1;
    C *x = scratch, *G = x + N, *b = G + N, *y = b + N, *band = y + N;
    const C hinv = C(2) * (C)L.inv_2h;
    const C cdiff = C(mp.mu) * hinv * hinv;
    const C inv_tau = (C)L.inv_tau, inv_2h = (C)L.inv_2h, beta = (C)L.beta;
    auto idx = [&](int i, int j) { return colmajor ? j * n + i : i * m + j; };
    auto pn_at = [&](int i, int j) { return (C)L.pn[(size_t)i * p + j]; };
    if (tid == 0) *s_err = 0;
    for (int q = tid; q < N; q += nt) {
        int i = q / m, j = q % m;
        x[idx(i, j)] = (C)L.u[(size_t)i * p + j];
    }
    TM::sync();
    // G at phi = pn + x and the Rada-Chen area term; returns the area term
    auto coeffs = [&]() -> C {
        C area = C(0);
        if (mp.model == 1) {
            double hs = 0.0;
            for (int q = tid; q < N; q += nt) {
                int i = q / m, j = q % m;
                hs += 0.5 + atan(((double)pn_at(i, j) + (double)x[idx(i, j)]) / mp.eps) / M_PI;
            }
            hs = TM::template sum<double>(hs, red);
            area = (C)(2.0 * mp.nu * (h2nm * hs - A1frac));
        }
        for (int q = tid; q < N; q += nt) {
            int i = q / m, j = q % m;
            int iS = min(i + 1, n - 1), iN = max(i - 1, 0), jE = min(j + 1, m - 1), jW = max(j - 1, 0);
            C gy = ((pn_at(iS, j) - pn_at(iN, j)) + (x[idx(iS, j)] - x[idx(iN, j)])) * inv_2h;
            C gx = ((pn_at(i, jE) - pn_at(i, jW)) + (x[idx(i, jE)] - x[idx(i, jW)])) * inv_2h;
            C w = L.wb ? C(__bfloat162float(L.wb[(size_t)i * p + j])) : (C)L.w[(size_t)i * p + j];
            G[idx(i, j)] = w * rsqrt_of<C>(gx * gx + gy * gy + beta);
        }
        TM::sync();
        return area;
    };
    auto faceG = [&](int i, int j, int i2, int j2) { return C(0.5) * (G[idx(i, j)] + G[idx(i2, j2)]); };
    auto resnorm = [&]() -> double {
        C area = coeffs();
        C acc = C(0);
        for (int q = tid; q < N; q += nt) {
            int i = q / m, j = q % m;
            const C xc = x[idx(i, j)], pc = pn_at(i, j);
            C fl = C(0);
            auto add = [&](int i2, int j2) { fl += faceG(i, j, i2, j2) * ((pn_at(i2, j2) - pc) + (x[idx(i2, j2)] - xc)); };
            if (i + 1 < n) add(i + 1, j);
            if (i > 0) add(i - 1, j);
            if (j + 1 < m) add(i, j + 1);
            if (j > 0) add(i, j - 1);
            size_t o = (size_t)i * p + j;
            C Lv = cdiff * fl - (C)L.F[o] - area - inv_tau * xc;
            C r = (L.has_rhs ? (C)L.rhs[o] : C(0)) - Lv;
            acc += r * r;
        }
        return sqrt((double)TM::template sum<C>(acc, red));
    };
    const double r0 = resnorm();
    double res = r0, res_prev = r0;
    int it = 0;
    while (it < maxit) {
        if (it > 0) {
            res = resnorm();
            if (res <= tol * r0 || res == 0.0) break;
            if (kF32 && res > 0.9 * res_prev) break;
            res_prev = res;
        }
        if (r0 == 0.0) break;
        C area = coeffs();
        for (int q = tid; q < N * bw1; q += nt) band[q] = C(0);
        TM::sync();
        for (int q = tid; q < N; q += nt) {
            int i = q / m, j = q % m, r = idx(i, j);
            const C pc = pn_at(i, j);
            C diag = C(0), pflux = C(0);
            auto off = [&](int i2, int j2) {
                C g = faceG(i, j, i2, j2);
                C a = cdiff * g;
                diag += a;
                pflux += g * (pn_at(i2, j2) - pc);
                int c = idx(i2, j2);
                if (c < r && MG_DBG_OK(r - c, bw1, kDbgCoarse)) band[(size_t)r * bw1 + (r - c)] = -a;
            };
            if (i + 1 < n) off(i + 1, j);
            if (i > 0) off(i - 1, j);
            if (j + 1 < m) off(i, j + 1);
            if (j > 0) off(i, j - 1);
            band[(size_t)r * bw1] = diag + inv_tau;
            size_t o = (size_t)i * p + j;
            b[r] = cdiff * pflux - (C)L.F[o] - area - (L.has_rhs ? (C)L.rhs[o] : C(0));
        }
        TM::sync();
        bool in_regs = false;
        if constexpr (NT == 32) in_regs = N <= 32 && bw <= kRegBand;
        if (in_regs) {
            // the tiny coarsest grids: the band factor in registers, one row per lane
            C xr;
            const bool ok = warp_band_solve<C>(band, b, N, bw, xr);
            TM::sync();
            if (!ok) {
                if (tid == 0) *s_err = 1;
                TM::sync();
                break;
            }
            if (tid < N) b[tid] = xr;
        } else {
            // right-looking banded Cholesky: band[r*bw1 + (r-c)] = L(r, c); the diagonal entry
            // keeps 1 / L(k, k) once column k is done
            for (int k = 0; k < N && !(*s_err); ++k) {
                if (tid == 0) {
                    C d = band[(size_t)k * bw1];
                    if (!(d > C(0))) (*s_err) = 1;
                    else band[(size_t)k * bw1] = rsqrt_of<C>(d);
                }
                TM::sync();
                if ((*s_err)) break;
                const C rkk = band[(size_t)k * bw1];
                const int last = min(k + bw, N - 1), cnt = last - k;
                for (int t = tid; t < cnt; t += nt)
                    if (MG_DBG_OK((size_t)(k + 1 + t) * bw1 + (1 + t), (size_t)N * bw1, kDbgCoarse))
                        band[(size_t)(k + 1 + t) * bw1 + (1 + t)] *= rkk;
                TM::sync();
                for (int t = tid; t < cnt * cnt; t += nt) {
                    // the trailing triangle: rows ii >= columns jj (integer indexing only)
                    const int ii = t / cnt, jj = t - ii * cnt;
                    if (jj > ii) continue;
                    int ri = k + 1 + ii, rj = k + 1 + jj;
                    if (!MG_DBG_OK((size_t)ri * bw1 + (ri - rj), (size_t)N * bw1, kDbgCoarse) ||
                        !MG_DBG_OK(ri - k, bw1, kDbgCoarse) || !MG_DBG_OK(rj - k, bw1, kDbgCoarse))
                        continue;
                    band[(size_t)ri * bw1 + (ri - rj)] -= band[(size_t)ri * bw1 + (ri - k)] * band[(size_t)rj * bw1 + (rj - k)];
                }
                TM::sync();
            }
            if ((*s_err)) break;
            // forward and backward substitution by warp 0
            if (tid < 32) {
                for (int r = 0; r < N; ++r) {
                    C s = C(0);
                    for (int c = max(0, r - bw) + tid; c < r; c += 32) s += band[(size_t)r * bw1 + (r - c)] * y[c];
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                    if (tid == 0) y[r] = (b[r] - s) * band[(size_t)r * bw1];
                    __syncwarp();
                }
                for (int r = N - 1; r >= 0; --r) {
                    C s = C(0);
                    int c1 = min(N - 1, r + bw);
                    for (int c = r + 1 + tid; c <= c1; c += 32) s += band[(size_t)c * bw1 + (c - r)] * b[c];
                    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
                    if (tid == 0) b[r] = (y[r] - s) * band[(size_t)r * bw1];
                    __syncwarp();
                }
            }
        }
        TM::sync();
        C dmax = C(0), pmax = C(1);
        for (int q = tid; q < N; q += nt) {
            const int i = colmajor ? q % n : q / m, j = colmajor ? q / n : q % m;
            dmax = max_t<C>(dmax, abs_t<C>(b[q] - x[q]));
            pmax = max_t<C>(pmax, abs_t<C>(pn_at(i, j) + b[q]));
        }
        dmax = TM::template max<C>(dmax, red);
        pmax = TM::template max<C>(pmax, red);
        for (int q = tid; q < N; q += nt) x[q] = b[q];
        TM::sync();
        ++it;
        if (dmax <= kStat * pmax) break;
    }
    for (int q = tid; q < N; q += nt) {
        int i = q / m, j = q % m;
        stc(L.u, (size_t)i * p + j, (size_t)n * p, kDbgCoarse, (T)x[idx(i, j)]);
    }
    *it_out = it;
    *res_out = res;
    TM::sync();
}

// ---------------------------------------------------------------------------------------
// The coarsest solve by AOS time marching (Algorithm 1, "using e.g. time-marching or AOS";
// Sec. 5: 100 iterations on the coarsest grid), `iters` iterations of step dt.  One iteration
// (additive operator splitting of d phi / ds = L(phi) - rhs, coefficients frozen at phi, the
// 1/tau term split evenly between rows and columns), in increment form: for l = rows, columns
//   ((1 + dt/tau) I - 2 dt A_l) y_l = u + dt (2 A_l pn - F - area - rhs),   u <- (y_x + y_y) / 2
// with A_l the mu/h^2-weighted face-G differences along l (the same step as the FP64 oracle's
// total-phi form, rewritten for phi = pn + u).  Scratch: 5 N values of C.
// ---------------------------------------------------------------------------------------
template <typename T, typename C, int NT>
__device__ void aos_solve_team(const CoarseGrid<T> &L, ModelParams mp, double A1frac, double h2nm, int iters,
                               double dt_, C *scratch, double *red) {
    using TM = Team<NT>;
    const int n = L.n, m = L.m, p = L.pitch, N = n * m;
    const int tid = threadIdx.x;
    C *x = scratch, *G = x + N, *yx = G + N, *dd = yx + N, *rr = dd + N;
    const C hinv = C(2) * (C)L.inv_2h;
    const C cdiff = C(mp.mu) * hinv * hinv;
    const C inv_tau = (C)L.inv_tau, inv_2h = (C)L.inv_2h, beta = (C)L.beta, dt = (C)dt_;
    auto pn_at = [&](int i, int j) { return (C)L.pn[(size_t)i * p + j]; };
    for (int q = tid; q < N; q += NT) x[q] = (C)L.u[(size_t)(q / m) * p + (q % m)];
    TM::sync();
    for (int it = 0; it < iters; ++it) {
        C area = C(0);
        if (mp.model == 1) {
            double hs = 0.0;
            for (int q = tid; q < N; q += NT)
                hs += 0.5 + atan(((double)pn_at(q / m, q % m) + (double)x[q]) / mp.eps) / M_PI;
            hs = TM::template sum<double>(hs, red);
            area = (C)(2.0 * mp.nu * (h2nm * hs - A1frac));
        }
        for (int q = tid; q < N; q += NT) {
            const int i = q / m, j = q % m;
            const int iS = min(i + 1, n - 1), iN = max(i - 1, 0), jE = min(j + 1, m - 1), jW = max(j - 1, 0);
            const C gy = ((pn_at(iS, j) - pn_at(iN, j)) + (x[iS * m + j] - x[iN * m + j])) * inv_2h;
            const C gx = ((pn_at(i, jE) - pn_at(i, jW)) + (x[i * m + jE] - x[i * m + jW])) * inv_2h;
            const C w = L.wb ? C(__bfloat162float(L.wb[(size_t)i * p + j])) : (C)L.w[(size_t)i * p + j];
            G[q] = w * rsqrt_of<C>(gx * gx + gy * gy + beta);
        }
        TM::sync();
        // rows (dir 0) into yx, then columns (dir 1) into x = (yx + y) / 2
        for (int dir = 0; dir < 2; ++dir) {
            const int nl = dir == 0 ? n : m, len = dir == 0 ? m : n, stp = dir == 0 ? 1 : m;
            for (int line = tid; line < nl; line += NT) {
                const int q0 = dir == 0 ? line * m : line;
                C cup = C(0), cdi = C(1), crh = C(0);
                for (int t = 0; t < len; ++t) {
                    const int q = q0 + t * stp;
                    const int i = q / m, j = q % m;
                    const C cp = t > 0 ? cdiff * C(0.5) * (G[q] + G[q - stp]) : C(0);
                    const C cn = t + 1 < len ? cdiff * C(0.5) * (G[q] + G[q + stp]) : C(0);
                    const C pc = pn_at(i, j);
                    C Apn = C(0);
                    if (t > 0) Apn += cp * (pn_at((q - stp) / m, (q - stp) % m) - pc);
                    if (t + 1 < len) Apn += cn * (pn_at((q + stp) / m, (q + stp) % m) - pc);
                    const size_t o = (size_t)i * p + j;
                    const C rhs = (L.has_rhs ? (C)L.rhs[o] : C(0));
                    C di = C(1) + dt * inv_tau + C(2) * dt * (cp + cn);
                    C r = x[q] + dt * (C(2) * Apn - (C)L.F[o] - area - rhs);
                    if (t > 0) {
                        const C wgt = (-C(2) * dt * cp) / cdi;
                        di -= wgt * cup;
                        r -= wgt * crh;
                    }
                    dd[q] = di;
                    rr[q] = r;
                    cup = -C(2) * dt * cn;
                    cdi = di;
                    crh = r;
                }
                C y = crh / cdi;
                for (int t = len - 1; t >= 0; --t) {
                    const int q = q0 + t * stp;
                    if (t < len - 1) {
                        const C cn = cdiff * C(0.5) * (G[q] + G[q + stp]);
                        y = (rr[q] + C(2) * dt * cn * y) / dd[q];
                    }
                    if (dir == 0) yx[q] = y;
                    else x[q] = C(0.5) * (yx[q] + y);
                }
            }
            TM::sync();
        }
    }
    for (int q = tid; q < N; q += NT) stc(L.u, (size_t)(q / m) * p + (q % m), (size_t)n * p, kDbgCoarse, (T)x[q]);
    TM::sync();
}

// The coarsest solve in the arithmetic type C; all threads of the (kCoarseThreads) block call
// it.  it_out / res_out are valid in thread 0.
template <typename T, typename C>
__device__ void coarse_solve_block(const CoarseGrid<T> &L, ModelParams mp, double A1frac, double h2nm,
                                   int maxit, double tol, C *scratch, double *red, int *s_err,
                                   int *it_out, double *res_out, int aos = 0, double aos_dt = 0.0) {
    if (aos) {
        if (threadIdx.x == 0) *s_err = 0;
        if (L.n * L.m <= kWarpCoarseMax) {
            if (threadIdx.x < 32) aos_solve_team<T, C, 32>(L, mp, A1frac, h2nm, maxit, aos_dt, scratch, red);
            __syncthreads();
        } else {
            aos_solve_team<T, C, kCoarseThreads>(L, mp, A1frac, h2nm, maxit, aos_dt, scratch, red);
        }
        *it_out = maxit;
        *res_out = 0.0;
        return;
    }
    if (L.n * L.m <= kWarpCoarseMax) {
        if (threadIdx.x < 32)
            coarse_solve_team<T, C, 32>(L, mp, A1frac, h2nm, maxit, tol, scratch, red, s_err, it_out, res_out);
        __syncthreads();
    } else {
        coarse_solve_team<T, C, kCoarseThreads>(L, mp, A1frac, h2nm, maxit, tol, scratch, red, s_err, it_out,
                                                res_out);
    }
}


}  // namespace segmg
