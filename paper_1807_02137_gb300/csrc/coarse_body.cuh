// coarse_body.cuh -- the coarsest-grid solve as a block-level device function, shared by the
// one-block coarse kernel and the bottom-of-cycle kernel (same arithmetic, same thread count).
#pragma once

#include "internal.h"
#include "reduce.cuh"

namespace segmg {

constexpr int kCoarseThreads = 1024;

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
// Coarsest solve (Algorithm 1, "compute the exact solution"), one block, FP64.
// Picard on the frozen coefficients: each step solves
//   (mu/h^2 sum_X G_X + 1/tau) phi - mu/h^2 sum_X G_X phi_X = -(F - pn/tau + area + rhs)
// (symmetric positive definite) by banded Cholesky with cells ordered along the shorter side,
// until the nonlinear residual falls below tol times its initial value, a step changes no
// value by more than 1e-14 of the largest, or maxit steps.
// ---------------------------------------------------------------------------------------
// All threads of the block must call it; scratch holds coarse_scratch_doubles(n, m) doubles.
template <typename T>
__device__ void coarse_solve_block(const CoarseGrid<T> &L, ModelParams mp, double A1frac, double h2nm,
                                   int maxit, double tol, double *scratch, double *red, int *s_err,
                                   int *it_out, double *res_out) {
    const int n = L.n, m = L.m, p = L.pitch, N = n * m;
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool colmajor = m > n;
    const int bw = colmajor ? n : m, bw1 = bw + 1;
    double *x = scratch, *G = x + N, *b = G + N, *y = b + N, *band = y + N;
    const double hinv = 2.0 * (double)L.inv_2h;
    const double cdiff = mp.mu * hinv * hinv;
    const double inv_tau = (double)L.inv_tau, inv_2h = (double)L.inv_2h, beta = (double)L.beta;
    auto idx = [&](int i, int j) { return colmajor ? j * n + i : i * m + j; };
    if (tid == 0) *s_err = 0;
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
            G[idx(i, j)] = (double)(L.wb ? T(__bfloat162float(L.wb[(size_t)i * p + j])) : L.w[(size_t)i * p + j]) / sqrt(gx * gx + gy * gy + beta);
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
        for (int k = 0; k < N && !(*s_err); ++k) {
            if (tid == 0) {
                double d = band[(size_t)k * bw1];
                if (!(d > 0.0)) (*s_err) = 1;
                else band[(size_t)k * bw1] = sqrt(d);
            }
            __syncthreads();
            if ((*s_err)) break;
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
        if ((*s_err)) break;
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
    *it_out = it;
    *res_out = res;
    __syncthreads();
}


}  // namespace segmg
