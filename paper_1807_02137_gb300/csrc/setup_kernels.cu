// setup_kernels.cu -- image-derived data (Sec. 2.2), initial level set and per-step fields
// (Sec. 5), region averages (eq. c1c2), mask and the Rada-Chen area term.
#include "arith.cuh"
#include "reduce.cuh"

namespace segmg {

namespace {

__device__ __forceinline__ int mirror(int t, int n) {
    if (n == 1) return 0;
    while (t < 0 || t >= n) {
        if (t < 0) t = -t - 1;
        if (t >= n) t = 2 * n - t - 1;
    }
    return t;
}

// Blur taps in the accumulation type of the blur: FP32 for the FP32 path, FP64 for FP64.
template <typename A>
struct Taps {
    A w[33];
};

template <typename T>
__global__ void k_copy(const T *src, int ps, T *dst, int pd, int n, int m) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i < n && j < m)
        stc(dst, (size_t)i * pd + j, (size_t)n * pd, kDbgSetup, ldc(src, (size_t)i * ps + j, (size_t)n * ps, kDbgSetup));
}

// The image copied into the finest grid's z; bit 2 of *flag is set when a value is NaN or Inf.
template <typename T>
__global__ void k_copy_check(const T *src, T *dst, int pd, int n, int m, int *flag) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    bool bad = false;
    if (i < n && j < m) {
        const T v = ldc(src, (size_t)i * m + j, (size_t)n * m, kDbgSetup);
        bad = !isfinite(v);
        stc(dst, (size_t)i * pd + j, (size_t)n * pd, kDbgSetup, v);
    }
    if (__any_sync(0xffffffffu, bad) && threadIdx.x == 0) atomicOr(flag, 2);
}

// Separable Gaussian G_sigma * z with mirror boundary; `dir` 0 = along rows, 1 = along columns.
template <typename T>
__global__ void k_blur(const T *src, T *dst, int n, int m, int ps, int pd, Taps<T> tp, int R, int dir) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i >= n || j >= m) return;
    const size_t lim = (size_t)n * ps;
    T a = T(0);
    for (int t = -R; t <= R; ++t) {
        const T v = dir == 0 ? ldc(src, (size_t)i * ps + mirror(j + t, m), lim, kDbgSetup)
                             : ldc(src, (size_t)mirror(i + t, n) * ps + j, lim, kDbgSetup);
        a += tp.w[t + R] * v;
    }
    stc(dst, (size_t)i * pd + j, (size_t)n * pd, kDbgSetup, a);
}

// Edge detector g = 1 / (1 + beta_edge |grad (G*z)|^2) (central differences, mirror ghosts),
// distance function d = prod_k (1 - exp(-dx^2 / 2s^2) exp(-dy^2 / 2s^2)) and the length
// weight w = g (Spencer-Chen) or d g (Rada-Chen).  Arithmetic in the storage precision; the
// two exponential factors of a marker depend on the column alone and on the row alone, so a
// block of 32 x 8 cells evaluates them once per column and row (40 instead of 256 per marker).
template <typename T>
__global__ void __launch_bounds__(256) k_edge_distance(const T *zb, T *w, T *d, int n, int m, int p, T beta_edge,
                                                       const double *mk, int k, T inv_s2, int model) {
    constexpr int KC = 32;                       // markers per shared-memory chunk
    __shared__ T ex[KC][32], ey[KC][8];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int j0 = blockIdx.x * 32, i0 = blockIdx.y * 8, j = j0 + tx, i = i0 + ty;
    T dd = T(1);
    for (int q0 = 0; q0 < k; q0 += KC) {
        const int kc = min(KC, k - q0);
        __syncthreads();                         // the previous chunk's factors are used up
        for (int e = tid; e < kc * 32; e += 256) {
            const int q = e >> 5, c = e & 31;
            const T dx = T(mk[2 * (q0 + q)]) - T(j0 + c);
            ex[q][c] = exp(-dx * dx * inv_s2);
        }
        for (int e = tid; e < kc * 8; e += 256) {
            const int q = e >> 3, r = e & 7;
            const T dy = T(mk[2 * (q0 + q) + 1]) - T(i0 + r);
            ey[q][r] = exp(-dy * dy * inv_s2);
        }
        __syncthreads();
        for (int q = 0; q < kc; ++q) dd *= T(1) - ex[q][tx] * ey[q][ty];
    }
    if (i >= n || j >= m) return;
    T zx = (zb[(size_t)i * p + mirror(j + 1, m)] - zb[(size_t)i * p + mirror(j - 1, m)]) * T(0.5);
    T zy = (zb[(size_t)mirror(i + 1, n) * p + j] - zb[(size_t)mirror(i - 1, n) * p + j]) * T(0.5);
    T g = T(1) / (T(1) + beta_edge * (zx * zx + zy * zy));
    size_t o = (size_t)i * p + j;
    const size_t lim = (size_t)n * p;
    stc(d, o, lim, kDbgSetup, dd);
    stc(w, o, lim, kDbgSetup, model == 1 ? dd * g : g);
}

// Signed distance (px, positive inside) to the boundary of a convex polygon given counter-
// clockwise, or to a circle of radius r0 about (cx, cy) when nh == 0.  The polygon's vertices
// go through shared memory in the storage precision, 64 edges at a time.
template <typename T>
__global__ void __launch_bounds__(256) k_initial_phi(T *pn, T *u, int n, int m, int p, const double *hull, int nh,
                                                     T cx, T cy, T r0) {
    constexpr int EC = 64;                       // edges per shared-memory chunk
    __shared__ T hx[EC + 1], hy[EC + 1];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    T px = T(j), py = T(i), val;
    if (nh == 0) {
        val = r0 - sqrt((px - cx) * (px - cx) + (py - cy) * (py - cy));
    } else {
        T dmin = T(1e30);
        bool inside = true;
        for (int q0 = 0; q0 < nh; q0 += EC) {
            const int ec = min(EC, nh - q0);
            __syncthreads();
            if (tid <= ec) {                     // vertices q0 .. q0 + ec (the last wraps to 0)
                const int v = q0 + tid == nh ? 0 : q0 + tid;
                hx[tid] = T(hull[2 * v]);
                hy[tid] = T(hull[2 * v + 1]);
            }
            __syncthreads();
            for (int e = 0; e < ec; ++e) {
                const T ax = hx[e], ay = hy[e], bx = hx[e + 1], by = hy[e + 1];
                const T ex = bx - ax, ey = by - ay;
                if (ex * (py - ay) - ey * (px - ax) < T(0)) inside = false;
                T t = ((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey);
                t = t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
                const T dx = px - (ax + t * ex), dy = py - (ay + t * ey);
                dmin = fmin(dmin, sqrt(dx * dx + dy * dy));
            }
        }
        val = inside ? dmin : -dmin;
    }
    if (i >= n || j >= m) return;
    size_t o = (size_t)i * p + j;
    const size_t lim = (size_t)n * p;
    stc(pn, o, lim, kDbgSetup, val);
    stc(u, o, lim, kDbgSetup, T(0));
}

// Fitting field of the step on every grid in one launch: lambda1 (z - c1)^2 - lambda2 (z - c2)^2
// (+ theta d for SC), in the storage precision.  Blocks of 32 x 8 cells, numbered grid by grid.
template <typename T>
__global__ void __launch_bounds__(256) k_fitting(FitGrids<T> G, const Scalars *sc, T lambda1, T lambda2, T theta,
                                                 int model) {
    __shared__ T c12[2];             // c1, c2 converted once per block
    if (threadIdx.x < 2 && threadIdx.y == 0) c12[threadIdx.x] = T(threadIdx.x == 0 ? sc->c1 : sc->c2);
    __syncthreads();
    int l = 0;
    while (l + 1 < G.nlev && (int)blockIdx.x >= G.first_block[l + 1]) ++l;
    const int b = blockIdx.x - G.first_block[l], bx = (G.m[l] + 31) / 32;
    const int j = (b % bx) * 32 + threadIdx.x, i = (b / bx) * 8 + threadIdx.y;
    if (i >= G.n[l] || j >= G.m[l]) return;
    const size_t o = (size_t)i * G.pitch[l] + j;
    const T z = G.z[l][o], c1 = c12[0], c2 = c12[1];
    T F = lambda1 * (z - c1) * (z - c1) - lambda2 * (z - c2) * (z - c2);
    if (model == 0) F += theta * G.d[l][o];
    stc(G.F[l], o, (size_t)G.n[l] * G.pitch[l], kDbgSetup, F);
}

// phi^n <- phi^n + u, u <- 0 (start of a pseudo-time step on the finest grid).
template <typename T>
__global__ void k_fold(LevelView<T> L) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i >= L.n || j >= L.m) return;
    size_t o = (size_t)i * L.pitch + j;
    const size_t lim = (size_t)L.n * L.pitch;
    stc(L.pn, o, lim, kDbgSetup, add_rn(L.pn[o], L.u[o]));
    stc(L.u, o, lim, kDbgSetup, T(0));
}

__device__ double block_sum_setup(double v, double *red) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        double s = tid < (nt + 31) / 32 ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (tid == 0) red[32] = s;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// Per-block partial sums over 32 x 32 tiles of: H z, H, (1-H) z, (1-H), u^2, pn^2 with
// H = H_eps(pn + u) = 1/2 + atan((pn + u) / eps) / pi (Sec. 2.1).  Each warp sums its 128 cells
// in the storage precision (pairwise, by shuffles); the block's eight warp sums are added in
// FP64 in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_region_partials(LevelView<T> L, T eps, double *part) {
    __shared__ double red[6][8];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, tid = threadIdx.y * 32 + threadIdx.x;
    T s[6] = {0, 0, 0, 0, 0, 0};     // per-thread sums in the storage precision (4 cells)
    for (int q = tid; q < 1024; q += 256) {
        int gi = i0 + q / 32, gj = j0 + q % 32;
        if (gi >= L.n || gj >= L.m) continue;
        size_t o = (size_t)gi * L.pitch + gj;
        T pn = L.pn[o], u = L.u[o], z = L.z[o];
        T H = T(0.5) + atan((pn + u) / eps) * T(M_1_PI);
        s[0] += H * z; s[1] += H; s[2] += (T(1) - H) * z; s[3] += T(1) - H; s[4] += u * u; s[5] += pn * pn;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        T v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) red[k][tid >> 5] = (double)v;
    }
    __syncthreads();
    if (tid < 6) {
        const double *r = red[tid];
        const double a0 = r[0] + r[4], a1 = r[1] + r[5], a2 = r[2] + r[6], a3 = r[3] + r[7];
        const int b = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
        part[(size_t)tid * nb + b] = (a0 + a2) + (a1 + a3);
    }
}

// The six totals over n per-block (or per-chunk) partials of each sum (FP64, fixed order) and
// c1, c2 (eq. c1c2).
__global__ void __launch_bounds__(256) k_region_final(const double *part, int n, Scalars *sc, int set_c) {
    __shared__ double red[33];
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int q = threadIdx.x; q < n; q += blockDim.x)
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += part[(size_t)k * n + q];
    double tot[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) tot[k] = block_sum(v[k], red);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 6; ++q) sc->sums[q] = tot[q];
        if (set_c) {
            sc->c1 = tot[1] > 0 ? tot[0] / tot[1] : 0.0;
            sc->c2 = tot[3] > 0 ? tot[2] / tot[3] : 0.0;
        }
    }
}

// Level-set energy (Sec. 2.2, eqs. scfunc / rcfunc) of the finest grid, pixel units: per 32 x 32
// tile the sums of the cell energy
//   mu w delta(phi) |grad phi|_beta + lambda1 (z - c1)^2 H + lambda2 (z - c2)^2 (1 - H) [+ theta d H]
// and of H, with phi = pn + u, H = H_eps(phi), delta = delta_eps(phi) and |grad phi|_beta by
// central differences with mirror ghosts (clamped neighbours).
template <typename T>
__global__ void __launch_bounds__(256) k_energy_partials(LevelView<T> L, ModelParams mp, const Scalars *sc,
                                                         double *part) {
    __shared__ double red[33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, tid = threadIdx.y * 32 + threadIdx.x;
    const int n = L.n, m = L.m, p = L.pitch;
    const T c1 = T(sc->c1), c2 = T(sc->c2), eps = T(mp.eps), beta = T(mp.beta);
    double se = 0.0, sh = 0.0;
    for (int q = tid; q < 1024; q += 256) {
        const int gi = i0 + q / 32, gj = j0 + q % 32;
        if (gi >= n || gj >= m) continue;
        const size_t o = (size_t)gi * p + gj;
        auto phi = [&](int i, int j) {
            const size_t r = (size_t)(i < 0 ? 0 : (i >= n ? n - 1 : i)) * p + (j < 0 ? 0 : (j >= m ? m - 1 : j));
            return L.pn[r] + L.u[r];
        };
        const T ph = phi(gi, gj);
        const T gx = (phi(gi, gj + 1) - phi(gi, gj - 1)) * T(0.5);
        const T gy = (phi(gi + 1, gj) - phi(gi - 1, gj)) * T(0.5);
        const T H = T(0.5) + atan(ph / eps) * T(M_1_PI);
        const T dl = eps * T(M_1_PI) / (eps * eps + ph * ph);
        const T z = L.z[o];
        T e = T(mp.mu) * weight_at(L, o) * dl * sqrt(gx * gx + gy * gy + beta) +
              T(mp.lambda1) * (z - c1) * (z - c1) * H + T(mp.lambda2) * (z - c2) * (z - c2) * (T(1) - H);
        if (mp.model == 0) e += T(mp.theta) * L.d[o] * H;
        se += (double)e;
        sh += (double)H;
    }
    const int b = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
    const double ve = block_sum_setup(se, red);
    const double vh = block_sum_setup(sh, red);
    if (tid == 0) {
        part[b] = ve;
        part[(size_t)nb + b] = vh;
    }
}

// E = sum of the cell energies + (Rada-Chen) nu n m (sum H / (n m) - A1 / (n m))^2, into *out.
__global__ void k_energy_final(const double *part, int nb, ModelParams mp, double nm, const Scalars *sc,
                               double *out) {
    __shared__ double red[33];
    double ve = 0.0, vh = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        ve += part[q];
        vh += part[(size_t)nb + q];
    }
    ve = block_sum_setup(ve, red);
    vh = block_sum_setup(vh, red);
    if (threadIdx.x == 0) {
        double E = ve;
        if (mp.model == 1) {
            const double a = vh / nm - sc->A1frac;
            E += mp.nu * nm * a * a;
        }
        *out = E;
    }
}

// Rada-Chen area term 2 nu (h^2 sum H(pn + uin) / (n0 m0) - A1 / (n0 m0)) of one grid.
template <typename T>
__global__ void __launch_bounds__(256) k_area_partials(LevelView<T> L, const T *uin, T eps, double *part) {
    __shared__ double red[33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, tid = threadIdx.y * 32 + threadIdx.x;
    T s = T(0);
    for (int q = tid; q < 1024; q += 256) {
        int gi = i0 + q / 32, gj = j0 + q % 32;
        if (gi >= L.n || gj >= L.m) continue;
        size_t o = (size_t)gi * L.pitch + gj;
        s += T(0.5) + atan((L.pn[o] + uin[o]) / eps) * T(M_1_PI);
    }
    double v = block_sum_warps(s, red);
    if (tid == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = v;
}

__global__ void __launch_bounds__(256) k_area_final(const double *part, int nb, double nu, double h2nm,
                                                    const Scalars *sc, double *out) {
    __shared__ double red[33];
    const double s = chunk_sum(part, 0, nb, red);
    if (threadIdx.x == 0) *out = 2.0 * nu * (h2nm * s - sc->A1frac);
}

template <typename T>
__global__ void k_mask(LevelView<T> L, uint8_t *mask) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i >= L.n || j >= L.m) return;
    size_t o = (size_t)i * L.pitch + j;
    stc(mask, (size_t)i * L.m + j, (size_t)L.n * L.m, kDbgSetup, (uint8_t)(add_rn(L.pn[o], L.u[o]) > T(0) ? 1 : 0));
}

__global__ void k_to_bf16(const float *src, __nv_bfloat16 *dst, int n, int m, int p) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i < n && j < m) stc(dst, (size_t)i * p + j, (size_t)n * p, kDbgSetup, __float2bfloat16_rn(src[(size_t)i * p + j]));
}

inline dim3 grid2(int n, int m) { return dim3((m + 31) / 32, (n + 7) / 8); }

}  // namespace

template <typename T>
void launch_energy(const LevelView<T> &L, ModelParams mp, double *partials, int npart, const Scalars *sc,
                   double *out, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32);
    k_energy_partials<T><<<grid, dim3(32, 8), 0, st>>>(L, mp, sc, partials);
    k_energy_final<<<1, 1024, 0, st>>>(partials, npart, mp, (double)L.n * L.m, sc, out);
}


template <typename T>
void launch_copy_in(const T *src, T *dst, int n, int m, int pitch, int *flag, cudaStream_t st) {
    k_copy_check<T><<<grid2(n, m), dim3(32, 8), 0, st>>>(src, dst, pitch, n, m, flag);
}
template <typename T>
void launch_copy_out(const T *src, T *dst, int n, int m, int pitch, cudaStream_t st) {
    k_copy<T><<<grid2(n, m), dim3(32, 8), 0, st>>>(src, pitch, dst, m, n, m);
}

template <typename T>
void launch_blur(const T *src, T *tmp, T *dst, int n, int m, int pitch_src, int pitch, const double *taps,
                 int R, cudaStream_t st) {
    Taps<T> tp;
    for (int t = 0; t <= 2 * R && t < 33; ++t) tp.w[t] = T(taps[t]);
    k_blur<T><<<grid2(n, m), dim3(32, 8), 0, st>>>(src, tmp, n, m, pitch_src, pitch, tp, R, 0);
    k_blur<T><<<grid2(n, m), dim3(32, 8), 0, st>>>(tmp, dst, n, m, pitch, pitch, tp, R, 1);
}

template <typename T>
void launch_edge_distance(const T *zb, T *w, T *d, int n, int m, int pitch, double beta_edge,
                          const double *mk, int k, double sigma_d, int model, cudaStream_t st) {
    const T inv_s2 = T(1.0 / (2.0 * sigma_d * sigma_d));
    k_edge_distance<T><<<grid2(n, m), dim3(32, 8), 0, st>>>(zb, w, d, n, m, pitch, T(beta_edge), mk, k,
                                                            inv_s2, model);
}

template <typename T>
void launch_initial_phi(T *pn, T *u, int n, int m, int pitch, const double *hull, int nh, double cx,
                        double cy, double r0, cudaStream_t st) {
    k_initial_phi<T><<<grid2(n, m), dim3(32, 8), 0, st>>>(pn, u, n, m, pitch, hull, nh, T(cx), T(cy), T(r0));
}

template <typename T>
void launch_fitting(const LevelView<T> *L, int nlev, const Scalars *sc, ModelParams mp, cudaStream_t st) {
    FitGrids<T> G{};
    int blocks = 0;
    G.nlev = nlev;
    for (int l = 0; l < nlev; ++l) {
        G.z[l] = L[l].z; G.d[l] = L[l].d; G.F[l] = L[l].F;
        G.n[l] = L[l].n; G.m[l] = L[l].m; G.pitch[l] = L[l].pitch;
        G.first_block[l] = blocks;
        blocks += ((L[l].m + 31) / 32) * ((L[l].n + 7) / 8);
    }
    k_fitting<T><<<blocks, dim3(32, 8), 0, st>>>(G, sc, T(mp.lambda1), T(mp.lambda2), T(mp.theta), mp.model);
}

template <typename T>
void launch_fold(const LevelView<T> &L, cudaStream_t st) {
    k_fold<T><<<grid2(L.n, L.m), dim3(32, 8), 0, st>>>(L);
}

template <typename T>
void launch_region_sums(const LevelView<T> &L, double eps, double *partials, int npart, Scalars *sc,
                        int finalize_c, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32);
    k_region_partials<T><<<grid, dim3(32, 8), 0, st>>>(L, T(eps), partials);
    if (sum_blocks(npart) == 1) {
        k_region_final<<<1, 256, 0, st>>>(partials, npart, sc, finalize_c);
    } else {   // chunk sums of the six arrays after them
        launch_chunk_sums(partials, npart, 6, partials + 6 * (size_t)npart, st);
        k_region_final<<<1, 256, 0, st>>>(partials + 6 * (size_t)npart, sum_blocks(npart), sc, finalize_c);
    }
}

template <typename T>
void launch_area(const LevelView<T> &L, const T *uin, double eps, double nu, double h2nm,
                 double *partials, int npart, double *out, const Scalars *sc, cudaStream_t st) {
    dim3 grid((L.m + 31) / 32, (L.n + 31) / 32);
    k_area_partials<T><<<grid, dim3(32, 8), 0, st>>>(L, uin, T(eps), partials);
    if (sum_blocks(npart) == 1) {
        k_area_final<<<1, 256, 0, st>>>(partials, npart, nu, h2nm, sc, out);
    } else {
        launch_chunk_sums(partials, npart, 1, partials + npart, st);
        k_area_final<<<1, 256, 0, st>>>(partials + npart, sum_blocks(npart), nu, h2nm, sc, out);
    }
}

template <typename T>
void launch_mask(const LevelView<T> &L, uint8_t *mask, cudaStream_t st) {
    k_mask<T><<<grid2(L.n, L.m), dim3(32, 8), 0, st>>>(L, mask);
}

void launch_to_bf16(const float *src, __nv_bfloat16 *dst, int n, int m, int pitch, cudaStream_t st) {
    k_to_bf16<<<grid2(n, m), dim3(32, 8), 0, st>>>(src, dst, n, m, pitch);
}

#define INST(T)                                                                                      \
    template void launch_copy_in<T>(const T *, T *, int, int, int, int *, cudaStream_t);             \
    template void launch_copy_out<T>(const T *, T *, int, int, int, cudaStream_t);                   \
    template void launch_blur<T>(const T *, T *, T *, int, int, int, int, const double *, int,        \
                                 cudaStream_t);                                                       \
    template void launch_edge_distance<T>(const T *, T *, T *, int, int, int, double, const double *, \
                                          int, double, int, cudaStream_t);                            \
    template void launch_initial_phi<T>(T *, T *, int, int, int, const double *, int, double, double, \
                                        double, cudaStream_t);                                        \
    template void launch_fitting<T>(const LevelView<T> *, int, const Scalars *, ModelParams, cudaStream_t); \
    template void launch_fold<T>(const LevelView<T> &, cudaStream_t);                                \
    template void launch_region_sums<T>(const LevelView<T> &, double, double *, int, Scalars *, int,  \
                                        cudaStream_t);                                                \
    template void launch_area<T>(const LevelView<T> &, const T *, double, double, double, double *,  \
                                 int, double *, const Scalars *, cudaStream_t);                       \
    template void launch_mask<T>(const LevelView<T> &, uint8_t *, cudaStream_t);                    \
    template void launch_energy<T>(const LevelView<T> &, ModelParams, double *, int, const Scalars *, \
                                   double *, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace segmg
