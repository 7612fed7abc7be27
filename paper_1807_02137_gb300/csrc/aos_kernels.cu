// aos_kernels.cu -- AOS time marching on a full grid (the AOS method the paper compares against
// in Table 6), for the current pseudo-time step.
//
// One iteration (additive operator splitting of d phi / ds = L(phi) - rhs, with the
// coefficients frozen at phi and the 1/tau term split evenly between the directions), in
// increment form phi = pn + u:
//   ((1 + dt/tau) I - 2 dt A_l) y_l = u + dt (2 A_l pn - F - area - rhs),  l = rows, columns,
//   u <- (y_rows + y_cols) / 2,
// with A_l the mu/h^2-weighted face-G differences along l and G from the coefficient snapshot.
// One thread solves one row (or column) by the Thomas algorithm; the eliminated diagonal and
// right-hand side go to two scratch grids.  The column pass also forms the per-block sums of
// (u_new - u)^2 and (pn + u)^2 for the relative-change stop.
#include "arith.cuh"
#include "reduce.cuh"

namespace segmg {

namespace {

template <typename T, int DIR>
__global__ void __launch_bounds__(128) k_aos_lines(LevelView<T> L, const double *area, T dt, T *yx, T *dd, T *rr,
                                                   double *part) {
    __shared__ double red[33];
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = L.n, m = L.m, p = L.pitch;
    const int nl = DIR == 0 ? n : m, len = DIR == 0 ? m : n;
    const size_t stp = DIR == 0 ? 1 : (size_t)p;
    const T ar = area ? T(area[0]) : T(0);
    double sd = 0.0, sp = 0.0;
    if (line < nl) {
        const size_t o0 = DIR == 0 ? (size_t)line * p : (size_t)line;
        T cup = T(0), cdi = T(1), crh = T(0);
        for (int t = 0; t < len; ++t) {
            const size_t o = o0 + t * stp;
            const T gc = L.G[o], pc = L.pn[o];
            T cp = T(0), cn = T(0), Apn = T(0);
            if (t > 0) {
                cp = L.cdiff * face(gc, L.G[o - stp], true);
                Apn += cp * (L.pn[o - stp] - pc);
            }
            if (t + 1 < len) {
                cn = L.cdiff * face(gc, L.G[o + stp], true);
                Apn += cn * (L.pn[o + stp] - pc);
            }
            const T rhs = L.has_rhs ? L.rhs[o] : T(0);
            T di = T(1) + dt * L.inv_tau + T(2) * dt * (cp + cn);
            T r = L.u[o] + dt * (T(2) * Apn - L.F[o] - ar - rhs);
            if (t > 0) {
                const T wgt = (-T(2) * dt * cp) / cdi;
                di -= wgt * cup;
                r -= wgt * crh;
            }
            dd[o] = di;
            rr[o] = r;
            cup = -T(2) * dt * cn;
            cdi = di;
            crh = r;
        }
        T y = crh / cdi;
        for (int t = len - 1; t >= 0; --t) {
            const size_t o = o0 + t * stp;
            if (t < len - 1) {
                const T cn = L.cdiff * face(L.G[o], L.G[o + stp], true);
                y = (rr[o] + T(2) * dt * cn * y) / dd[o];
            }
            if (DIR == 0) {
                stc(yx, o, (size_t)L.n * L.pitch, kDbgOther, y);
            } else {
                const T uo = L.u[o], un = T(0.5) * (yx[o] + y);
                sd += (double)(un - uo) * (double)(un - uo);
                sp += (double)(L.pn[o] + uo) * (double)(L.pn[o] + uo);
                stc(L.u, o, (size_t)L.n * L.pitch, kDbgOther, un);
            }
        }
    }
    if (DIR == 1) {
        const double a = block_sum(sd, red), b = block_sum(sp, red);
        if (threadIdx.x == 0) {
            part[2 * blockIdx.x] = a;
            part[2 * blockIdx.x + 1] = b;
        }
    }
}

__global__ void k_aos_final(const double *part, int nb, double *out) {
    __shared__ double red[33];
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        a += part[2 * q];
        b += part[2 * q + 1];
    }
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

}  // namespace

template <typename T>
void launch_aos_iteration(const LevelView<T> &L, const double *area, double dt, double *partials, double *sums,
                          cudaStream_t st) {
    const int br = (L.n + 127) / 128, bc = (L.m + 127) / 128;
    k_aos_lines<T, 0><<<br, 128, 0, st>>>(L, area, T(dt), L.t, L.r, L.f, partials);
    // the column pass needs the row results (L.t) and scratch other than L.t: G stays, f is free
    k_aos_lines<T, 1><<<bc, 128, 0, st>>>(L, area, T(dt), L.t, L.r, L.f, partials);
    k_aos_final<<<1, 1024, 0, st>>>(partials, bc, sums);
}

template void launch_aos_iteration<float>(const LevelView<float> &, const double *, double, double *, double *,
                                          cudaStream_t);
template void launch_aos_iteration<double>(const LevelView<double> &, const double *, double, double *, double *,
                                           cudaStream_t);

}  // namespace segmg
