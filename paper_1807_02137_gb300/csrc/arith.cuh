// arith.cuh -- device arithmetic shared by the smoother kernels.
//
// The fused and the per-phase smoother kernels must produce bit-identical results (the fused
// kernel only reorganises memory traffic).  Every operation of the relaxation formulas below
// is therefore written with explicitly rounded intrinsics (or one fixed hardware approximation),
// which the compiler never contracts or reorders, so both kernels execute the same sequence of
// operations.
#pragma once

#include <cstdint>
#include "internal.h"

namespace segmg {

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

// Division in the relaxation formulas: the hardware approximate quotient in FP32 (about 2 ulp,
// deterministic), IEEE division in FP64.  Both smoother paths call this same function.
__device__ __forceinline__ float div_relax(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_relax(double a, double b) { return __ddiv_rn(a, b); }

// Face coefficient of a face that exists: the arithmetic mean of the two cell values of
// G = w / |grad phi|_beta (Sec. 2.2, eq. abcdrc: G_{i+1/2,j}); a boundary face carries no flux.
template <typename T>
__device__ __forceinline__ T face(T gc, T gn, bool has) {
    return has ? mul_rn(add_rn(gc, gn), T(0.5)) : T(0);
}

// Twice the face value, G_c + G_X.  A kernel whose faces only enter products and sums that are
// then multiplied by cdiff can use these with cdiff / 2: halving is exact, so every product, sum
// and the final values are the same numbers as with face() and cdiff (and comparisons between
// faces keep their outcome), while the four multiplications by 1/2 drop out.
template <typename T>
__device__ __forceinline__ T face2(T gc, T gn, bool has) {
    return has ? add_rn(gc, gn) : T(0);
}

// G = w / |grad phi|_beta at a cell from the four neighbour values of pn and u (central
// differences, spacing h; mirror ghosts are supplied by the caller as clamped neighbours).
// FP32 uses the hardware reciprocal square root (about 2 ulp); FP64 the IEEE square root and
// division.  Every kernel that forms G uses this one function, so G is the same everywhere.
__device__ __forceinline__ float g_of(float w, float s) { return __fmul_rn(w, rsqrtf(s)); }
__device__ __forceinline__ double g_of(double w, double s) { return __ddiv_rn(w, __dsqrt_rn(s)); }

template <typename T>
__device__ __forceinline__ T cell_G(T w, T pS, T pN, T pE, T pW, T uS, T uN, T uE, T uW, T inv_2h,
                                    T beta) {
    T gy = mul_rn(add_rn(sub_rn(pS, pN), sub_rn(uS, uN)), inv_2h);
    T gx = mul_rn(add_rn(sub_rn(pE, pW), sub_rn(uE, uW)), inv_2h);
    T s = fma_rn(gx, gx, fma_rn(gy, gy, beta));
    return g_of(w, s);
}

// GSLEX-I point update (eq. gslexrc) in increment form.  With the row divided by delta the
// frozen coefficients are a_X = mu G_X / h^2 and S = sum a_X + 1/tau; the snapshot has folded
// phi^n and the right-hand sides into f, so the update of the increment is
//     u = (sum_X a_X u_X - f) / (sum_X a_X + 1/tau).
// aS..aW are the face values G_X (the factor mu/h^2 = cdiff is applied here).
template <typename T>
__device__ __forceinline__ T point_relax(T cdiff, T inv_tau, T aS, T aN, T aE, T aW, T uS, T uN,
                                         T uE, T uW, T f) {
    T num = mul_rn(aS, uS);
    num = fma_rn(aN, uN, num);
    num = fma_rn(aE, uE, num);
    num = fma_rn(aW, uW, num);
    T den = add_rn(add_rn(aS, aN), add_rn(aE, aW));
    return div_relax(fma_rn(cdiff, num, -f), fma_rn(cdiff, den, inv_tau));
}

// A point update with a relaxation weight: u_old + omega (g - u_old).
template <typename T>
__device__ __forceinline__ T relax_weighted(T omega, T g, T u_old) {
    return fma_rn(omega, sub_rn(g, u_old), u_old);
}

// One cell of a partial-line run: face values along the line (previous / next cell) and across
// it (two sides), the two across-line neighbour values and f.
template <typename T>
struct RunCell {
    T ap, an, ax1, ax2;
    T ux1, ux2;
    T f;
};

// Partial-line update (Sec. 4.3, step III) of one 32-cell piece of a line, by a whole warp
// (lane t: piece position t).  Each run of member cells (bit t of mk) is a tridiagonal system
// coupled through the in-line coefficients, with the values just outside the run fixed; the
// system is diagonally dominant (Sec. 3.2).  Every other lane carries an identity row, so the
// runs decouple and one parallel cyclic reduction solves all of them at once: each doubling
// step s = 1, 2, 4, 8, 16 eliminates the couplings to positions t - s and t + s, and the loop
// stops as soon as no coupling is left (after ceil(log2(longest run)) steps; the remaining
// steps would change no value).
//   own         this lane's value at the start of the phase (0 for lanes >= len);
//   endp, endn  the values just before / after the piece (their coefficients are zero at a
//               domain edge);  at(t) the RunCell of position t (called for member lanes only).
// Returns true on member lanes, with the new value in x.  All 32 lanes must call it together,
// with the same mk, len, endp and endn.
template <typename T, typename At>
__device__ __forceinline__ bool pcr_piece(uint32_t mk, int len, T cdiff, T inv_tau, T own, T endp, T endn, At at,
                                          T &x) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool mem = (mk >> lane) & 1u;
    T prevv = __shfl_up_sync(kFull, own, 1), nextv = __shfl_down_sync(kFull, own, 1);
    if (lane == 0) prevv = endp;
    if (lane == len - 1) nextv = endn;
    T a = T(0), b = T(1), c = T(0), d = T(0);
    if (mem) {
        const RunCell<T> cc = at(lane);
        const T lo = mul_rn(cdiff, cc.ap), up = mul_rn(cdiff, cc.an);
        const T sum = add_rn(add_rn(cc.ap, cc.an), add_rn(cc.ax1, cc.ax2));
        b = -fma_rn(cdiff, sum, inv_tau);
        const T across = fma_rn(cc.ax2, cc.ux2, mul_rn(cc.ax1, cc.ux1));
        d = fma_rn(-cdiff, across, cc.f);
        const bool pm = lane > 0 && ((mk >> (lane - 1)) & 1u);
        const bool nm = lane < 31 && lane + 1 < len && ((mk >> (lane + 1)) & 1u);
        if (pm) a = lo; else d = fma_rn(-lo, prevv, d);
        if (nm) c = up; else d = fma_rn(-up, nextv, d);
    }
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        if (!__any_sync(kFull, a != T(0) || c != T(0))) break;
        T am = __shfl_up_sync(kFull, a, s), bm = __shfl_up_sync(kFull, b, s);
        T cm = __shfl_up_sync(kFull, c, s), dm = __shfl_up_sync(kFull, d, s);
        T ap = __shfl_down_sync(kFull, a, s), bp = __shfl_down_sync(kFull, b, s);
        T cp = __shfl_down_sync(kFull, c, s), dp = __shfl_down_sync(kFull, d, s);
        if (lane < s) { am = T(0); bm = T(1); cm = T(0); dm = T(0); }
        if (lane + s > 31) { ap = T(0); bp = T(1); cp = T(0); dp = T(0); }
        const T al = div_relax(-a, bm), ga = div_relax(-c, bp);
        b = fma_rn(ga, ap, fma_rn(al, cm, b));
        d = fma_rn(ga, dp, fma_rn(al, dm, d));
        a = mul_rn(al, am);
        c = mul_rn(ga, cp);
    }
    x = div_relax(d, b);
    return mem;
}

// Asynchronous global -> shared copy of one element (4 or 8 bytes); zero-fill when !pred.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *smem, const T *gmem, bool pred) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int sz = pred ? (int)sizeof(T) : 0;
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(sz) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <typename T> struct VecOf;
template <> struct VecOf<float> { using type = float4; static constexpr int n = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ int clamp_idx(int v, int hi) { return v < 0 ? 0 : (v > hi ? hi : v); }

// Loads rows i0-2 .. i0+33 and columns j0-2 .. j0+33 of one or two pitched grid functions into
// dst[36][37] arrays, indices clamped into the domain (the mirror ghosts of the central
// differences).  The 36 x 40 window from column j0-4 is read with 16-byte vector loads where it
// lies inside the domain (per-element clamped loads at the edges); all of a thread's loads are
// issued before its shared-memory stores.  NT threads (tid < NT).
template <typename T, int NT = 256>
__device__ __forceinline__ void load_halo2(T (*dA)[37], const T *sA, T (*dB)[37], const T *sB, int i0, int j0,
                                           int n, int m, int p, int tid) {
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n, NV = 40 / VN, NVEC = 36 * NV, PER = (NVEC + NT - 1) / NT;
    T xa[PER][VN], xb[PER][VN];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = tid + k * NT;
        if (q >= NVEC) break;
        const int a = q / NV, gi = i0 - 2 + a, gj = j0 - 4 + (q % NV) * VN;
        if (gi >= 0 && gi < n && gj >= 0 && gj + VN <= m &&
            MG_DBG_OK((size_t)gi * p + gj + VN - 1, (size_t)n * p, kDbgHaloLoad)) {
            const size_t o = (size_t)gi * p + gj;
            V va = __ldg(reinterpret_cast<const V *>(sA + o));
            memcpy(xa[k], &va, sizeof(V));
            if (sB) {
                V vb = __ldg(reinterpret_cast<const V *>(sB + o));
                memcpy(xb[k], &vb, sizeof(V));
            }
        } else {
            const size_t ro = (size_t)clamp_idx(gi, n - 1) * p;
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const size_t o = ro + clamp_idx(gj + e, m - 1);
                xa[k][e] = ldc(sA, o, (size_t)n * p, kDbgHaloLoad);
                if (sB) xb[k][e] = ldc(sB, o, (size_t)n * p, kDbgHaloLoad);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = tid + k * NT;
        if (q >= NVEC) break;
        const int a = q / NV, b0 = (q % NV) * VN - 2;
#pragma unroll
        for (int e = 0; e < VN; ++e) {
            const int b = b0 + e;
            if (b >= 0 && b < 36) {
                dA[a][b] = xa[k][e];
                if (sB) dB[a][b] = xb[k][e];
            }
        }
    }
}

// Loads the 32 x 32 tile at (i0, j0) of one or two pitched grid functions into dst[32][33]
// (indices clamped into the domain; those values are never used), vector loads, NT threads.
template <typename T, int NT = 256>
__device__ __forceinline__ void load_tile32(T (*dA)[33], const T *sA, T (*dB)[33], const T *sB, int i0, int j0,
                                            int n, int m, int p, int tid) {
    using V = typename VecOf<T>::type;
    constexpr int VN = VecOf<T>::n, NV = 32 / VN, NVEC = 32 * NV, PER = (NVEC + NT - 1) / NT;
    T xa[PER][VN], xb[PER][VN];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = tid + k * NT;
        if (q >= NVEC) break;
        const int a = q / NV, gi = i0 + a, gj = j0 + (q % NV) * VN;
        if (gi < n && gj + VN <= m && MG_DBG_OK((size_t)gi * p + gj + VN - 1, (size_t)n * p, kDbgHaloLoad)) {
            const size_t o = (size_t)gi * p + gj;
            V va = __ldg(reinterpret_cast<const V *>(sA + o));
            memcpy(xa[k], &va, sizeof(V));
            if (sB) {
                V vb = __ldg(reinterpret_cast<const V *>(sB + o));
                memcpy(xb[k], &vb, sizeof(V));
            }
        } else {
            const size_t ro = (size_t)clamp_idx(gi, n - 1) * p;
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                const size_t o = ro + clamp_idx(gj + e, m - 1);
                xa[k][e] = ldc(sA, o, (size_t)n * p, kDbgHaloLoad);
                if (sB) xb[k][e] = ldc(sB, o, (size_t)n * p, kDbgHaloLoad);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = tid + k * NT;
        if (q >= NVEC) break;
        const int a = q / NV, b0 = (q % NV) * VN;
#pragma unroll
        for (int e = 0; e < VN; ++e) {
            dA[a][b0 + e] = xa[k][e];
            if (sB) dB[a][b0 + e] = xb[k][e];
        }
    }
}

// One-dimensional bilinear taps (Sec. 3.1): fine 2I+1 takes coarse I; fine 2I+2 the mean of
// coarse I and I+1; fine 0 (and fine n-1 for odd n) the single nearest coarse value.
__device__ __forceinline__ int bl_taps(int p, int nc, int *idx, float *wt) {
    if (p & 1) { idx[0] = (p - 1) / 2; wt[0] = 1.0f; return 1; }
    if (p == 0) { idx[0] = 0; wt[0] = 1.0f; return 1; }
    int I = p / 2 - 1;
    if (I + 1 < nc) { idx[0] = I; idx[1] = I + 1; wt[0] = 0.5f; wt[1] = 0.5f; return 2; }
    idx[0] = I; wt[0] = 1.0f;
    return 1;
}

// One-dimensional full-weighting taps (Sec. 3.1): coarse I sits on fine 2I+1; (1/4, 1/2, 1/4)
// on 2I, 2I+1, 2I+2, or (1/2, 1/2) on 2I, 2I+1 when fine 2I+2 does not exist.
__device__ __forceinline__ int fw_taps(int I, int n, int *idx, float *wt) {
    int q = 2 * I + 1;
    if (q + 1 < n) {
        idx[0] = q - 1; idx[1] = q; idx[2] = q + 1;
        wt[0] = 0.25f; wt[1] = 0.5f; wt[2] = 0.25f;
        return 3;
    }
    idx[0] = q - 1; idx[1] = q;
    wt[0] = 0.5f; wt[1] = 0.5f;
    return 2;
}

// Sum of squares of the residual values a thread visits: accumulated in the storage precision
// (a handful of values per thread), then widened to FP64 for the block and grid reductions.
// FP64 arithmetic is slow on this GPU, so the per-cell work stays in FP32 on the FP32 path.
template <typename T>
__device__ __forceinline__ T add_square(T acc, T r) { return fma_rn(r, r, acc); }

// Member mask of one 32-cell piece of a line from its star mask (bit t = position t):
// starred cells, plus for every starred cell without a starred neighbour its next cell, or
// its previous cell when it is the last cell of the piece (Sec. 4.3, "a single starred
// pixel is updated collectively with its immediate neighbour").  `len` = valid cells (1..32).
__device__ __forceinline__ uint32_t members_of(uint32_t star, int len) {
    uint32_t valid = len >= 32 ? 0xffffffffu : ((1u << len) - 1u);
    star &= valid;
    uint32_t single = star & ~(star << 1) & ~(star >> 1);
    uint32_t next = (single << 1) & valid;
    uint32_t last = single & ~(valid >> 1);   // singles at position len-1
    uint32_t prev = last >> 1;
    return star | next | prev;
}

}  // namespace segmg
