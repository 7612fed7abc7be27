// internal.h -- shared declarations of the CUDA library behind include/segmg.h.
//
// Storage: every grid function of level l is an n_l x m_l row-major array with a row pitch
// (in elements) rounded up to a multiple of 32, so rows start on 128-byte (f32) or 256-byte
// (f64) boundaries.  The unknown of a pseudo-time step is stored split as phi = pn + u:
// pn is phi^n restricted to the level (fixed during the step) and u the increment.  This keeps
// FP32 differences and the time term exact to the increment's own precision instead of the
// precision of |phi| (which reaches hundreds of pixels).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "debug.cuh"

namespace segmg {

constexpr int kChunk = 32;        // partial-line groups are cut at multiples of 32 cells
constexpr int kMaxLevels = 16;
constexpr int kMaxCoarseCells = 4096;
constexpr int kMaxCoarseBand = 64;
constexpr int kLoopMaxCycles = 128;   // cycle cap of an attempt run by the device step loop

// Partial-line group membership is stored as one 32-bit mask per 32-cell piece of a line:
// mrow[(k * n + i) * npm + (j >> 5)] bit (j & 31) for sweeps A (k = 0) and B (k = 1) along row
// i, and mcol[(k * m + j) * npn + (i >> 5)] bit (i & 31) for sweeps C (k = 0) and D (k = 1)
// along column j (npm = ceil(m / 32), npn = ceil(n / 32)).

template <typename T>
struct LevelView {
    int n, m, pitch;
    int level;
    T cdiff;        // mu / h^2
    T inv_tau;      // 1 / tau (0 for tau = inf)
    T Sigma;
    T inv_2h;       // 1 / (2h), central differences
    T beta;
    T *pn, *u, *u0, *rhs, *w, *z, *d, *F, *G, *f, *r, *upre;
    T *t;                      // the fused sweeps' second buffer: A and C read u and write t,
                               // B and D read t and write u (a sweep never reads what it writes)
    uint32_t *mrow, *mcol;     // member masks (see above)
    int npm, npn;
    const __nv_bfloat16 *wb;   // mixed precision: the length weight w stored in BF16 (else NULL)
    uint8_t *cls;              // Hybrid Smoother 1 only: per cell 1 << (index of the smallest of
                               // A..D) if the cell is in D, else 0 (else NULL)
    const T *omega;            // relaxation weights of the Hybrid Smoother 2 point updates
                               // (phi += omega (g - phi)); NULL: plain updates
    int has_rhs;    // 0 on the finest grid (zero right-hand side)
};

// Device-resident scalars (double) shared by the kernels of one handle.
struct Scalars {
    double c1, c2;           // region averages
    double A1frac;           // initial polygon area / (n m)
    double area[kMaxLevels]; // Rada-Chen area term of each level (lagged)
    double norm2;            // sum r^2 of the last finest residual
    double norm2_0;          // sum r^2 of L(phi^n)
    double sums[8];          // sum H z, sum H, sum (1-H) z, sum (1-H), sum u^2, sum phi_n^2
    double coarse_res;       // last coarsest nonlinear residual
    double aos[2];           // AOS on the finest grid: sum (u_new - u)^2, sum (pn + u)^2
    int picard;              // Picard iterations of the last coarsest solve
    int err;                 // 1 = non-positive Cholesky pivot
    int halt;                // nonzero: a batch skips this image's V-cycles (set by the host when
                             // the image gives up a step; cleared by every step's start)
    // the step loop on the device (one graph launch runs an attempt's V-cycles): V-cycles run,
    // why the loop ended (1 tolerance, 2 stalled, 3 cycle cap, 4 diverged or non-finite, 5 an
    // error bit), and rho after each V-cycle (1-based)
    int loop_j, loop_stop;
    double loop_rho[kLoopMaxCycles + 1];
};

struct ModelParams {
    int model;
    double mu, lambda1, lambda2, theta, nu, eps, beta;
};

// Member bit of cell (i, j) in sweep 0..3 (A, B, C, D).
template <typename T>
__device__ __forceinline__ bool member_bit(const LevelView<T> &L, int sweep, int i, int j) {
    if (sweep < 2)
        return (ldc(L.mrow, ((size_t)sweep * L.n + i) * L.npm + (j >> 5), (size_t)2 * L.n * L.npm, kDbgMaskLoad) >>
                (j & 31)) & 1u;
    return (ldc(L.mcol, ((size_t)(sweep - 2) * L.m + j) * L.npn + (i >> 5), (size_t)2 * L.m * L.npn, kDbgMaskLoad) >>
            (i & 31)) & 1u;
}

// The length weight w of cell o: BF16 storage in mixed precision, else the storage type.
template <typename T>
__device__ __forceinline__ T weight_at(const LevelView<T> &L, size_t o) {
    const size_t lim = (size_t)L.n * L.pitch;
    return L.wb ? T(__bfloat162float(ldc(L.wb, o, lim, kDbgSnapshot))) : ldc(L.w, o, lim, kDbgSnapshot);
}

// ---- launchers (each enqueues on `st`) -------------------------------------------------

// setup_kernels.cu
template <typename T>
void launch_blur(const T *src, T *tmp, T *dst, int n, int m, int pitch_src, int pitch, const double *taps,
                 int R, cudaStream_t st);
template <typename T>
void launch_edge_distance(const T *zb, T *w, T *d, int n, int m, int pitch, double beta_edge,
                          const double *mk, int k, double sigma_d, int model, cudaStream_t st);
// The n x m image (row-major, no padding) into the pitched finest z; bit 2 of *flag is set
// when a value is NaN or Inf.
template <typename T>
void launch_copy_in(const T *src, T *dst, int n, int m, int pitch, int *flag, cudaStream_t st);
template <typename T>
void launch_copy_out(const T *src, T *dst, int n, int m, int pitch, cudaStream_t st);
template <typename T>
void launch_initial_phi(T *pn, T *u, int n, int m, int pitch, const double *hull, int nh,
                        double cx, double cy, double r0, cudaStream_t st);
template <typename T>
void launch_restrict(const T *f, int n, int m, int pf, T *c, T *c2, int pc, cudaStream_t st);
// Up to three fields of the same grid restricted in one launch (c2[q] may be NULL).
template <typename T>
struct RestrictFields {
    const T *f[3];
    T *c[3], *c2[3];
    int nf;
};
template <typename T>
void launch_restrict_fields(const RestrictFields<T> &F, int n, int m, int pf, int pc, cudaStream_t st);
// Per-grid pointers and sizes of the fitting fields of all grids (one launch).
template <typename T>
struct FitGrids {
    const T *z[kMaxLevels], *d[kMaxLevels];
    T *F[kMaxLevels];
    int n[kMaxLevels], m[kMaxLevels], pitch[kMaxLevels], first_block[kMaxLevels];
    int nlev;
};
template <typename T>
void launch_fitting(const LevelView<T> *L, int nlev, const Scalars *sc, ModelParams mp, cudaStream_t st);
template <typename T>
void launch_fold(const LevelView<T> &L, cudaStream_t st);
template <typename T>
void launch_region_sums(const LevelView<T> &L, double eps, double *partials, int npart,
                        Scalars *sc, int finalize_c, cudaStream_t st);
template <typename T>
void launch_mask(const LevelView<T> &L, uint8_t *mask, cudaStream_t st);
void launch_to_bf16(const float *src, __nv_bfloat16 *dst, int n, int m, int pitch, cudaStream_t st);
template <typename T>
void launch_area(const LevelView<T> &L, const T *uin, double eps, double nu, double h2_over_nm,
                 double *partials, int npart, double *out, const Scalars *sc, cudaStream_t st);
template <typename T>
void launch_energy(const LevelView<T> &L, ModelParams mp, double *partials, int npart, const Scalars *sc,
                   double *out, cudaStream_t st);
int num_partials(int n, int m);

// smooth_kernels.cu
template <typename T>
void launch_snapshot(const LevelView<T> &L, const double *area, cudaStream_t st);
constexpr int kTileShapes = 6;   // fused-sweep tile shapes (rows x columns, threads): 32x64 256, 32x32 128,
                                 // 64x64 512, 32x64 512, 32x32 256, 32x32 512 (see smooth_kernels.cu)
template <typename T>
void launch_sweep_fused(const LevelView<T> &L, int sweep, int shape, cudaStream_t st);
template <typename T>
void launch_sweep_phased(const LevelView<T> &L, int sweep, cudaStream_t st);

// line_smoothers.cu: GSLINE-I (zebra columns) and the Hybrid Smoother 1 blocks
template <typename T>
void launch_gsline(const LevelView<T> &L, cudaStream_t st);
template <typename T>
void launch_hs1_blocks(const LevelView<T> &L, cudaStream_t st);

// sweep_tma.cu: the fused sweep for FP32 storage with TMA-staged tiles.  A SweepMaps holds the
// tensor maps (CUtensorMap, 128 bytes each) of u, t, G and f of one grid for one tile shape.
struct SweepMaps {
    alignas(64) unsigned char u[128];
    alignas(64) unsigned char t[128];
    alignas(64) unsigned char G[128];
    alignas(64) unsigned char f[128];
};
// Tensor maps of the TMA-staged snapshot of one FP32 grid (snapshot_tma.cu): pn, u and w boxes
// of 36 rows (w in BF16 when mixed), F and rhs tiles of 32 x 32.
struct SnapMaps {
    alignas(64) unsigned char P[128];
    alignas(64) unsigned char U[128];
    alignas(64) unsigned char W[128];
    alignas(64) unsigned char F[128];
    alignas(64) unsigned char R[128];
    bool mixed = false;
};
void prepare_snapshot_tma();
bool encode_snapshot_maps(const LevelView<float> &L, SnapMaps *M);
// The snapshot of an FP32 grid (the operations of launch_snapshot); a copy that does not
// complete within wait_limit try_wait rounds sets bit 4 of *err.
void launch_snapshot_tma(const LevelView<float> &L, const double *area, const SnapMaps &M, int *err,
                         long long wait_limit, cudaStream_t st);
// The same snapshot (8 warps per tile) that also writes each tile's sum of r^2, r = rhs - L(pn + u)
// at the state it reads, to partials: bitwise the partials of launch_residual_tma's norm.
// The first snapshot of a coarse grid right after its restriction (u = u0): also completes the
// FAS right-hand side, rhs += L(pn + u0), written back and used in f (the separate mode-1
// residual launch then does not run).
void launch_snapshot_fas_tma(const LevelView<float> &L, const double *area, const SnapMaps &M, int *err,
                             long long wait_limit, cudaStream_t st);
// The first snapshot of grid L's post-smoothing: first applies the coarse-grid correction
// u += P (u_c - u0_c) from grid C (Algorithm 1's interpolation) and writes u (the separate
// interpolation launch then does not run).
void launch_snapshot_interp_tma(const LevelView<float> &L, const LevelView<float> &C, const double *area,
                                const SnapMaps &M, int *err, long long wait_limit, cudaStream_t st);
void launch_snapshot_norm_tma(const LevelView<float> &L, const double *area, const SnapMaps &M, double *partials,
                              int *err, long long wait_limit, cudaStream_t st);
// Tensor maps of the TMA-staged residual kernels of one FP32 grid (residual_tma.cu): pn, u and w
// boxes of 37 rows and F and rhs tiles of 33 x 36 (the residual with restriction), and the u0
// box of 36 rows (the FAS right-hand side).
struct ResMaps {
    alignas(64) unsigned char P37[128];
    alignas(64) unsigned char U37[128];
    alignas(64) unsigned char W37[128];
    alignas(64) unsigned char F33[128];
    alignas(64) unsigned char R33[128];
    alignas(64) unsigned char U0[128];
};
void prepare_residual_tma();
bool encode_residual_maps(const LevelView<float> &L, ResMaps *R);
// launch_residual for an FP32 grid (uin = the grid's u, or its u0 when uin_is_u0; out may be
// NULL in mode 0 when only the norm is wanted) and launch_residual_restrict, with the same
// operations; a copy that does not complete within wait_limit try_wait rounds sets bit 4 of *err.
void launch_residual_tma(const LevelView<float> &L, int uin_is_u0, const double *area, float *out, int mode,
                         double *partials, int npart, double *norm_out, const SnapMaps &M, const ResMaps &R, int *err,
                         long long wait_limit, cudaStream_t st);
void launch_residual_restrict_tma(const LevelView<float> &L, const LevelView<float> &C, const double *area,
                                  const ResMaps &R, int *err, long long wait_limit, cudaStream_t st);
// Sums np FP64 partials in a fixed order into *out (one block).
// Sum of np partials into *out in a fixed order.  Above 1024 partials the chunk sums are kept
// in the ceil(np / 1024) doubles after the partials, so the buffer must hold that many more.
void launch_sum_partials(double *partials, int np, double *out, cudaStream_t st);
// stage[k * G + b] = sum of part[k * np + 1024 b .. 1024 (b + 1)) for k < K, G = ceil(np / 1024).
void launch_chunk_sums(const double *part, int np, int K, double *stage, cudaStream_t st);
void prepare_sweep_tma();
bool encode_sweep_maps(const LevelView<float> &L, int shape, SweepMaps *M);
// One n x m grid function (FP32: elem 4, BF16: elem 2) with row pitch `pitch` elements as a 2-D
// tensor map with box RW x RH (zero fill outside the grid); false when the driver refuses it.
bool encode_map_2d(void *out, void *base, int elem, int n, int m, int pitch, int RH, int RW);
constexpr long long kDefaultWaitLimit = 1LL << 22;   // try_wait rounds before a TMA wait gives up
void launch_sweep_tma(const LevelView<float> &L, int sweep, int shape, const SweepMaps &M, int *err,
                      long long wait_limit, cudaStream_t st);

// learned.cu: learned relaxation weights (inference and training)
int learned_nparam();
int learned_crop();
size_t learned_record_floats();
void prepare_learned_kernels();
template <typename T>
void launch_omega_infer(const LevelView<T> &L, const __nv_bfloat16 *net, T *omega, cudaStream_t st);
template <typename T>
void launch_record_crops(const LevelView<T> &L, const int *origins, int count, float *data, int first,
                         cudaStream_t st);
void launch_train_step(float *theta, float *mom, float *vel, const float *data, const int *idx, int batch,
                       float *grad, float *loss, float *gmean, float *lmean, float lr, int step, int loss_kind,
                       cudaStream_t st);

// cycle_kernels.cu
template <typename T>
void launch_residual(const LevelView<T> &L, const T *uin, const double *area, T *out, int mode,
                     double *partials, int npart, double *norm_out, cudaStream_t st);
template <typename T>
void launch_interp_add(const LevelView<T> &Lf, const LevelView<T> &Lc, cudaStream_t st);
template <typename T>
void launch_coarse_solve(const LevelView<T> &L, int fp64, ModelParams mp, double A1frac,
                         double h2_over_nm, int maxit, double tol, double *scratch, Scalars *sc,
                         int aos, double aos_dt, cudaStream_t st);   // fp64: FP64 arithmetic for FP32
                                                                    // storage; aos: AOS iterations
template <typename T>
void launch_aos_iteration(const LevelView<T> &L, const double *area, double dt, double *partials, double *sums,
                          cudaStream_t st);
void prepare_coarse_kernels();
// FP32 grids: the residual and the full weighting of r and u onto the coarse grid in one kernel
void launch_residual_restrict(const LevelView<float> &L, const LevelView<float> &C, const double *area,
                              cudaStream_t st);

// Scratch elements (of the storage type) of the coarsest solve on an n x m grid.
__host__ __device__ inline size_t coarse_scratch_elems(int n, int m) {
    size_t N = (size_t)n * m, bw = (size_t)(m > n ? n : m);
    return 4 * N + N * (bw + 1);
}

// bottom_kernel.cu: grids lb .. L-1 of a V-cycle (FP32 storage, Spencer-Chen model) in one block
struct BottomArgs {
    int lb, L, nu1, nu2;
    int coarse_fp64;   // the coarsest solve in FP64 arithmetic (mixed precision) or FP32
    int coarse_aos;    // the coarsest solve by AOS iterations (step aos_dt)
    double aos_dt;
    LevelView<float> g[kMaxLevels];
    ModelParams mp;
    double A1frac, h2nm_coarse, coarse_tol;
    int coarse_maxit;
    Scalars *sc;
};
constexpr size_t kBottomSmemMax = 200 * 1024;
constexpr int kBottomThreads = 1024;   // threads of the bottom kernels' blocks
size_t bottom_smem_bytes(const int *n, const int *m, int lb, int L, int coarse_fp64);
void prepare_bottom_kernel();
void launch_bottom(const BottomArgs &A, size_t smem, cudaStream_t st);
// The bottom of the V-cycle from grid A.lb spread over a cluster of `tiles` CTAs (one per 32 x 32
// tile, at most kClusterMaxTiles), CTA 0 holding grids A.lb+1 .. L-1.  smem = cluster_smem_bytes
// of the shared memory of grids A.lb+1 .. L-1; cluster_fits returns how many such clusters can
// be resident (0: none or out of range; negative: minus the CUDA error of the query).
constexpr int kClusterMaxTiles = 16;
constexpr size_t kClusterSmemMax = 220 * 1024;   // dynamic, beside the kernel's static shared memory
size_t cluster_smem_bytes(size_t bottom_bytes);
int cluster_fits(int tiles, size_t smem);
void launch_cluster(const BottomArgs &A, int tiles, size_t smem, cudaStream_t st);

}  // namespace segmg
