/*
 * segmg.h -- C ABI of the GB300 (sm_103a) multigrid solver for level-set selective
 * segmentation.  Method: Roberts, Chen, Irion, "A multigrid algorithm with non-standard
 * smoother for two selective models in variational segmentation" (arXiv 1807.02137).
 *
 * The library solves the discretised Euler-Lagrange equation of the Spencer-Chen model
 * (Sec. 2.2, eq. scel) or the Rada-Chen model (eq. rcel, discretised as eqs. rcabcd/abcdrc) by
 * nonlinear FAS V-cycles (Sec. 3.1, Algorithm 1) whose smoother is Hybrid Smoother 2
 * (Sec. 4.3), run in a parallel ordering (checkerboard point updates plus partial-line solves
 * on alternating lines).  Because the stationary equation has no bounded solution for generic
 * images, each call to the solver advances one implicit pseudo-time step
 *     N(phi) - delta(phi) (phi - phi^n) / tau = 0,
 * whose solution set equals that of the row-scaled equation
 *     L(phi) = mu div_h(w grad phi / |grad phi|_beta) - F - (phi - phi^n)/tau = 0,
 * and the FAS residual is measured on L.  The paper's stationary equation is tau = inf.
 *
 * Conventions shared by every entry point:
 *   - images and grid functions are n x m, row-major, element [i*m + j], i = row (down),
 *     j = column (right); pixel units (finest spacing h = 1);
 *   - markers are k pairs (x, y) = (column, row) of doubles in HOST memory;
 *   - "device" pointers are CUDA device memory owned by the caller, "host" pointers are host
 *     memory owned by the caller; the library never frees caller memory;
 *   - the element type of an image / phi buffer is float for MG_F32 and MG_MIXED, double for
 *     MG_F64;
 *   - every function returns MG_OK (0) or a negative MG_ERR_* code; mg_strerror() names it and
 *     mg_last_error() returns the detail text of the last failure on the calling thread;
 *   - work is enqueued on the handle's stream; only calls that return host values wait for it;
 *   - handles are not thread-safe; distinct handles may be used from distinct threads.
 */
#ifndef SEGMG_H
#define SEGMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MG_OK = 0,
    MG_ERR_ARG = -1,        /* invalid argument (size, pointer, parameter) */
    MG_ERR_NAN = -2,        /* NaN or Inf in the input image or in a residual norm */
    MG_ERR_CUDA = -3,       /* a CUDA runtime call failed (detail in mg_last_error) */
    MG_ERR_DIVERGED = -4,   /* residual grew by more than 1e3 over its initial value */
    MG_ERR_TIMEOUT = -5,    /* an iteration cap was reached without meeting the tolerance, or a
                               bounded wait on the device gave up (mg_set_wait_limit) */
    MG_ERR_NOT_SPD = -6,    /* coarsest-grid Cholesky met a non-positive pivot */
    MG_ERR_NOMEM = -7,      /* device allocation failed */
    MG_ERR_STATE = -8       /* call out of order (e.g. mg_vcycle before mg_begin_step) */
};

enum { MG_MODEL_SC = 0, MG_MODEL_RC = 1 };       /* Spencer-Chen / Rada-Chen (Sec. 2.2) */
enum { MG_F32 = 0, MG_F64 = 1, MG_MIXED = 2 };  /* storage and smoothing precision; MG_MIXED = FP32
                                                    with the image-derived weight w held in BF16 */
/* Smoothers.  Hybrid Smoother 2 (Sec. 4.3, the paper's Algorithm 3), three kernel variants with
 * the same results: one kernel per sweep with tiles staged by the Tensor Memory Accelerator
 * (FP64 storage: by vector loads), one kernel per phase, or one kernel per sweep with vector
 * loads.  The paper's other smoothers, in parallel orderings: GSLINE-I (Sec. 3.2, Algorithm 1;
 * even columns, then odd columns) and Hybrid Smoother 1 (Sec. 4.2, Algorithm 2; GSLINE-I, then
 * the arrow-system blocks of the set D in 16 classes (i mod 4, j mod 4)). */
enum {
    MG_SMOOTH_FUSED = 0,
    MG_SMOOTH_PHASED = 1,
    MG_SMOOTH_FUSED_VEC = 2,
    MG_SMOOTH_GSLINE = 3,
    MG_SMOOTH_HS1 = 4
};

enum { MG_COARSE_PICARD = 0, MG_COARSE_AOS = 1 };   /* coarsest-grid solver */

typedef struct mg_handle_s *mg_handle;

/* Parameters.  Model weights follow Sec. 2.2 (eqs. rcfunc, scfunc); the smoother and cycle
 * settings follow Sec. 3-4 and Sec. 5 ("Parameter choices", "Number of smoothing steps"). */
typedef struct {
    int model;             /* MG_MODEL_SC or MG_MODEL_RC */
    double mu;             /* length-term weight (> 0) */
    double lambda1;        /* inside fitting weight (>= 0) */
    double lambda2;        /* outside fitting weight (>= 0) */
    double theta;          /* Spencer-Chen distance weight (>= 0) */
    double nu;             /* Rada-Chen area weight (>= 0) */
    double eps;            /* smoothed Heaviside width (> 0) */
    double beta;           /* |grad phi|_beta = sqrt(|grad phi|^2 + beta) (> 0) */
    double beta_edge;      /* edge detector g(s) = 1 / (1 + beta_edge s), s = |grad G*z|^2 */
    double sigma_blur;     /* Gaussian blur of the image before differencing (px, > 0) */
    double sigma_d;        /* width of the marker distance function (px, > 0) */
    double Sigma;          /* jump threshold: max/min of the four coefficients (> 1) */
    double tau;            /* pseudo-time step (px^2-time units, > 0; 0 means infinity) */
    int nu1, nu2;          /* pre- and post-smoothing outer iterations (>= 0) */
    int levels;            /* number of grids, finest included (>= 1) */
    int precision;         /* MG_F32, MG_F64 or MG_MIXED (norms and c1/c2 sums are FP64 in every
                              mode; the coarsest solve is FP32 with MG_F32, else FP64) */
    int smoother;          /* MG_SMOOTH_* */
    int coarse_maxit;      /* Picard cap of the coarsest solve (>= 1) */
    double coarse_tol;     /* relative residual target of the coarsest solve */
    int use_graph;         /* 1: replay each V-cycle as a captured CUDA graph */
    int coarse_solver;     /* MG_COARSE_PICARD, or MG_COARSE_AOS: coarse_maxit AOS iterations of
                              step aos_dt (Algorithm 1 "time-marching or AOS"; Sec. 5 uses 100) */
    double aos_dt;         /* AOS artificial time step (> 0) */
    double stall_ratio;    /* pseudo-time step control of mg_solve_step / mg_solve / the batch: an
                              attempt at a step is rejected when, from its 4th V-cycle on,
                              rho_j > stall_ratio * rho_{j-2}, when a V-cycle diverges or returns a
                              non-finite residual, or when the cycle cap is reached; phi is then
                              restored to phi^n and the step is retried with tau / 2.  0 switches
                              the control off (0 <= stall_ratio < 1; default 0.6) */
    int max_halvings;      /* rejected attempts allowed per step (>= 0; default 10) */
} mg_params;

/* Counters and scalars of the current state (mg_get_stats). */
typedef struct {
    int n, m, levels, precision;
    int steps;             /* pseudo-time steps ended so far */
    int cycles_step;       /* V-cycles in the current / last step */
    int cycles_total;
    int picard_last;       /* Picard iterations of the last coarsest solve */
    double rho;            /* last ||L(phi)|| / ||L(phi^n)|| */
    double res0;           /* ||L(phi^n)|| of the current step */
    double eta;            /* last ||phi^{n+1} - phi^n|| / ||phi^n|| */
    double c1, c2;         /* region averages (eq. c1c2) */
    double A1;             /* area of the initial polygon (px^2) */
    size_t device_bytes;   /* device memory held by the handle */
    long long launches;    /* kernels launched by the handle so far (graph nodes included) */
    long long learned_accepted;   /* V-cycles run with learned relaxation weights and kept */
    long long learned_rejected;   /* ... and rejected (rerun with the plain smoother) */
    int bottom_level;      /* first grid of the one-block bottom kernel, -1 when it is not used */
    int cluster_level;     /* first grid of the cluster bottom kernel, -1 when it is not used */
    double tau;            /* pseudo-time step of the next / current step (halved by the control) */
    int attempts_rejected; /* step attempts rejected by the step control so far */
} mg_stats;

/* Optional device allocator (for example a framework's caching allocator).  alloc returns a
 * device pointer of at least `bytes` bytes, 256-byte aligned, usable on `stream`; free
 * releases it.  A NULL mg_allocator selects cudaMallocAsync / cudaFreeAsync. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} mg_allocator;

/* Fills *p with the defaults: Spencer-Chen, mu = 1, lambda1 = lambda2 = 10, theta = 1,
 * nu = 1, eps = 1, beta = 1e-6, beta_edge = 1, sigma_blur = 1, sigma_d = 0.05 max(n, m),
 * Sigma = 2, tau = 1, V(2,2), levels = as many halvings as keep min(n, m) >= 4 (at most 12),
 * MG_F32, fused smoother, coarse_maxit = 100, coarse_tol = 1e-13, use_graph = 1,
 * stall_ratio = 0.6, max_halvings = 10. */
int mg_default_params(mg_params *p, int n, int m);

/* Builds a solver for one n x m image (Sec. 2.2 data, Sec. 5 initialisation):
 *   image      device, n*m elements of the precision's type, read during the call only;
 *   markers_xy host, k (x, y) pairs inside [0, m-1] x [0, n-1], k >= 1;
 *   p          parameters (copied);  alloc may be NULL;  stream may be NULL (the library
 *              then creates its own non-blocking stream).
 * Computes the blurred image, edge detector g, distance function d, weight w (g for SC,
 * d g for RC), their restrictions to every grid, the initial level set (signed distance to
 * the convex hull of the markers; a disc of radius 0.05 max(n, m) for fewer than three or
 * collinear markers) and the initial c1, c2.  Allocates all device memory the solver needs
 * (mg_stats.device_bytes).  Errors: MG_ERR_ARG (sizes, markers, parameters, a coarsest grid
 * above 4096 cells or 64 cells on its shorter side), MG_ERR_NAN (non-finite image),
 * MG_ERR_NOMEM, MG_ERR_CUDA.  On error *out is NULL and nothing is leaked. */
int mg_setup(mg_handle *out, const void *image, int n, int m, const double *markers_xy, int k,
             const mg_params *p, const mg_allocator *alloc, void *stream);

/* Re-runs the set-up of mg_setup on a new image and marker set of the same size, reusing the
 * handle's memory (no allocation).  Same arguments and errors as mg_setup. */
int mg_reset(mg_handle h, const void *image, const double *markers_xy, int k);

/* Starts a pseudo-time step from the current phi: phi^n = phi, fitting fields of every grid
 * from c1, c2, and the reference norm ||L(phi^n)|| (written to *res0 if not NULL; waits for
 * the stream). */
int mg_begin_step(mg_handle h, double *res0);

/* One FAS V-cycle (Algorithm 1, gamma = 1) with nu1 / nu2 outer iterations of Hybrid
 * Smoother 2 per grid and the FP64 coarsest solve; writes rho = ||L(phi)|| / ||L(phi^n)||
 * (FP64 accumulation) to *rho if not NULL (waits for the stream).  MG_ERR_STATE before
 * mg_begin_step; MG_ERR_NAN / MG_ERR_DIVERGED / MG_ERR_NOT_SPD as detected. */
int mg_vcycle(mg_handle h, double *rho);

/* Ends the step: new c1, c2 from the current phi (Sec. 5) and
 * eta = ||phi - phi^n|| / ||phi^n|| (to *eta if not NULL, and the call waits for the stream;
 * with eta NULL the call only enqueues, and mg_stats reads eta later). */
int mg_end_step(mg_handle h, double *eta);

/* mg_begin_step, then V-cycles until rho <= tol or max_cycles, then mg_end_step.
 * With the step control on (params.stall_ratio > 0) an attempt that stalls, diverges or reaches
 * max_cycles is rejected: phi is restored to phi^n, tau is halved (it stays halved for the
 * following steps) and the step starts again, up to params.max_halvings times.  The paper solves
 * the stationary equation and stops on the relative change (Sec. 5), so it has no rule for the
 * pseudo-time steps; this is the reading this library takes for them.
 * *cycles (may be NULL) gets the V-cycles of all attempts, *rho the last residual ratio.
 * Returns MG_ERR_TIMEOUT (state still valid: the last attempt's phi) when no attempt reached tol. */
int mg_solve_step(mg_handle h, double tol, int max_cycles, int *cycles, double *rho);

/* Pseudo-time steps (each by mg_solve_step) until eta < eta_stop or max_steps; *steps gets
 * the number taken.  A step that reaches its cycle cap does not stop the run. */
int mg_solve(mg_handle h, double tol, int max_cycles, double eta_stop, int max_steps, int *steps);

/* Segmentation mask: mask[i*m + j] = 1 where phi > 0 else 0.  mask: device, n*m bytes. */
int mg_mask(mg_handle h, unsigned char *mask);

/* Copies phi (device, n*m elements of the precision's type) out of / into the solver. */
int mg_get_phi(mg_handle h, void *phi);
int mg_set_phi(mg_handle h, const void *phi);

/* Overrides c1, c2 (eq. c1c2) for the next mg_begin_step. */
int mg_set_regions(mg_handle h, double c1, double c2);

/* Copies one internal field of grid `level` (device, n_l*m_l elements of the precision's type;
 * n_l = n >> level): field 0 = phi, 1 = w, 2 = z, 3 = d, 4 = F (fitting field of the step),
 * 5 = FAS right-hand side, 6 = G of the last coefficient snapshot, 7 = the relaxation weights
 * (mg_set_learned / mg_set_omega).  For tests and diagnostics. */
int mg_get_level(mg_handle h, int level, int field, void *out);

int mg_get_stats(mg_handle h, mg_stats *s);

/* Bound of the device-side waits of the FP32 kernels staged by the Tensor Memory Accelerator
 * (fused sweep, coefficient snapshot, residual kernels: the copies of a tile into shared memory
 * complete on an mbarrier; each wait polls it at most `rounds` times, default 4,194,304).  When a wait gives up, the block records it, waits once more (with the
 * default bound) for the copies it has in flight, and ends; the next mg_vcycle / mg_solve_step
 * returns MG_ERR_TIMEOUT and the handle stays usable.  rounds = 0 makes every such wait give up at
 * once (for tests of that path).  A diagnostic setting of this implementation; the paper has no
 * counterpart.  Errors: MG_ERR_ARG (rounds < 0). */
int mg_set_wait_limit(mg_handle h, long long rounds);

/* Host-side fault injection for tests of the error paths (no counterpart in the paper): the
 * `cycle`-th V-cycle (1-based, counted from the start of the current or next step attempt) run
 * after this call reports a residual ratio of 1e9, as a diverged V-cycle would; mg_vcycle then
 * returns MG_ERR_DIVERGED and the step control of mg_solve_step rejects the attempt.  It fires
 * once; 0 cancels it.  The device state is left as the V-cycle computed it.  Errors: MG_ERR_ARG. */
int mg_inject_divergence(mg_handle h, int cycle);

/* Index bounds checks of the debug build (no counterpart in the paper).  A library compiled with
 * -DMG_DEBUG compares the index of each checked global-memory access of its kernels with the size
 * of the buffer it addresses; an out-of-range access is skipped (a load reads 0), never trapped,
 * and recorded in device error words (one set per compiled source file).  mg_debug_status waits
 * for the device, ORs the words of all files into *out and, if clear is nonzero, zeroes them.
 * In the default build it reports enabled = 0 and nothing else.  Errors: MG_ERR_ARG (NULL out),
 * MG_ERR_CUDA. */
typedef struct mg_debug_info {
    int enabled;                 /* 1: the library was built with MG_DEBUG */
    int first_site;              /* site of the first out-of-range index one file recorded, -1: none
                                  * (0 set-up, 1 tile loads, 2 snapshot, 3 mask stores, 4 mask
                                  * loads, 5 sweeps, 6 residual / restriction, 7 interpolation,
                                  * 8 bottom kernels, 9 coarsest solve, 10 other smoothers) */
    long long first_index;       /* that index (elements of the addressed buffer) */
    unsigned long long sites;    /* bit s: site s saw an out-of-range index */
    long long count;             /* out-of-range accesses skipped, all files */
} mg_debug_info;
int mg_debug_status(mg_debug_info *out, int clear);

/* Test of the reporting path of the debug build: a one-thread kernel passes the index limit + 5
 * through the check of site 10 with no memory access behind it, so mg_debug_status then shows
 * site 10, that index and one more count.  Synchronous.  Does nothing in the default build. */
int mg_debug_selftest(void);

/* Whole pipeline through host buffers: copies the float image to the device, runs mg_setup (or
 * mg_reset on the context kept from the previous call, see below), then mg_solve(tol,
 * max_cycles, eta_stop, max_steps) with the given parameters (precision forced to MG_F32), and
 * copies the mask (and phi if phi_host is not NULL) back.  All host buffers are n*m elements
 * (page-locked buffers copy fastest); stats may be NULL.  Synchronous. */
int mg_segment_host(const float *image_host, int n, int m, const double *markers_xy, int k,
                    const mg_params *p, double tol, int max_cycles, double eta_stop,
                    int max_steps, unsigned char *mask_host, float *phi_host, mg_stats *stats);

/* mg_segment_host keeps its handle, device buffers and stream after a successful call: the next
 * call on the same device with the same size and parameters (and at most max(k, 16) markers)
 * reuses them through mg_reset, which redoes the image's set-up, so only the copies, the set-up
 * kernels and the solve remain per call.  Calls are serialised by a lock.  A call with another
 * size or other parameters, or a failed call, frees the kept context first.
 * mg_segment_host_release frees it (before cudaDeviceReset, for example). */
void mg_segment_host_release(void);

/* Tile-shape autotuner (a tuning step of this implementation; the paper has no counterpart):
 * inside a pseudo-time step (after mg_begin_step), times one outer smoothing iteration of every
 * grid but the coarsest with each fused-sweep tile shape (rows x columns of cells, threads per
 * tile: 0 = 32x64/256, 1 = 32x32/128, 2 = 64x64/512, 3 = 32x64/512, 4 = 32x32/256,
 * 5 = 32x32/512) over `reps` repetitions and keeps the fastest per grid; writes the choices to
 * shapes[0..levels-2] if not NULL.  Then, when the bottom kernel is in use, it times `reps`
 * V-cycles with the one-block bottom kernel starting at the largest grid that fits and at the next
 * two coarser grids, and with the cluster bottom kernel (mg_set_cluster_level) from the grid before
 * and from that largest grid where such a cluster fits, and keeps the fastest
 * (mg_stats.bottom_level, mg_stats.cluster_level).  The state is restored, and the
 * results of later solves do not depend on these choices (every choice computes the same
 * values).  Waits. */
int mg_autotune(mg_handle h, int reps, int *shapes);
/* Sets the fused-sweep tile shape of grids 0..levels-2 (values 0..5 as above). */
int mg_set_tile_shapes(mg_handle h, const int *shapes);
/* AOS time marching on the finest grid for the current pseudo-time step: the AOS method the
 * paper compares against in Table 6 (additive operator splitting of d phi / ds = L(phi) - rhs,
 * coefficients frozen per iteration, the 1/tau term split evenly between rows and columns):
 *   phi <- 1/2 sum_{l = rows, columns} ((1 + dt/tau) I - 2 dt A_l)^{-1} (phi + dt c).
 * Runs up to max_iter iterations of step dt (> 0), stopping when the relative change
 * ||phi^{k+1} - phi^k|| / ||phi^k|| is at most eta (the paper's stopping test).  *iters and
 * *rho (host, may be NULL) get the iterations run and ||L(phi)|| / ||L(phi^n)||.  Call between
 * mg_begin_step and mg_end_step; waits.  Errors: MG_ERR_ARG, MG_ERR_STATE, MG_ERR_CUDA. */
int mg_aos(mg_handle h, double dt, int max_iter, double eta, int *iters, double *rho);

/* Learned relaxation weights (an extension in the spirit of Sec. 4, which designs the smoother
 * cell by cell from the local coefficients).  Every non-member point update of Hybrid Smoother 2
 * becomes phi += omega (g - phi), with omega = 2 sigmoid(z) in (0, 2) and z from a network of
 * three 3x3 convolutions.  The network is 5 -> 16 (ReLU) -> 16 (ReLU) -> 1 channels with zero
 * padding at the grid boundary.  Its input per cell is its four face values of G (S, N, E, W;
 * zero on a boundary face) divided by their sum, and log(max / min of the existing faces) / 8.
 * Inference stores weights and activations in BF16 and accumulates in FP32.  The weights apply
 * on the grids the per-grid kernels smooth; the one-block bottom kernel smooths without them.
 *   theta    host, mg_learned_nparam() floats (3201): W1 (16,5,3,3), b1 (16), W2 (16,16,3,3),
 *            b2 (16), W3 (1,16,3,3), b3; NULL keeps the current parameters;
 *   mode     0 off; 1 every V-cycle after the first of a step runs with the weights and is kept
 *            only if its residual falls at least as fast as the last plain V-cycle's, else the
 *            state is restored and the V-cycle rerun plain, and the next 1, 2, 4 or 8 V-cycles
 *            (doubling with consecutive rejections) run plain; 2 always with the weights;
 *   refresh  V-cycles between two inferences (>= 1); the weights are computed from the first
 *            snapshot of each grid in a V-cycle that infers.
 * Requires MG_SMOOTH_FUSED or MG_SMOOTH_FUSED_VEC.  Errors: MG_ERR_ARG, MG_ERR_NOMEM. */
int mg_set_learned(mg_handle h, const float *theta, int mode, int refresh);
int mg_learned_nparam(void);
/* Fixed relaxation weights of grid `level` (host, n_l x m_l values of the storage type, row
 * major), used by every following V-cycle; NULL switches them off.  Grids the bottom kernel
 * smooths are refused (MG_ERR_ARG). */
int mg_set_omega(mg_handle h, int level, const void *omega);

/* Training of the learned weights on crops of 24 x 24 cells recorded from solves.  A crop record
 * holds 7 planes of 24 x 24 floats: the row-scaled coefficients c_S, c_N, c_E, c_W
 * (mu/h^2 times the face values of G), the snapshot right-hand side f, the increment u, and in
 * the last plane [0] = 1/tau, [1] = (i0 + j0) mod 2 of the crop origin.  Loss of a crop: one
 * red and one black weighted point update on the cells at least one cell inside, then 1/2 the
 * mean of r^2 = (f - (sum_X c_X u_X - S u))^2 over the cells at least two inside,
 * S = sum_X c_X + 1/tau.  Gradients by reverse mode in FP32; Adam (lr, 0.9, 0.999, 1e-8). */
typedef struct mg_trainer_s *mg_trainer;
/* capacity crops, batches of at most batch_max; theta0 host (NULL: He-normal hidden layers
 * from `seed`, zero output layer: omega = 1, the plain smoother). */
int mg_trainer_create(mg_trainer *out, int capacity, int batch_max, unsigned long long seed, const float *theta0);
/* Appends `count` crops of h's finest grid at seeded random origins (the current increment and
 * the last snapshot's coefficients and f); stops at capacity.  Waits. */
int mg_trainer_record(mg_trainer t, mg_handle h, int count);
/* Appends `count` crop records from host memory. */
int mg_trainer_load(mg_trainer t, const float *records, int count);
int mg_trainer_count(mg_trainer t);
/* The training loss: 0 (the default) the residual as above; 1 its high-frequency part, the
 * quantity a multigrid smoother is responsible for (the coarse grid corrects the smooth part):
 * v = 4 r - (the sum of r at the four neighbours), loss = 1/2 the mean of v^2 over the same cells
 * (the 5-point Laplacian of r, whose symbol vanishes on smooth modes and peaks on the
 * checkerboard mode).  Errors: MG_ERR_ARG. */
int mg_trainer_set_loss(mg_trainer t, int kind);
/* Mean loss and gradient over the crops idx[0..batch-1] (host) without a step. */
int mg_trainer_grad(mg_trainer t, const int *idx, int batch, float *grad, double *loss);
/* `iters` Adam steps on random batches; *loss gets the last batch's mean loss.  Waits. */
int mg_trainer_train(mg_trainer t, int iters, int batch, double lr, double *loss);
int mg_trainer_get(mg_trainer t, float *theta);
void mg_trainer_destroy(mg_trainer t);

/* Energy of the current level set (Sec. 2.2: eq. scfunc for Spencer-Chen, eq. rcfunc for
 * Rada-Chen; the diagnostic the paper reports after each cycle in Table 7), on the finest grid
 * in pixel units, with the current c1, c2:
 *   E = sum_ij [mu w delta_eps(phi) |grad phi|_beta + lambda1 (z - c1)^2 H + lambda2 (z - c2)^2 (1 - H)]
 *       + theta sum_ij d H                      (Spencer-Chen; w = g)
 *       + nu n m (sum_ij H / (n m) - A1 / (n m))^2   (Rada-Chen; w = d g)
 * with H = H_eps(phi) and central differences with mirror ghosts.  Sums are FP64.  *E (host)
 * receives it; waits for the handle's stream.  Errors: MG_ERR_ARG (NULL), MG_ERR_CUDA. */
int mg_energy(mg_handle h, double *E);

/* The bottom of the V-cycle in one block: with MG_F32 / MG_MIXED storage, the Spencer-Chen
 * model and the fused smoother, the grids from a first one down to the coarsest run as one
 * kernel of one 1024-thread block instead of one launch per grid and phase.  The first grid is
 * one whose whole sub-cycle (pn, u, w, F, rhs, G, f, u0, masks and the coarsest solve's scratch)
 * fits in 200 KB of shared memory: by default the first such grid with at most 1024 cells (one
 * per thread; larger grids run faster as per-grid launches), else the largest such grid;
 * mg_set_bottom_level and mg_autotune change it.  It performs the same operations per cell as
 * the per-grid kernels, so the results are identical.  enable = 1 (the default at set-up) or 0;
 * *first_level (may be NULL) gets the first grid it covers, -1 when it does not apply.  At
 * set-up the cluster bottom kernel (mg_set_cluster_level) is also chosen, from the largest grid
 * the one-block kernel can start at, when that grid has at most 16 tiles of 32 x 32 and such a
 * cluster fits the GPU; this call and mg_set_bottom_level switch the cluster off.
 * Errors: MG_ERR_ARG. */
int mg_set_bottom_kernel(mg_handle h, int enable, int *first_level);
/* Sets the first grid of the one-block bottom kernel (a tuning step of this implementation; the
 * paper has no counterpart): `level` from the largest grid whose sub-cycle fits the kernel's
 * shared memory (see mg_set_bottom_kernel) to levels - 2, or -1 for none.  A later start runs
 * more grids through the per-grid kernels; the results are the same either way.  mg_autotune
 * also chooses it (mg_stats.bottom_level).  Errors: MG_ERR_ARG (level out of that range, or the
 * bottom kernel does not apply). */
int mg_set_bottom_level(mg_handle h, int level);
/* Runs the bottom of the V-cycle from grid `level` as one thread-block cluster (a tuning step of
 * this implementation; the paper has no counterpart): one 1024-thread CTA per 32 x 32 tile of
 * that grid, neighbours exchanged through distributed shared memory, and CTA 0 running the
 * coarser grids like the one-block kernel.  `level` from the grid before the largest one the
 * one-block kernel can start at, to levels - 2, with at most 16 tiles; -1 switches it off (the
 * one-block kernel, if on, then takes over).  The results are the same either way.  mg_autotune
 * also chooses it (mg_stats.cluster_level).  Errors: MG_ERR_ARG (out of range, or no such cluster
 * fits the GPU). */
int mg_set_cluster_level(mg_handle h, int level);

/* Batches (many images at once; no counterpart in the paper): `count` images of
 * their own sizes solved together.  Each V-cycle of mg_batch_solve_step is one CUDA graph
 * launch whose branches are the images' V-cycles; a branch is a conditional graph node that
 * the device skips once that image's residual has reached the tolerance.
 *   images[i]   device, n[i]*m[i] floats (read during the call);  markers[i] host, k[i] pairs;
 *   params[i]   per-image parameters (MG_F32 or MG_MIXED), e.g. from mg_default_params;
 *   stream      may be NULL (own non-blocking stream).
 * Images' handles are owned by the batch: use mg_batch_handle(b, i) for mg_mask, mg_get_phi,
 * mg_get_stats of image i, never mg_destroy.  Errors as mg_setup. */
typedef struct mg_batch_s *mg_batch;
int mg_batch_setup(mg_batch *out, int count, const void *const *images, const int *n, const int *m,
                   const double *const *markers, const int *k, const mg_params *params, void *stream);
/* One pseudo-time step of every image (begin, V-cycles until every rho <= tol, end), with the
 * step control of mg_solve_step per image: an attempt that stalls, diverges or reaches max_cycles
 * V-cycles halts that image; when no image is left running, the halted ones restart together
 * from their phi^n with tau / 2 (at most params.max_halvings times each).  The results equal
 * those of mg_solve_step on each image alone.  cycles[i] / rho[i] (host, may be NULL) get each
 * image's V-cycles (all attempts) and final rho.  MG_ERR_TIMEOUT when an image did not reach
 * tol.  To solve new images of the same sizes, call mg_reset on mg_batch_handle(b, i). */
int mg_batch_solve_step(mg_batch b, double tol, int max_cycles, int *cycles, double *rho);
/* Tile shapes for the batch as a whole: runs mg_autotune on every image, then times `reps`
 * launches of the batch graph (every image running) with those per-image choices and with each
 * single tile shape on every grid of every image, and keeps the fastest.  The images' phi is
 * restored; results of later steps do not depend on the choice.  Waits. */
int mg_batch_autotune(mg_batch b, int reps);
mg_handle mg_batch_handle(mg_batch b, int i);
void mg_batch_destroy(mg_batch b);

/* Diagnostic timing of the smoother kernels on grid `level` at the current state: runs `reps`
 * outer smoothing iterations eagerly with CUDA events on the handle's stream and writes the
 * mean milliseconds per launch of [0] the snapshot kernel, [1..4] the sweeps A, B, C, D,
 * [5] the residual kernel to ms[0..5].  Changes phi like real smoothing does.  Waits. */
int mg_time_kernels(mg_handle h, int level, int reps, double *ms);

/* Times, on grid `level` inside a step, the residual kernels a V-cycle runs there, `reps` times
 * each (CUDA events on the handle's stream): mean milliseconds of [0] the residual norm
 * ||rhs - L(phi)|| (the per-tile kernel and the final FP64 sum; the norm goes to a scratch
 * slot, not to the step's norms) and [1] the residual with full weighting into grid level + 1
 * (Sec. 3.1: the coarse right-hand side's restriction and the restriction of u; -1 on the
 * coarsest grid) to ms[0..1].  Writes grid level + 1's right-hand side, u and u0 as a V-cycle
 * does.  MG_ERR_STATE outside a step, MG_ERR_ARG for a bad level or reps < 1.  Waits. */
int mg_time_residuals(mg_handle h, int level, int reps, double *ms);

/* Times the Hybrid Smoother 2 sweeps of grid `level` as a V-cycle's graph replays them: one
 * snapshot at the current state, then the sweeps A..D of `reps` outer iterations (1..256)
 * captured back to back in one CUDA graph (the snapshot's lagged coefficients and member masks
 * serve every sweep), launched once untimed and once between two CUDA events on the handle's
 * stream; ms[0] gets the mean milliseconds per sweep, the graph's kernel boundaries included.
 * Changes phi like real smoothing does.  MG_ERR_STATE outside a step; MG_ERR_ARG for a bad
 * level or reps, or another smoother.  Waits. */
int mg_time_sweeps_graph(mg_handle h, int level, int reps, double *ms);

/* Residual norm ||L(phi)||_2 of one grid function, with no device allocation.  The paper has no
 * counterpart: this serves callers that cannot allocate device memory when they need the norm,
 * such as code whose device memory is owned by a framework's pool or a running real-time loop
 * that may not call cudaMalloc (it synchronises the device).  It computes the same quantity as the
 * reference norm of mg_begin_step for a step starting at phi (zero increment, finest grid,
 * spacing 1, no FAS right-hand side), and agrees with it to about 1e-12 relative (the per-tile
 * partial sums may be added in another order):
 *   phi, w, F  device, n*m dense row-major arrays of float (MG_F32) or double (MG_F64): the level
 *              set, the length weight w and the fitting field F (mg_get_level fields 0, 1, 4);
 *   p          uses mu, beta, model and precision; only MG_MODEL_SC is accepted;
 *   norm       host, receives the FP64-accumulated norm;  stream may be NULL (default stream).
 * Its scratch is one file-scope device array sized for 65,536 tiles of 32 x 32 cells (for example
 * 8192 x 8192); larger grids, and grids of more than 65,535 tile rows, get MG_ERR_ARG before any
 * device access.  The array's device address is looked up on the first call made on each device
 * (with that device current) and kept for the life of the process; after cudaDeviceReset on a
 * device the kept address is no longer valid, and this entry point must not be called on that
 * device again.  Every call shares the array: calls
 * that overlap on the GPU race on it.  The call waits for its stream.  Errors: MG_ERR_ARG,
 * MG_ERR_CUDA (mg_last_error is not updated). */
int mg_residual_norm_noalloc(const void *phi, const void *w, const void *F, int n, int m,
                             const mg_params *p, double *norm, void *stream);

/* The CUDA stream (cudaStream_t) the handle enqueues its work on: the caller's stream given
 * to mg_setup, or the library's own non-blocking stream when that was NULL. */
void *mg_get_stream(mg_handle h);

/* Releases the handle and its device memory (after waiting for its stream). */
void mg_destroy(mg_handle h);

const char *mg_strerror(int code);
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
