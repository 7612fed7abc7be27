// host.cu -- driver of the FAS V-cycle and the C ABI declared in include/segmg.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <mutex>
#include <random>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/segmg.h"
#include "internal.h"

namespace segmg {
void prepare_smoother_kernels();

// Readers of the MG_DEBUG error words, one per translation unit (registered at load time).
using DebugReader = int (*)(unsigned long long *, int);
static std::vector<DebugReader> &debug_readers() {
    static std::vector<DebugReader> v;
    return v;
}
int register_debug_reader(int (*read)(unsigned long long *words, int clear)) {
    debug_readers().push_back(read);
    return (int)debug_readers().size();
}
}

namespace {

using namespace segmg;

thread_local std::string g_err;

// NVTX range for profilers (no cost without one).  The ranges mark host-side work: per level in
// eager mode (use_graph = 0); with graphs, the V-cycle range encloses the graph launch.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// Per-V-cycle log of the step control (JSON lines appended to the file named by the SEGMG_LOG
// environment variable; nothing when it is unset).
void log_cycle(int step, int attempt, int cycle, double rho, double tau, double ms) {
    static const char *path = std::getenv("SEGMG_LOG");
    if (!path || !*path) return;
    if (FILE *f = std::fopen(path, "a")) {
        std::fprintf(f, "{\"step\": %d, \"attempt\": %d, \"cycle\": %d, \"rho\": %.17g, \"tau\": %.17g, \"ms\": %.4f}\n",
                     step, attempt, cycle, rho, tau, ms);
        std::fclose(f);
    }
}

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? MG_ERR_NOMEM : MG_ERR_CUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                       \
    } while (0)

#define CKL()                                                                                      \
    do {                                                                                           \
        cudaError_t e_ = cudaGetLastError();                                                       \
        if (e_ != cudaSuccess) return fail(MG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
    } while (0)

// The end of one V-cycle of the device step loop: rho of the V-cycle (the same FP64 expression
// as the host's), the step control's tests in the host's order, and the loop condition.
__global__ void k_step_loop(cudaGraphConditionalHandle h, Scalars *sc, double tol, int max_cycles,
                            double stall_ratio) {
    const int j = sc->loop_j + 1;
    sc->loop_j = j;
    const double res0 = sqrt(sc->norm2_0);
    const double rho = res0 > 0 ? sqrt(sc->norm2) / res0 : sqrt(sc->norm2);
    sc->loop_rho[j] = rho;
    int stop = 0;
    if (sc->err != 0) stop = 5;
    else if (!isfinite(rho) || rho > 1e3) stop = 4;
    else if (rho <= tol) stop = 1;
    else if (stall_ratio > 0 && j >= 4 && rho > stall_ratio * sc->loop_rho[j - 2]) stop = 2;
    else if (j >= max_cycles) stop = 3;
    sc->loop_stop = stop;
    cudaGraphSetConditional(h, stop == 0 ? 1u : 0u);
}

template <typename T>
__global__ void k_phi_out(const T *pn, const T *u, int n, int m, int p, T *out) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i < n && j < m) out[(size_t)i * m + j] = pn[(size_t)i * p + j] + u[(size_t)i * p + j];
}

template <typename T>
__global__ void k_phi_in(const T *in, int n, int m, int p, T *pn, T *u) {
    const int j = blockIdx.x * 32 + threadIdx.x, i = blockIdx.y * 8 + threadIdx.y;
    if (i < n && j < m) {
        pn[(size_t)i * p + j] = in[(size_t)i * m + j];
        u[(size_t)i * p + j] = T(0);
    }
}

// Convex hull of 2-D points (monotone chain), counter-clockwise in (x, y); returns the hull
// vertex list (x0, y0, x1, y1, ...).
std::vector<double> hull_of(const double *xy, int k) {
    std::vector<std::pair<double, double>> pts(k);
    for (int q = 0; q < k; ++q) pts[q] = {xy[2 * q], xy[2 * q + 1]};
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    auto cross = [](const std::pair<double, double> &o, const std::pair<double, double> &a,
                    const std::pair<double, double> &b) {
        return (a.first - o.first) * (b.second - o.second) - (a.second - o.second) * (b.first - o.first);
    };
    std::vector<std::pair<double, double>> h(2 * pts.size() + 2);
    int c = 0;
    for (size_t q = 0; q < pts.size(); ++q) {
        while (c >= 2 && cross(h[c - 2], h[c - 1], pts[q]) <= 0) --c;
        h[c++] = pts[q];
    }
    for (int q = (int)pts.size() - 2, lo = c + 1; q >= 0; --q) {
        while (c >= lo && cross(h[c - 2], h[c - 1], pts[q]) <= 0) --c;
        h[c++] = pts[q];
    }
    if (c > 1) --c;
    std::vector<double> out;
    for (int q = 0; q < c; ++q) { out.push_back(h[q].first); out.push_back(h[q].second); }
    return out;
}

struct SolverBase {
    virtual ~SolverBase() {}
    virtual int reset(const void *image, const double *mk, int k) = 0;
    virtual int begin_step(double *res0) = 0;
    // begin_step without its host round trip; finish_begin (after the attempt) reads the norm
    virtual int begin_step_deferred() = 0;
    virtual int finish_begin() = 0;
    virtual int vcycle(double *rho) = 0;
    virtual int end_step(double *eta) = 0;
    virtual int mask(unsigned char *out) = 0;
    virtual int mask_async(unsigned char *out) = 0;   // enqueued only (the caller synchronises)
    virtual int get_phi(void *out) = 0;
    virtual int set_phi(const void *in) = 0;
    virtual int set_regions(double c1, double c2) = 0;
    virtual int get_level(int l, int field, void *out) = 0;
    virtual int stats(mg_stats *s) = 0;
    // host-side values that need no device read (stats() copies the device scalars and waits)
    virtual int rows() const = 0;
    virtual int cols() const = 0;
    virtual int steps_done() const = 0;
    virtual double last_eta() const = 0;
    virtual cudaStream_t stream() const = 0;
    virtual int time_kernels(int level, int reps, double *ms) = 0;
    virtual int time_residuals(int level, int reps, double *ms) = 0;
    virtual int time_sweeps_graph(int level, int reps, double *ms) = 0;
    virtual int autotune(int reps, int *out) = 0;
    virtual int set_shapes(const int *shapes) = 0;
    virtual int set_bottom(int enable) = 0;
    virtual int set_bottom_level(int level) = 0;
    virtual int set_cluster_level(int level) = 0;
    virtual int energy(double *E) = 0;
    virtual int aos(double dt, int max_iter, double eta, int *iters, double *rho) = 0;
    virtual int set_learned(const float *theta, int mode, int refresh) = 0;
    virtual int set_omega(int l, const void *w) = 0;
    virtual int record_crops(float *data, int first, int count, unsigned long long seed) = 0;
    // pseudo-time step control (mg_solve_step): the parameters, a restart of the current step
    // from phi^n with a new tau, and the bookkeeping of the step's V-cycles
    virtual const mg_params &params() const = 0;
    virtual int restart_step(double tau) = 0;
    virtual void set_cycles_step(int c) = 0;
    virtual int set_wait_limit(long long rounds) = 0;
    virtual int inject_divergence(int cycle) = 0;
    // one attempt's V-cycles in one graph launch (the device step loop); MG_ERR_STATE when it
    // does not apply (the caller then runs V-cycles one by one)
    virtual int loop_attempt(double tol, int max_cycles, std::vector<double> &hist, int &stop) = 0;
};

template <typename T>
struct Level {
    int n = 0, m = 0, pitch = 0;
    double h = 1;
    T *pn = nullptr, *u = nullptr, *u0 = nullptr, *rhs = nullptr, *w = nullptr, *z = nullptr, *d = nullptr;
    T *F = nullptr, *G = nullptr, *f = nullptr, *r = nullptr, *upre = nullptr, *t = nullptr;
    uint32_t *mrow = nullptr, *mcol = nullptr;
    __nv_bfloat16 *wb = nullptr;   // mixed precision only
    uint8_t *cls = nullptr;        // Hybrid Smoother 1 only
    SweepMaps maps[kTileShapes];   // FP32 storage: tensor maps of the TMA sweep, per tile shape
    SnapMaps smaps;                // FP32 storage: tensor maps of the TMA snapshot
    ResMaps rmaps;                 // FP32 storage: tensor maps of the TMA residual kernels
};

template <typename T>
struct Solver final : SolverBase {
    mg_params p{};
    int n = 0, m = 0, nlev = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    mg_allocator al{};
    bool use_al = false;
    void *pool = nullptr;
    size_t pool_bytes = 0;
    Level<T> lv[kMaxLevels];
    Scalars *dsc = nullptr;
    Scalars *hsc = nullptr;   // pinned host mirror
    double *partials = nullptr;
    int npart = 0;
    double *coarse = nullptr;
    double *dmk = nullptr;    // markers (2 * kcap)
    double *dhull = nullptr;  // hull (2 * kcap + 4)
    double *hstage = nullptr; // pinned host staging of markers, hull, A1 / (n m) and the eta sums (6 kcap + 11)
    int kcap = 0;
    double A1 = 0, res0 = 0, rho = 0;
    bool res0_pending = false;   // a step begun without waiting: res0 not read yet
    bool res0_in_hsc = false;    // ... and the host mirror holds it (an attempt's graph copied it)
    // eta of the last step: end_step enqueues the copy of its two sums to the staging buffer and
    // the first reader waits for the stream (a step needs no host round trip for it)
    mutable double eta = 0;
    mutable bool eta_pending = false;
    int steps = 0, cycles_step = 0, cycles_total = 0;
    int rejected = 0;             // step attempts rejected by the step control
    double tau0 = 1.0;            // tau of the parameters (the step control halves p.tau)
    long long graph_epoch = 0;    // counts drop_graphs(): a batch rebuilds its graph when it changed
    long long wait_limit = kDefaultWaitLimit;   // try_wait rounds of the TMA sweep's bounded waits
    int inject_cycle = 0;         // mg_inject_divergence: V-cycle (of a step attempt) that reports
                                  // a diverged residual once; 0 = none
    bool in_step = false;
    cudaGraphExec_t gexec = nullptr;
    long long launches = 0, graph_nodes = 0;
    int shape[kMaxLevels] = {};   // fused-sweep tile shape per grid (mg_autotune)
    int lb = -1;                  // first grid of the one-block bottom kernel (-1: not used)
    int lb_first = -1;            // the largest grid it can start at (-1: it does not apply)
    int fas_level = -1;           // the grid whose next snapshot completes its FAS right-hand side
    int interp_level = -1;        // the grid whose next snapshot first applies the coarse correction
    int lc = -1;                  // first grid of the cluster bottom kernel (-1: not used); it runs
                                  // grids lc .. nlev-1 (lb is then unused)
    int lc_tiles = 0;
    size_t lc_smem = 0;
    // learned relaxation weights of the point updates (learned.cu)
    int learn_mode = 0;           // 0 off; 1 per V-cycle acceptance; 2 always; 3 fixed weights
    int learn_refresh = 4;        // V-cycles between inferences
    int learn_since = 0;          // V-cycles since the last inference
    bool use_omega = false;       // view() hands out the weight grids
    bool infer_pending[kMaxLevels] = {};
    __nv_bfloat16 *net = nullptr; // BF16 parameters
    T *omega_buf[kMaxLevels] = {};
    bool omega_valid[kMaxLevels] = {};   // the grid's weights are set (fixed) or inferred
    T *ubak = nullptr;            // finest-grid increment saved before a learned V-cycle (and
                                  // while mg_autotune times V-cycles)
    cudaGraphExec_t gexec_l = nullptr, gexec_li = nullptr;   // learned V-cycle; with inference
    cudaGraphExec_t gloop = nullptr;   // device step loop (while node around the V-cycle)
    double gloop_tol = -1.0;
    int gloop_max = -1;
    long long gloop_nodes = 0;
    // the fused form of the loop (FP32 storage): the finest grid's first snapshot of each V-cycle
    // also computes the norm of the state the previous V-cycle left, run at the end of the
    // previous loop iteration, before its step-control tests; gloop_first: kernels of that part
    bool gloop_fused = false;
    long long gloop_first = 0;
    int skip_first_snapshot = 0;   // capture of the rest of a V-cycle: the first smoothing of the
                                   // finest grid starts after its snapshot
    long long nodes_l = 0, nodes_li = 0;
    double plain_rate = -1.0;     // contraction of the last plain V-cycle of the step
    int learn_skip = 0, learn_backoff = 1;   // plain V-cycles left before the next learned try
    long long learned_acc = 0, learned_rej = 0;
    size_t lb_smem = 0;
    ModelParams mp{};

    ~Solver() override { release(); }

    void drop_graphs() {
        ++graph_epoch;
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gexec_l) cudaGraphExecDestroy(gexec_l);
        if (gexec_li) cudaGraphExecDestroy(gexec_li);
        if (gloop) cudaGraphExecDestroy(gloop);
        gexec = gexec_l = gexec_li = gloop = nullptr;
    }

    void release() {
        if (st) cudaStreamSynchronize(st);
        drop_graphs();
        for (auto &b : omega_buf) { if (b) cudaFree(b); b = nullptr; }
        if (ubak) cudaFree(ubak);
        if (net) cudaFree(net);
        ubak = nullptr;
        net = nullptr;
        if (pool) {
            if (use_al) al.free(pool, pool_bytes, st, al.ctx);
            else cudaFreeAsync(pool, st);
            if (st) cudaStreamSynchronize(st);
        }
        pool = nullptr;
        if (hsc) cudaFreeHost(hsc);
        hsc = nullptr;
        if (hstage) cudaFreeHost(hstage);
        hstage = nullptr;
        if (own_stream && st) cudaStreamDestroy(st);
        st = nullptr;
    }

    cudaStream_t stream() const override { return st; }

    LevelView<T> view(int l) const {
        const Level<T> &L = lv[l];
        LevelView<T> v;
        v.n = L.n; v.m = L.m; v.pitch = L.pitch; v.level = l;
        v.cdiff = (T)(p.mu / (L.h * L.h));
        v.inv_tau = (T)(p.tau > 0 ? 1.0 / p.tau : 0.0);
        v.Sigma = (T)p.Sigma;
        v.inv_2h = (T)(1.0 / (2.0 * L.h));
        v.beta = (T)p.beta;
        v.pn = L.pn; v.u = L.u; v.u0 = L.u0; v.rhs = L.rhs; v.w = L.w; v.z = L.z; v.d = L.d;
        v.F = L.F; v.G = L.G; v.f = L.f; v.r = L.r; v.upre = L.upre; v.t = L.t;
        v.mrow = L.mrow; v.mcol = L.mcol; v.npm = (L.m + 31) / 32; v.npn = (L.n + 31) / 32;
        v.wb = L.wb;
        v.cls = L.cls;
        v.omega = use_omega && omega_valid[l] ? omega_buf[l] : nullptr;
        v.has_rhs = l > 0 ? 1 : 0;
        return v;
    }

    double h2nm(int l) const { return lv[l].h * lv[l].h / ((double)n * m); }

    int init(int n_, int m_, const mg_params &p_, const mg_allocator *a, cudaStream_t s, int k) {
        p = p_; n = n_; m = m_; nlev = p.levels;
        tau0 = p.tau;
        mp = ModelParams{p.model, p.mu, p.lambda1, p.lambda2, p.theta, p.nu, p.eps, p.beta};
        if (s) st = s;
        else { CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own_stream = true; }
        if (a && a->alloc && a->free) { al = *a; use_al = true; }
        // layout
        size_t off = 0;
        auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
        std::vector<std::pair<void **, size_t>> plan;
        int nn = n, mm = m;
        for (int l = 0; l < nlev; ++l) {
            Level<T> &L = lv[l];
            L.n = nn; L.m = mm; L.pitch = (mm + 31) / 32 * 32; L.h = std::ldexp(1.0, l);
            size_t fb = (size_t)L.n * L.pitch * sizeof(T);
            T **fields[] = {&L.pn, &L.u, &L.w, &L.z, &L.d, &L.F, &L.G, &L.f, &L.r, &L.t};
            for (T **f : fields) plan.push_back({(void **)f, take(fb)});
            if (l > 0) {
                plan.push_back({(void **)&L.u0, take(fb)});
                plan.push_back({(void **)&L.rhs, take(fb)});
            }
            if (p.smoother == MG_SMOOTH_PHASED) plan.push_back({(void **)&L.upre, take(fb)});
            if (p.precision == MG_MIXED) plan.push_back({(void **)&L.wb, take((size_t)L.n * L.pitch * 2)});
            if (p.smoother == MG_SMOOTH_HS1) plan.push_back({(void **)&L.cls, take((size_t)L.n * L.pitch)});
            plan.push_back({(void **)&L.mrow, take(sizeof(uint32_t) * 2 * (size_t)L.n * ((L.m + 31) / 32))});
            plan.push_back({(void **)&L.mcol, take(sizeof(uint32_t) * 2 * (size_t)L.m * ((L.n + 31) / 32))});
            nn /= 2; mm /= 2;
        }
        npart = num_partials(n, m);
        kcap = std::max(k, 16);
        size_t o_sc = take(sizeof(Scalars));
        size_t o_part = take(sizeof(double) * 8 * (size_t)npart);
        size_t o_coarse = take(sizeof(double) * coarse_scratch_elems(lv[nlev - 1].n, lv[nlev - 1].m));
        size_t o_mk = take(sizeof(double) * 2 * kcap);
        size_t o_hull = take(sizeof(double) * (4 * kcap + 8));
        pool_bytes = off;
        if (use_al) {
            pool = al.alloc(pool_bytes, st, al.ctx);
            if (!pool) return fail(MG_ERR_NOMEM, "allocator returned NULL");
        } else {
            CK(cudaMallocAsync(&pool, pool_bytes, st));
        }
        CK(cudaMemsetAsync(pool, 0, pool_bytes, st));
        char *base = (char *)pool;
        for (auto &pr : plan) *pr.first = base + pr.second;
        dsc = (Scalars *)(base + o_sc);
        partials = (double *)(base + o_part);
        coarse = (double *)(base + o_coarse);
        dmk = (double *)(base + o_mk);
        dhull = (double *)(base + o_hull);
        CK(cudaMallocHost(&hsc, sizeof(Scalars)));
        CK(cudaMallocHost(&hstage, sizeof(double) * (6 * (size_t)kcap + 11)));
        if constexpr (std::is_same<T, float>::value) {
            if (p.smoother == MG_SMOOTH_FUSED)
                for (int l = 0; l < nlev; ++l)
                    for (int sh = 0; sh < kTileShapes; ++sh)
                        if (!encode_sweep_maps(view(l), sh, &lv[l].maps[sh]))
                            return fail(MG_ERR_CUDA, "cuTensorMapEncodeTiled failed for a grid");
            for (int l = 0; l < nlev; ++l)
                if (!encode_snapshot_maps(view(l), &lv[l].smaps) || !encode_residual_maps(view(l), &lv[l].rmaps))
                    return fail(MG_ERR_CUDA, "cuTensorMapEncodeTiled failed for a grid (snapshot, residual)");
        }
        // default tile shapes (what mg_autotune chooses on grids up to 1024^2): 32 x 32 tiles (256
        // threads on the finest grid, 512 below) where they all fit one wave of 8 blocks per SM;
        // 32 x 64 tiles on larger grids, where the smaller halo share counts
        {
            int dev = 0, sms = 1;
            if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            for (int l = 0; l < nlev - 1; ++l) {
                const long tiles = (long)((lv[l].n + 31) / 32) * ((lv[l].m + 31) / 32);
                shape[l] = tiles <= 8L * std::max(sms, 1) ? (l == 0 ? 4 : 5) : 0;
            }
        }
        set_bottom(1);
        default_cluster();
        return MG_OK;
    }

    // By default the bottom of the V-cycle runs on a thread-block cluster from the largest grid the
    // bottom kernel takes (lb_first), when that grid has at most kClusterMaxTiles tiles and such a
    // cluster fits; the one-block kernel otherwise.  (On the 1024^2 bench the autotuner's choice
    // too: 64^2 on four CTAs, 0.25 ms per step less than the one-block kernel from 32^2.)
    void default_cluster() {
        if (lb_first < 0) return;
        const int l = lb_first;
        const int tiles = ((lv[l].n + 31) / 32) * ((lv[l].m + 31) / 32);
        if (tiles > kClusterMaxTiles) return;
        int ns[kMaxLevels], ms[kMaxLevels];
        for (int k = 0; k < nlev; ++k) { ns[k] = lv[k].n; ms[k] = lv[k].m; }
        const size_t bytes = cluster_smem_bytes(bottom_smem_bytes(ns, ms, l + 1, nlev, p.precision == MG_MIXED));
        if (cluster_fits(tiles, bytes) < 1) return;
        lc = l;   // the one-block kernel's start (lb) stays: it takes over if the cluster is switched off
        lc_tiles = tiles;
        lc_smem = bytes;
    }

    // The bottom kernel runs grids lb .. nlev-1 in one block when the storage is FP32 (or mixed),
    // the model is Spencer-Chen, the fused smoother is selected and at least two grids fit in
    // its shared memory (lb_first: the largest grid that fits).  By default it starts at the
    // first of those grids with at most one cell per thread (the block's fast path; larger grids
    // run faster as per-grid launches), or at lb_first when there is none.
    int set_bottom(int enable) override {
        lb = lb_first = -1;
        lb_smem = 0;
        lc = -1;   // an explicit choice of the one-block bottom (or none) replaces the cluster
        if (sizeof(T) == 4 && p.model == MG_MODEL_SC && fused()) {
            int ns[kMaxLevels], ms[kMaxLevels];
            for (int l = 0; l < nlev; ++l) { ns[l] = lv[l].n; ms[l] = lv[l].m; }
            for (int l = nlev - 2; l >= 0; --l) {
                size_t b = bottom_smem_bytes(ns, ms, l, nlev, p.precision == MG_MIXED);
                if (b > kBottomSmemMax) break;
                lb_first = l;
            }
        }
        if (enable && lb_first >= 0) {
            int l = lb_first;
            while (l < nlev - 2 && lv[l].n * lv[l].m > kBottomThreads) ++l;
            use_bottom_from(lv[l].n * lv[l].m <= kBottomThreads ? l : lb_first);
        }
        drop_graphs();
        return lb;
    }

    void use_bottom_from(int l) {
        int ns[kMaxLevels], ms[kMaxLevels];
        for (int k = 0; k < nlev; ++k) { ns[k] = lv[k].n; ms[k] = lv[k].m; }
        lb = l;
        lb_smem = l >= 0 ? bottom_smem_bytes(ns, ms, l, nlev, p.precision == MG_MIXED) : 0;
    }

    // The cluster bottom kernel from grid `level`: grids level+1 .. nlev-1 must fit the one-block
    // kernel's shared memory beside the tile, and grid `level` must have at most
    // kClusterMaxTiles tiles of 32 x 32.
    int set_cluster_level(int level) override {
        if (level == -1) {
            lc = -1;
            drop_graphs();
            return MG_OK;
        }
        if (lb_first < 0 || level < lb_first - 1 || level > nlev - 2)
            return fail(MG_ERR_ARG, "cluster level out of range (or the bottom kernel does not apply)");
        int ns[kMaxLevels], ms[kMaxLevels];
        for (int k = 0; k < nlev; ++k) { ns[k] = lv[k].n; ms[k] = lv[k].m; }
        const int tiles = ((lv[level].n + 31) / 32) * ((lv[level].m + 31) / 32);
        const size_t bytes = cluster_smem_bytes(bottom_smem_bytes(ns, ms, level + 1, nlev, p.precision == MG_MIXED));
        const int fits = cluster_fits(tiles, bytes);
        if (fits < 1)
            return fail(MG_ERR_ARG, "the grid does not fit one thread-block cluster (" + std::to_string(tiles) +
                                        " CTAs, " + std::to_string(bytes) + " bytes of shared memory each: " +
                                        std::to_string(fits) + ")");
        lc = level;
        lc_tiles = tiles;
        lc_smem = bytes;
        drop_graphs();
        return MG_OK;
    }

    int set_bottom_level(int level) override {
        if (level != -1 && (lb_first < 0 || level < lb_first || level > nlev - 2))
            return fail(MG_ERR_ARG, "bottom level out of range (or the bottom kernel does not apply)");
        lc = -1;
        use_bottom_from(level);
        drop_graphs();
        return MG_OK;
    }

    int aos(double dt, int max_iter, double eta_stop, int *iters, double *rhoout) override {
        if (!in_step) return fail(MG_ERR_STATE, "mg_aos outside a step");
        if (!(dt > 0) || max_iter < 1) return fail(MG_ERR_ARG, "dt <= 0 or max_iter < 1");
        drop_graphs();
        int it = 0;
        while (it < max_iter) {
            area_term(0, lv[0].u);
            snapshot(0, view(0));
            launch_aos_iteration<T>(view(0), area_ptr(), dt, partials, dsc->aos, st);
            launches += area_launches() + 4;
            ++it;
            CKL();
            double s2[2];
            CK(cudaMemcpyAsync(s2, dsc->aos, sizeof(s2), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (!std::isfinite(s2[0])) return fail(MG_ERR_NAN, "non-finite AOS iterate");
            if (std::sqrt(s2[0]) <= eta_stop * std::sqrt(s2[1])) break;
        }
        area_term(0, lv[0].u);
        norm_residual(&dsc->norm2);
        launches += area_launches() + norm_launches();
        CK(cudaMemcpyAsync(hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        rho = res0 > 0 ? std::sqrt(hsc->norm2) / res0 : std::sqrt(hsc->norm2);
        if (iters) *iters = it;
        if (rhoout) *rhoout = rho;
        return MG_OK;
    }

    int energy(double *E) override {
        launch_energy<T>(view(0), mp, partials, npart, dsc, &dsc->sums[7], st);
        launches += 2;
        CKL();
        CK(cudaMemcpyAsync(E, &dsc->sums[7], sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        return MG_OK;
    }

    void launch_bottom_cycle(bool cluster = false) {
        if constexpr (std::is_same<T, float>::value) {
            const int first = cluster ? lc : lb;
            BottomArgs a{};
            a.lb = first; a.L = nlev; a.nu1 = p.nu1; a.nu2 = p.nu2;
            a.coarse_fp64 = p.precision == MG_MIXED;
            a.coarse_aos = p.coarse_solver == MG_COARSE_AOS;
            a.aos_dt = p.aos_dt;
            for (int l = first; l < nlev; ++l) a.g[l] = view(l);
            a.mp = mp;
            a.A1frac = A1 / ((double)n * m);
            a.h2nm_coarse = h2nm(nlev - 1);
            a.coarse_tol = p.coarse_tol;
            a.coarse_maxit = p.coarse_maxit;
            a.sc = dsc;
            if (cluster) launch_cluster(a, lc_tiles, lc_smem, st);
            else launch_bottom(a, lb_smem, st);
        }
    }

    int reset(const void *image, const double *mk, int k) override {
        if (k > kcap) return fail(MG_ERR_ARG, "more markers than at set-up");
        // the kernels read the initial contour's area from the device scalars, so the captured
        // graphs stay valid; only a tau changed by the step control is restored (and they go)
        if (p.tau != tau0) {
            p.tau = tau0;
            drop_graphs();
        }
        in_step = false;
        rejected = 0;
        steps = cycles_step = cycles_total = 0;
        rho = eta = res0 = 0;
        eta_pending = res0_pending = res0_in_hsc = false;
        Level<T> &L0 = lv[0];
        CK(cudaMemsetAsync(dsc, 0, sizeof(Scalars), st));
        // the image's finiteness is checked while it is copied in and read back at the end of
        // the set-up (no value of the image decides an index, so a NaN only spoils values)
        launch_copy_in<T>((const T *)image, L0.z, n, m, L0.pitch, &dsc->err, st);
        // blur taps (Sec. 2.2 edge detector applied to the smoothed image)
        int R = std::min(16, (int)std::ceil(3.0 * p.sigma_blur));
        std::vector<double> taps(2 * R + 1);
        double s = 0;
        for (int t = -R; t <= R; ++t) { taps[t + R] = std::exp(-(double)t * t / (2 * p.sigma_blur * p.sigma_blur)); s += taps[t + R]; }
        for (double &t : taps) t /= s;
        launch_blur<T>(L0.z, L0.G, L0.f, n, m, L0.pitch, L0.pitch, taps.data(), R, st);
        // markers, hull and the initial area go through pinned staging (asynchronous copies)
        double *smk = hstage, *shull = hstage + 2 * kcap, *sA1 = hstage + 6 * kcap + 8;
        std::memcpy(smk, mk, sizeof(double) * 2 * k);
        CK(cudaMemcpyAsync(dmk, smk, sizeof(double) * 2 * k, cudaMemcpyHostToDevice, st));
        launch_edge_distance<T>(L0.f, L0.w, L0.d, n, m, L0.pitch, p.beta_edge, dmk, k, p.sigma_d, p.model, st);
        for (int l = 1; l < nlev; ++l) {
            Level<T> &Pf = lv[l - 1], &Lc = lv[l];
            RestrictFields<T> F{};
            F.f[0] = Pf.w; F.c[0] = Lc.w;
            F.f[1] = Pf.z; F.c[1] = Lc.z;
            F.f[2] = Pf.d; F.c[2] = Lc.d;
            F.nf = 3;
            launch_restrict_fields<T>(F, Pf.n, Pf.m, Pf.pitch, Lc.pitch, st);
        }
        if (p.precision == MG_MIXED)   // w in BF16 on every grid (restricted in FP32 first)
            for (int l = 0; l < nlev; ++l)
                launch_to_bf16((const float *)lv[l].w, lv[l].wb, lv[l].n, lv[l].m, lv[l].pitch, st);
        // initial level set: convex hull of the markers (Sec. 5)
        std::vector<double> hull = k >= 3 ? hull_of(mk, k) : std::vector<double>();
        int nh = (int)hull.size() / 2;
        double area = 0;
        for (int q = 0; q < nh; ++q) {
            int r = (q + 1) % nh;
            area += hull[2 * q] * hull[2 * r + 1] - hull[2 * r] * hull[2 * q + 1];
        }
        area *= 0.5;
        double cx = 0, cy = 0, r0 = 0.05 * std::max(n, m);
        if (nh < 3 || !(area > 0)) {
            nh = 0;
            for (int q = 0; q < k; ++q) { cx += mk[2 * q]; cy += mk[2 * q + 1]; }
            cx /= k; cy /= k;
            area = M_PI * r0 * r0;
        } else {
            std::memcpy(shull, hull.data(), sizeof(double) * hull.size());
            CK(cudaMemcpyAsync(dhull, shull, sizeof(double) * hull.size(), cudaMemcpyHostToDevice, st));
        }
        A1 = area;
        launch_initial_phi<T>(L0.pn, L0.u, n, m, L0.pitch, dhull, nh, cx, cy, r0, st);
        *sA1 = area / ((double)n * m);
        CK(cudaMemcpyAsync(&dsc->A1frac, sA1, sizeof(double), cudaMemcpyHostToDevice, st));
        launch_region_sums<T>(view(0), p.eps, partials, npart, dsc, 1, st);
        // copy-in, two blur passes, edge / distance, initial phi, region sums (2), restrictions
        launches += 5 + norm_launches() + (nlev - 1) + (p.precision == MG_MIXED ? nlev : 0);
        CKL();
        CK(cudaMemcpyAsync(hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));   // the staging buffer is free again; the image's check
        if (hsc->err & 2) {
            CK(cudaMemsetAsync(&dsc->err, 0, sizeof(int), st));
            return fail(MG_ERR_NAN, "image has NaN or Inf values");
        }
        return MG_OK;
    }

    int area_term(int l, const T *uin) {
        if (p.model != MG_MODEL_RC) return MG_OK;
        launch_area<T>(view(l), uin, p.eps, p.nu, h2nm(l), partials, num_partials(lv[l].n, lv[l].m),
                       &dsc->area[l], dsc, st);
        return MG_OK;
    }

    const double *area_ptr() const { return p.model == MG_MODEL_RC ? dsc->area : nullptr; }

    int begin_step(double *r0out) override { return begin_step_impl(r0out, true); }
    int begin_step_deferred() override { return begin_step_impl(nullptr, false); }

    // The reference norm of a step begun by begin_step_deferred: read from the scalars that the
    // attempt's graph launch copied back, else copied and waited for here.
    int finish_begin() override {
        if (!res0_pending) return MG_OK;
        if (!res0_in_hsc) {
            CK(cudaMemcpyAsync(hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
        }
        res0 = std::sqrt(hsc->norm2_0);
        res0_pending = res0_in_hsc = false;
        if (!std::isfinite(res0)) {
            in_step = false;
            return fail(MG_ERR_NAN, "non-finite initial residual");
        }
        return MG_OK;
    }

    // wait = false: everything is enqueued and the reference norm is read later (finish_begin),
    // so a step's first host round trip is the one after its V-cycles
    int begin_step_impl(double *r0out, bool wait) {
        Range range("begin step");
        launch_fold<T>(view(0), st);
        for (int l = 1; l < nlev; ++l) {
            Level<T> &Pf = lv[l - 1], &Lc = lv[l];
            launch_restrict<T>(Pf.pn, Pf.n, Pf.m, Pf.pitch, Lc.pn, nullptr, Lc.pitch, st);
        }
        LevelView<T> views[kMaxLevels];
        for (int l = 0; l < nlev; ++l) views[l] = view(l);
        launch_fitting<T>(views, nlev, dsc, mp, st);
        area_term(0, lv[0].u);
        norm_residual(&dsc->norm2_0);
        launches += 1 + (nlev - 1) + 1 + area_launches() + norm_launches();   // fold, restrictions, fitting, norm
        CKL();
        if (wait) {
            CK(cudaMemcpyAsync(hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            res0 = std::sqrt(hsc->norm2_0);
        }
        rho = 1.0;
        plain_rate = -1.0;
        learn_since = 0;
        learn_skip = 0;
        learn_backoff = 1;
        // the last residual norm starts at the reference one (rho = 1 until a V-cycle runs)
        CK(cudaMemcpyAsync(&dsc->norm2, &dsc->norm2_0, sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(&dsc->halt, 0, sizeof(int), st));
        if (wait && !std::isfinite(res0)) return fail(MG_ERR_NAN, "non-finite initial residual");
        in_step = true;
        cycles_step = 0;
        res0_pending = !wait;
        res0_in_hsc = false;
        if (r0out) *r0out = res0;
        return MG_OK;
    }

    // kernels per call of each enqueue helper (for the launch counter)
    // (a chunked FP64 sum adds a launch above 1024 partials)
    int sum_launches(int l) const { return num_partials(lv[l].n, lv[l].m) > 1024 ? 2 : 1; }
    int area_launches(int l = 0) const { return p.model == MG_MODEL_RC ? 1 + sum_launches(l) : 0; }
    int norm_launches(int l = 0) const { return 1 + sum_launches(l); }
    bool fused() const { return p.smoother == MG_SMOOTH_FUSED || p.smoother == MG_SMOOTH_FUSED_VEC; }
    // kernels of one outer smoothing iteration after the snapshot on grid l
    int smoother_launches(int l) const {
        if (p.smoother == MG_SMOOTH_PHASED) return 16;
        if (fused()) return 4;
        int k = 0;
        for (int par = 0; par < 2; ++par) k += (lv[l].m - par + 1) / 2 > 0;
        if (p.smoother == MG_SMOOTH_HS1)
            for (int c = 0; c < 16; ++c) k += (lv[l].n - c / 4 + 3) / 4 > 0 && (lv[l].m - c % 4 + 3) / 4 > 0;
        return k;
    }

    // sum r^2 of the finest residual r = -L(phi) into *norm_out (r itself is not kept for FP32
    // storage)
    void norm_residual(double *norm_out) {
        if constexpr (std::is_same<T, float>::value)
            launch_residual_tma(view(0), 0, area_ptr(), nullptr, 0, partials, npart, norm_out, lv[0].smaps,
                                lv[0].rmaps, &dsc->err, wait_limit, st);
        else launch_residual<T>(view(0), lv[0].u, area_ptr(), lv[0].r, 0, partials, npart, norm_out, st);
    }

    // The coefficient snapshot of grid l (v = view(l)): TMA-staged for FP32 storage.
    void snapshot(int l, const LevelView<T> &v) {
        if constexpr (std::is_same<T, float>::value)
            launch_snapshot_tma(v, area_ptr(), lv[l].smaps, &dsc->err, wait_limit, st);
        else launch_snapshot<T>(v, area_ptr(), st);
    }

    // One directional sweep k of grid l with tile shape sh.
    void sweep(int l, const LevelView<T> &v, int k, int sh) {
        if (p.smoother == MG_SMOOTH_PHASED) {
            launch_sweep_phased<T>(v, k, st);
        } else if (p.smoother == MG_SMOOTH_FUSED_VEC) {
            launch_sweep_fused<T>(v, k, sh, st);
        } else {
            if constexpr (std::is_same<T, float>::value)
                launch_sweep_tma(v, k, sh, lv[l].maps[sh], &dsc->err, wait_limit, st);
            else launch_sweep_fused<T>(v, k, sh, st);
        }
    }

    // The smoother after the snapshot: four directional sweeps of Hybrid Smoother 2, or GSLINE-I
    // (and the Hybrid Smoother 1 blocks).
    void relax(int l, const LevelView<T> &v, int sh) {
        if (p.smoother == MG_SMOOTH_GSLINE || p.smoother == MG_SMOOTH_HS1) {
            launch_gsline<T>(v, st);
            if (p.smoother == MG_SMOOTH_HS1) launch_hs1_blocks<T>(v, st);
        } else {
            for (int k = 0; k < 4; ++k) sweep(l, v, k, sh);
        }
    }

    void smooth(int l) {
        Range range("smoothing iteration");
        LevelView<T> v = view(l);
        if (l == 0 && skip_first_snapshot) {
            skip_first_snapshot = 0;   // area term and snapshot are in the loop's first part
            launches -= area_launches(l) + 1;
        } else {
            area_term(l, lv[l].u);
            if (l == fas_level) {   // the first snapshot after the restriction also completes the rhs
                if constexpr (std::is_same<T, float>::value)
                    launch_snapshot_fas_tma(v, area_ptr(), lv[l].smaps, &dsc->err, wait_limit, st);
                fas_level = -1;
            } else if (l == interp_level) {   // the first snapshot after the coarse grid applies its correction
                if constexpr (std::is_same<T, float>::value)
                    launch_snapshot_interp_tma(v, view(l + 1), area_ptr(), lv[l].smaps, &dsc->err, wait_limit, st);
                interp_level = -1;
            } else {
                snapshot(l, v);
            }
        }
        if (use_omega && infer_pending[l] && omega_buf[l]) {
            launch_omega_infer<T>(v, net, omega_buf[l], st);   // weights from this snapshot's G
            infer_pending[l] = false;
            ++launches;
        }
        relax(l, v, shape[l]);
        launches += area_launches(l) + 1 + smoother_launches(l);
    }

    void cycle(int l) {
        static const char *kLevelNames[kMaxLevels] = {"grid 0", "grid 1", "grid 2", "grid 3", "grid 4", "grid 5",
                                                      "grid 6", "grid 7", "grid 8", "grid 9", "grid 10", "grid 11",
                                                      "grid 12", "grid 13", "grid 14", "grid 15"};
        Range range(kLevelNames[l]);
        if (l == 0) fas_level = interp_level = -1;   // nothing pending from an enqueue cut short
        if (l == lc) {
            launch_bottom_cycle(true);
            ++launches;
            return;
        }
        if (l == lb) {
            launch_bottom_cycle();
            ++launches;
            return;
        }
        if (l == nlev - 1) {
            launch_coarse_solve<T>(view(l), p.precision == MG_MIXED, mp, A1 / ((double)n * m), h2nm(l),
                                   p.coarse_maxit, p.coarse_tol, coarse, dsc, p.coarse_solver == MG_COARSE_AOS,
                                   p.aos_dt, st);
            ++launches;
            return;
        }
        for (int t = 0; t < p.nu1; ++t) smooth(l);
        Level<T> &L = lv[l], &C = lv[l + 1];
        area_term(l, L.u);
        if constexpr (std::is_same<T, float>::value) {
            launch_residual_restrict_tma(view(l), view(l + 1), area_ptr(), L.rmaps, &dsc->err, wait_limit, st);
            launches += 1;
        } else {
            launch_residual<T>(view(l), L.u, area_ptr(), L.r, 0, partials, 0, nullptr, st);
            launch_restrict<T>(L.r, L.n, L.m, L.pitch, C.rhs, nullptr, C.pitch, st);
            launch_restrict<T>(L.u, L.n, L.m, L.pitch, C.u, C.u0, C.pitch, st);
            launches += 3;
        }
        // FAS right-hand side on grid l+1: rhs += L(pn + u0).  FP32 storage with a pre-smoothing
        // on grid l+1 by the per-grid kernels: its first snapshot completes it (fas_level);
        // otherwise a residual launch here
        const bool fas_in_snapshot = std::is_same<T, float>::value && p.nu1 >= 1 && l + 1 != lc && l + 1 != lb &&
                                     l + 1 < nlev - 1;
        if (fas_in_snapshot) {
            fas_level = l + 1;
            launches += area_launches(l);
        } else {
            area_term(l + 1, C.u0);
            if constexpr (std::is_same<T, float>::value)
                launch_residual_tma(view(l + 1), 1, area_ptr(), C.rhs, 1, partials, 0, nullptr, C.smaps, C.rmaps,
                                    &dsc->err, wait_limit, st);
            else launch_residual<T>(view(l + 1), C.u0, area_ptr(), C.rhs, 1, partials, 0, nullptr, st);
            launches += area_launches(l) + area_launches(l + 1) + 1;
        }
        cycle(l + 1);
        // the coarse-grid correction: in the first post-smoothing snapshot (FP32 storage, the
        // Spencer-Chen model: the Rada-Chen area term before a snapshot reads the corrected u),
        // else its own launch
        if (std::is_same<T, float>::value && p.nu2 >= 1 && p.model == MG_MODEL_SC) {
            interp_level = l;
        } else {
            launch_interp_add<T>(view(l), view(l + 1), st);
            ++launches;
        }
        for (int t = 0; t < p.nu2; ++t) smooth(l);
    }

    void enqueue_vcycle(bool readback = true) {
        cycle(0);
        area_term(0, lv[0].u);
        norm_residual(&dsc->norm2);
        launches += area_launches() + norm_launches();
        if (readback) cudaMemcpyAsync(hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, st);
    }

    // One V-cycle (ending with the finest residual norm on the device) captured into a graph,
    // for composition into a batch graph.  Returns the graph and its kernel count.
    int capture_vcycle(cudaGraph_t *g, long long *nodes) {
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        long long before = launches;
        enqueue_vcycle(false);
        *nodes = launches - before;
        launches = before;
        cudaError_t e = cudaStreamEndCapture(st, g);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        return MG_OK;
    }

    int set_shapes(const int *sh) override {
        for (int l = 0; l < nlev - 1; ++l)
            if (sh[l] < 0 || sh[l] >= kTileShapes) return fail(MG_ERR_ARG, "tile shape out of range");
        for (int l = 0; l < nlev - 1; ++l) shape[l] = sh[l];
        drop_graphs();
        return MG_OK;
    }

    // Picks the fused-sweep tile shape of every grid by timing one outer smoothing iteration
    // (snapshot + four sweeps, `reps` times, replayed as a graph when the solver uses graphs)
    // per shape; the state is restored afterwards.
    int autotune(int reps, int *out) {
        if (!in_step) return fail(MG_ERR_STATE, "mg_autotune outside a step");
        if (!fused()) return fail(MG_ERR_ARG, "autotune applies to the fused Hybrid Smoother 2");
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        for (int l = 0; l < nlev - 1; ++l) {
            Level<T> &L = lv[l];
            const size_t row = (size_t)L.m * sizeof(T), pitchb = (size_t)L.pitch * sizeof(T);
            float best = 1e30f;
            int arg = 0;
            for (int sh = 0; sh < kTileShapes; ++sh) {
                CK(cudaMemcpy2DAsync(L.r, pitchb, L.u, pitchb, row, L.n, cudaMemcpyDeviceToDevice, st));
                LevelView<T> v = view(l);
                auto enqueue = [&]() {
                    for (int r = 0; r < reps; ++r) {
                        area_term(l, L.u);
                        snapshot(l, v);
                        for (int k = 0; k < 4; ++k) sweep(l, v, k, sh);
                    }
                };
                // With graphs, time a captured graph of the iterations: eager launches would
                // measure the host's launch rate on the small grids, not the kernels.
                cudaGraphExec_t ge = nullptr;
                if (p.use_graph) {
                    cudaGraph_t g;
                    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                    enqueue();
                    cudaError_t e = cudaStreamEndCapture(st, &g);
                    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
                    e = cudaGraphInstantiate(&ge, g, 0);
                    cudaGraphDestroy(g);
                    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
                }
                float t = 0;
                for (int warm = 0; warm < 2; ++warm) {
                    CK(cudaEventRecord(e0, st));
                    if (ge) CK(cudaGraphLaunch(ge, st));
                    else enqueue();
                    CK(cudaEventRecord(e1, st));
                    CK(cudaEventSynchronize(e1));
                    CK(cudaEventElapsedTime(&t, e0, e1));
                }
                if (ge) cudaGraphExecDestroy(ge);
                CKL();
                CK(cudaMemcpy2DAsync(L.u, pitchb, L.r, pitchb, row, L.n, cudaMemcpyDeviceToDevice, st));
                if (t < best) { best = t; arg = sh; }
            }
            shape[l] = arg;
            if (out) out[l] = arg;
        }
        drop_graphs();   // shapes are baked into the graphs
        int rc = MG_OK;
        if (lb >= 0 && (learn_mode == 0 || learn_mode == 3)) rc = tune_bottom(reps, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return rc;
    }

    // Times `reps` V-cycles (after one untimed) for each way of running the bottom of the V-cycle:
    // the one-block kernel from lb_first, lb_first + 1, lb_first + 2, and the cluster kernel from
    // lb_first - 1 and lb_first where such a cluster fits; keeps the fastest.  The finest increment
    // (saved in ubak: a V-cycle writes every other finest-grid scratch field) and the device
    // scalars are restored after each candidate (the coarse grids are rebuilt by every V-cycle).
    int tune_bottom(int reps, cudaEvent_t e0, cudaEvent_t e1) {
        Level<T> &L = lv[0];
        const size_t row = (size_t)L.m * sizeof(T), pitchb = (size_t)L.pitch * sizeof(T);
        if (!ubak) CK(cudaMalloc(&ubak, sizeof(T) * (size_t)L.n * L.pitch));
        Scalars saved;
        CK(cudaMemcpyAsync(&saved, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const long long launches0 = launches;
        float best = 1e30f;
        int best_lb = lb, best_lc = lc;
        struct Cand { bool cluster; int level; };
        Cand cands[5];
        int nc = 0;
        for (int c = lb_first; c <= std::min(lb_first + 2, nlev - 2); ++c) cands[nc++] = {false, c};
        for (int c = std::max(lb_first - 1, 0); c <= std::min(lb_first, nlev - 2); ++c) cands[nc++] = {true, c};
        for (int k = 0; k < nc; ++k) {
            if (cands[k].cluster) {
                if (set_cluster_level(cands[k].level) != MG_OK) continue;   // no such cluster fits
            } else {
                lc = -1;
                use_bottom_from(cands[k].level);
                drop_graphs();
            }
            CK(cudaMemcpy2DAsync(ubak, pitchb, L.u, pitchb, row, L.n, cudaMemcpyDeviceToDevice, st));
            int rc = cycle_plain();   // captures this candidate's graph
            float t = 0;
            if (rc == MG_OK) {
                CK(cudaEventRecord(e0, st));
                for (int r = 0; r < reps && rc == MG_OK; ++r) rc = cycle_plain();
                CK(cudaEventRecord(e1, st));
                CK(cudaEventSynchronize(e1));
                CK(cudaEventElapsedTime(&t, e0, e1));
            }
            CK(cudaMemcpy2DAsync(L.u, pitchb, ubak, pitchb, row, L.n, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(dsc, &saved, sizeof(Scalars), cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));
            if (rc != MG_OK) return rc;
            if (t < best) {
                best = t;
                best_lb = lb;
                best_lc = lc;
            }
        }
        launches = launches0;
        use_bottom_from(best_lb);
        lc = -1;
        if (best_lc >= 0) set_cluster_level(best_lc);
        drop_graphs();
        return MG_OK;
    }

    // Enqueues one V-cycle, replayed from a graph captured once per kind (plain, learned,
    // learned with inference).
    int run_cycle(cudaGraphExec_t &ge, long long &nodes) {
        if (p.use_graph) {
            if (!ge) {
                cudaGraph_t g;
                bool pend[kMaxLevels];
                std::copy(std::begin(infer_pending), std::end(infer_pending), pend);
                CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
                long long before = launches;
                enqueue_vcycle();
                nodes = launches - before;
                launches = before;
                std::copy(std::begin(pend), std::end(pend), infer_pending);
                cudaError_t e = cudaStreamEndCapture(st, &g);
                if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
                e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) { ge = nullptr; return fail(MG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e)); }
            }
            CK(cudaGraphLaunch(ge, st));
            launches += nodes;
        } else {
            enqueue_vcycle();
            CKL();
        }
        CK(cudaStreamSynchronize(st));
        return MG_OK;
    }

    int cycle_plain() {
        use_omega = (learn_mode == 3);
        std::fill(std::begin(infer_pending), std::end(infer_pending), false);
        int rc = learn_mode == 3 ? run_cycle(gexec_l, nodes_l) : run_cycle(gexec, graph_nodes);
        use_omega = false;
        return rc;
    }

    int cycle_learned() {
        const bool infer = learn_since == 0 || learn_since >= learn_refresh;
        use_omega = true;
        for (int l = 0; l < nlev; ++l) infer_pending[l] = infer && omega_buf[l] != nullptr;
        int rc = infer ? run_cycle(gexec_li, nodes_li) : run_cycle(gexec_l, nodes_l);
        use_omega = false;
        std::fill(std::begin(infer_pending), std::end(infer_pending), false);
        learn_since = infer ? 1 : learn_since + 1;
        return rc;
    }

    double current_rho() const { return res0 > 0 ? std::sqrt(hsc->norm2) / res0 : std::sqrt(hsc->norm2); }

    int vcycle(double *rhoout) override {
        Range range("V-cycle");
        if (!in_step) return fail(MG_ERR_STATE, "mg_vcycle before mg_begin_step");
        const double rho_prev = rho > 0 ? rho : 1.0;
        int rc;
        if (learn_mode == 0 || learn_mode == 3) {
            rc = cycle_plain();
        } else if (learn_mode == 2) {
            rc = cycle_learned();
        } else if (plain_rate < 0 || learn_skip > 0) {
            // the first V-cycle of the step, or a back-off after a rejected learned V-cycle:
            // plain, and its rate is the reference
            rc = cycle_plain();
            if (!rc) plain_rate = current_rho() / rho_prev;
            if (learn_skip > 0) --learn_skip;
        } else {
            // learned V-cycle, kept only if it contracts at least as fast as the last plain one
            Level<T> &F = lv[0];
            const size_t row = (size_t)F.m * sizeof(T), pb = (size_t)F.pitch * sizeof(T);
            CK(cudaMemcpy2DAsync(ubak, pb, F.u, pb, row, F.n, cudaMemcpyDeviceToDevice, st));
            rc = cycle_learned();
            if (!rc) {
                const double r = current_rho();
                if (std::isfinite(r) && r / rho_prev <= plain_rate) {
                    ++learned_acc;
                    learn_backoff = 1;
                } else {
                    ++learned_rej;
                    learn_skip = learn_backoff;                  // plain for a while, doubling
                    learn_backoff = std::min(2 * learn_backoff, 8);
                    CK(cudaMemcpy2DAsync(F.u, pb, ubak, pb, row, F.n, cudaMemcpyDeviceToDevice, st));
                    rc = cycle_plain();
                    if (!rc) plain_rate = current_rho() / rho_prev;
                }
            }
        }
        if (rc) return rc;
        ++cycles_step;
        ++cycles_total;
        rho = current_rho();
        if (inject_cycle > 0 && cycles_step == inject_cycle) {   // host-side fault injection
            inject_cycle = 0;
            rho = 1e9;
        }
        if (rhoout) *rhoout = rho;
        if (hsc->err & 1) return fail(MG_ERR_NOT_SPD, "coarsest Cholesky: non-positive pivot");
        if (hsc->err & 4) {   // reported once: the word is cleared so the handle stays usable
            CK(cudaMemsetAsync(&dsc->err, 0, sizeof(int), st));
            CK(cudaStreamSynchronize(st));
            return fail(MG_ERR_TIMEOUT, "a tile copy into shared memory did not complete within the wait limit");
        }
        if (!std::isfinite(rho)) return fail(MG_ERR_NAN, "non-finite residual");
        if (rho > 1e3) return fail(MG_ERR_DIVERGED, "residual grew by more than 1e3");
        return MG_OK;
    }

    // Learned relaxation weights: parameters (host FP32, NULL keeps the current ones), mode and
    // inference interval.  Weight grids exist on the grids the per-grid kernels smooth.
    int set_learned(const float *theta, int mode, int refresh) override {
        if (mode < 0 || mode > 2 || refresh < 1) return fail(MG_ERR_ARG, "mode must be 0..2, refresh >= 1");
        if (mode > 0 && !fused()) return fail(MG_ERR_ARG, "learned weights apply to the fused Hybrid Smoother 2");
        if (theta) {
            const int np = learned_nparam();
            std::vector<__nv_bfloat16> hb(np);
            for (int k = 0; k < np; ++k) hb[k] = __float2bfloat16(theta[k]);
            if (!net) CK(cudaMalloc(&net, sizeof(__nv_bfloat16) * np));
            CK(cudaMemcpy(net, hb.data(), sizeof(__nv_bfloat16) * np, cudaMemcpyHostToDevice));
        }
        if (mode > 0 && !net) return fail(MG_ERR_ARG, "no parameters given");
        if (mode > 0) {
            int rc = alloc_omega();
            if (rc) return rc;
            for (int l = 0; l < nlev; ++l) omega_valid[l] = omega_buf[l] != nullptr;   // inferred before use
        }
        learn_mode = mode;
        learn_refresh = refresh;
        learn_since = 0;
        plain_rate = -1.0;
        drop_graphs();
        return MG_OK;
    }

    int alloc_omega() {
        const int top = lb >= 0 ? lb : nlev - 1;
        for (int l = 0; l < top; ++l)
            if (!omega_buf[l]) CK(cudaMalloc(&omega_buf[l], sizeof(T) * (size_t)lv[l].n * lv[l].pitch));
        if (!ubak) CK(cudaMalloc(&ubak, sizeof(T) * (size_t)lv[0].n * lv[0].pitch));
        return MG_OK;
    }

    // Training crops of the finest grid's current frozen system (coefficients and f of the last
    // snapshot, the current increment u) at seeded random origins.
    int record_crops(float *data, int first, int count, unsigned long long seed) override {
        const int c = learned_crop();
        const Level<T> &L = lv[0];
        if (L.n < c || L.m < c) return fail(MG_ERR_ARG, "finest grid smaller than a crop");
        std::mt19937_64 rng(seed);
        std::vector<int> org(2 * count);
        for (int k = 0; k < count; ++k) {
            org[2 * k] = (int)(rng() % (unsigned long long)(L.n - c + 1));
            org[2 * k + 1] = (int)(rng() % (unsigned long long)(L.m - c + 1));
        }
        int *d = nullptr;
        CK(cudaMallocAsync(&d, sizeof(int) * 2 * count, st));
        CK(cudaMemcpyAsync(d, org.data(), sizeof(int) * 2 * count, cudaMemcpyHostToDevice, st));
        launch_record_crops<T>(view(0), d, count, data, first, st);
        ++launches;
        CKL();
        CK(cudaFreeAsync(d, st));
        CK(cudaStreamSynchronize(st));
        return MG_OK;
    }

    // Fixed relaxation weights of grid l (host, n_l x m_l of the storage type; NULL: none).
    int set_omega(int l, const void *w) override {
        if (l < 0 || l >= nlev - 1) return fail(MG_ERR_ARG, "level");
        if (lb >= 0 && l >= lb) return fail(MG_ERR_ARG, "grid smoothed by the bottom kernel (disable it first)");
        if (!fused()) return fail(MG_ERR_ARG, "weights apply to the fused Hybrid Smoother 2");
        int rc = alloc_omega();
        if (rc) return rc;
        if (w) {
            const Level<T> &L = lv[l];
            CK(cudaMemcpy2D(omega_buf[l], (size_t)L.pitch * sizeof(T), w, (size_t)L.m * sizeof(T),
                            (size_t)L.m * sizeof(T), L.n, cudaMemcpyHostToDevice));
            if (learn_mode != 3) std::fill(std::begin(omega_valid), std::end(omega_valid), false);
            omega_valid[l] = true;
            learn_mode = 3;
        } else {
            omega_valid[l] = false;
            bool any = false;
            for (bool b : omega_valid) any = any || b;
            if (!any && learn_mode == 3) learn_mode = 0;
        }
        drop_graphs();
        return MG_OK;
    }

    const mg_params &params() const override { return p; }

    // phi = phi^n again on the finest grid (the increment zeroed), nothing else changed
    // The step loop graph: reset the loop counter, then a while node whose body is one V-cycle
    // (captured) and k_step_loop, then the copy of the scalars to the host.
    // Whether the fused form of the step loop applies: FP32 storage, the V-cycle starts with a
    // smoothing iteration of the finest grid run by the per-grid kernels.
    bool loop_fusable() const {
        if constexpr (!std::is_same<T, float>::value) return false;
        else return p.nu1 >= 1 && nlev >= 2 && lb != 0 && lc != 0 && !use_omega;
    }

    // The fused loop's first part: the area term and the finest grid's snapshot, which also
    // writes the norm of the state it reads to dsc->norm2.
    int capture_first(cudaGraph_t *g, long long *nodes) {
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        area_term(0, lv[0].u);
        if constexpr (std::is_same<T, float>::value)
            launch_snapshot_norm_tma(view(0), area_ptr(), lv[0].smaps, partials, &dsc->err, wait_limit, st);
        launch_sum_partials(partials, npart, &dsc->norm2, st);
        *nodes = area_launches() + 1 + sum_launches(0);
        cudaError_t e = cudaStreamEndCapture(st, g);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        return MG_OK;
    }

    // The rest of a V-cycle after that snapshot (no norm at its end).
    int capture_rest(cudaGraph_t *g, long long *nodes) {
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        long long before = launches;
        skip_first_snapshot = 1;
        cycle(0);
        skip_first_snapshot = 0;
        *nodes = launches - before;
        launches = before;
        cudaError_t e = cudaStreamEndCapture(st, g);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        return MG_OK;
    }

    // first part; while (go) { rest of the V-cycle; first part (the next V-cycle's snapshot, with
    // the norm of the state this V-cycle left); the step control's tests (set go) }.  The snapshot
    // of the V-cycle that does not run when the attempt stops is the only extra work.
    int build_loop_fused(double tol, int max_cycles) {
        cudaGraph_t gf = nullptr, gr = nullptr, G = nullptr;
        long long nf = 0, nr = 0;
        int rc = capture_first(&gf, &nf);
        if (!rc) rc = capture_rest(&gr, &nr);
        if (rc) {
            if (gf) cudaGraphDestroy(gf);
            return rc;
        }
        cudaError_t e = cudaGraphCreate(&G, 0);
        cudaGraphNode_t ms = nullptr, f0 = nullptr, wn = nullptr, cr = nullptr, cf = nullptr, kn = nullptr,
                        mc = nullptr;
        if (e == cudaSuccess) {
            cudaMemsetParams mp_{};
            mp_.dst = &dsc->loop_j;
            mp_.value = 0;
            mp_.elementSize = sizeof(int);
            mp_.width = 1;
            mp_.height = 1;
            e = cudaGraphAddMemsetNode(&ms, G, nullptr, 0, &mp_);
        }
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&f0, G, &ms, 1, gf);
        cudaGraphConditionalHandle hw{};
        cudaGraph_t body = nullptr;
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hw, G, 1, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) {
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = hw;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&wn, G, &f0, nullptr, 1, &cp);
            if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
        }
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&cr, body, nullptr, 0, gr);
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&cf, body, &cr, 1, gf);
        if (e == cudaSuccess) {
            Scalars *sc = dsc;
            double t = tol, sr = p.stall_ratio;
            int mx = max_cycles;
            void *args[] = {&hw, (void *)&sc, &t, &mx, &sr};
            cudaKernelNodeParams kp = {};
            kp.func = (void *)k_step_loop;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(1);
            kp.kernelParams = args;
            e = cudaGraphAddKernelNode(&kn, body, &cf, 1, &kp);
        }
        if (e == cudaSuccess) e = cudaGraphAddMemcpyNode1D(&mc, G, &wn, 1, hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gloop, G, 0);
        if (gf) cudaGraphDestroy(gf);
        if (gr) cudaGraphDestroy(gr);
        if (G) cudaGraphDestroy(G);
        if (e != cudaSuccess) {
            gloop = nullptr;
            return fail(MG_ERR_CUDA, std::string("fused step loop graph: ") + cudaGetErrorString(e));
        }
        gloop_tol = tol;
        gloop_max = max_cycles;
        gloop_nodes = nr;
        gloop_first = nf;
        gloop_fused = true;
        return MG_OK;
    }

    int build_loop(double tol, int max_cycles) {
        if (gloop) { cudaGraphExecDestroy(gloop); gloop = nullptr; }
        if (loop_fusable()) return build_loop_fused(tol, max_cycles);
        gloop_fused = false;
        cudaGraph_t vg = nullptr, G = nullptr;
        long long nodes = 0;
        int rc = capture_vcycle(&vg, &nodes);
        if (rc) return rc;
        cudaError_t e = cudaGraphCreate(&G, 0);
        cudaGraphNode_t ms = nullptr, wn = nullptr, child = nullptr, kn = nullptr, mc = nullptr;
        if (e == cudaSuccess) {
            cudaMemsetParams mp_{};
            mp_.dst = &dsc->loop_j;
            mp_.value = 0;
            mp_.elementSize = sizeof(int);
            mp_.width = 1;
            mp_.height = 1;
            e = cudaGraphAddMemsetNode(&ms, G, nullptr, 0, &mp_);
        }
        cudaGraphConditionalHandle hc{};
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hc, G, 1, cudaGraphCondAssignDefault);
        cudaGraph_t body = nullptr;
        if (e == cudaSuccess) {
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = hc;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            e = cudaGraphAddNode(&wn, G, &ms, nullptr, 1, &cp);
            if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
        }
        if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&child, body, nullptr, 0, vg);
        if (e == cudaSuccess) {
            Scalars *sc = dsc;
            double t = tol, sr = p.stall_ratio;
            int mx = max_cycles;
            void *args[] = {&hc, (void *)&sc, &t, &mx, &sr};
            cudaKernelNodeParams kp = {};
            kp.func = (void *)k_step_loop;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(1);
            kp.kernelParams = args;
            e = cudaGraphAddKernelNode(&kn, body, &child, 1, &kp);
        }
        if (e == cudaSuccess) e = cudaGraphAddMemcpyNode1D(&mc, G, &wn, 1, hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gloop, G, 0);
        if (vg) cudaGraphDestroy(vg);
        if (G) cudaGraphDestroy(G);
        if (e != cudaSuccess) { gloop = nullptr; return fail(MG_ERR_CUDA, std::string("step loop graph: ") + cudaGetErrorString(e)); }
        gloop_tol = tol;
        gloop_max = max_cycles;
        gloop_nodes = nodes;
        return MG_OK;
    }

    int loop_attempt(double tol, int max_cycles, std::vector<double> &hist, int &stop) override {
        // per-V-cycle host decisions (learned weights, injected faults) or no graphs: not here
        if (!p.use_graph || learn_mode != 0 || inject_cycle > 0 || max_cycles > kLoopMaxCycles)
            return MG_ERR_STATE;
        if (!in_step) return fail(MG_ERR_STATE, "step loop outside a step");
        if (!gloop || gloop_tol != tol || gloop_max != max_cycles) {
            int rc = build_loop(tol, max_cycles);
            if (rc) return rc;
        }
        CK(cudaGraphLaunch(gloop, st));
        CK(cudaStreamSynchronize(st));
        res0_in_hsc = res0_pending;   // the graph copied the scalars back, the reference norm with them
        const int j = hsc->loop_j;
        stop = hsc->loop_stop;
        hist.assign(hsc->loop_rho + 1, hsc->loop_rho + 1 + j);
        cycles_step += j;
        cycles_total += j;
        if (gloop_fused)   // the first part once before the loop and once per V-cycle
            launches += (long long)(j + 1) * gloop_first + (long long)j * (gloop_nodes + 1) + 1;
        else
            launches += (long long)j * (gloop_nodes + 1) + 1;
        rho = j > 0 ? hist.back() : 1.0;
        if (hsc->err & 1) return fail(MG_ERR_NOT_SPD, "coarsest Cholesky: non-positive pivot");
        if (hsc->err & 4) {
            CK(cudaMemsetAsync(&dsc->err, 0, sizeof(int), st));
            CK(cudaStreamSynchronize(st));
            return fail(MG_ERR_TIMEOUT, "a tile copy into shared memory did not complete within the wait limit");
        }
        if (stop == 4) return std::isfinite(rho) ? fail(MG_ERR_DIVERGED, "residual grew by more than 1e3")
                                                 : fail(MG_ERR_NAN, "non-finite residual");
        return MG_OK;
    }

    int zero_increment() {
        Level<T> &F = lv[0];
        CK(cudaMemset2DAsync(F.u, (size_t)F.pitch * sizeof(T), 0, (size_t)F.m * sizeof(T), F.n, st));
        return MG_OK;
    }

    int inject_divergence(int cycle) override {
        if (cycle < 0) return fail(MG_ERR_ARG, "cycle < 0");
        inject_cycle = cycle;
        return MG_OK;
    }

    int set_wait_limit(long long rounds) override {
        if (rounds < 0) return fail(MG_ERR_ARG, "wait limit < 0");
        wait_limit = rounds;
        drop_graphs();   // the limit is a launch argument baked into the graphs
        return MG_OK;
    }
    void set_cycles_step(int c) override { cycles_step = c; }

    // Rejects the current attempt at a step: phi = phi^n again (the increment u of the finest
    // grid is zeroed; the coarse grids are rebuilt by every V-cycle) and the following attempts
    // and steps use `tau` (the graphs, which hold 1/tau, are captured again).
    int restart_step(double tau) override {
        if (!in_step) return fail(MG_ERR_STATE, "restart outside a step");
        Level<T> &F = lv[0];
        CK(cudaMemset2DAsync(F.u, (size_t)F.pitch * sizeof(T), 0, (size_t)F.m * sizeof(T), F.n, st));
        p.tau = tau;
        ++rejected;
        drop_graphs();
        in_step = false;
        return MG_OK;
    }

    int end_step(double *etaout) override {
        Range range("end step");
        if (!in_step) return fail(MG_ERR_STATE, "mg_end_step before mg_begin_step");
        launch_region_sums<T>(view(0), p.eps, partials, npart, dsc, 1, st);
        launches += norm_launches();   // region partials and their (chunked) sums
        CKL();
        CK(cudaMemcpyAsync(eta_sums(), &dsc->sums[4], 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        eta_pending = true;
        ++steps;
        in_step = false;
        if (etaout) {
            CK(cudaStreamSynchronize(st));
            *etaout = last_eta();
        }
        return MG_OK;
    }

    // the two sums of eta (sum of u^2, sum of phi_n^2) in the pinned staging buffer
    double *eta_sums() const { return hstage + 6 * (size_t)kcap + 9; }

    int mask(unsigned char *out) override {
        if (int rc = mask_async(out)) return rc;
        CK(cudaStreamSynchronize(st));
        return MG_OK;
    }

    int mask_async(unsigned char *out) override {
        launch_mask<T>(view(0), out, st);
        ++launches;
        CKL();
        return MG_OK;
    }

    int get_phi(void *out) override {
        dim3 grid((m + 31) / 32, (n + 7) / 8);
        k_phi_out<T><<<grid, dim3(32, 8), 0, st>>>(lv[0].pn, lv[0].u, n, m, lv[0].pitch, (T *)out);
        ++launches;
        CKL();
        CK(cudaStreamSynchronize(st));
        return MG_OK;
    }

    int set_phi(const void *in) override {
        dim3 grid((m + 31) / 32, (n + 7) / 8);
        k_phi_in<T><<<grid, dim3(32, 8), 0, st>>>((const T *)in, n, m, lv[0].pitch, lv[0].pn, lv[0].u);
        CKL();
        in_step = false;
        CK(cudaStreamSynchronize(st));
        return MG_OK;
    }

    int set_regions(double c1, double c2) override {
        double c[2] = {c1, c2};
        CK(cudaMemcpyAsync(&dsc->c1, c, sizeof(c), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        return MG_OK;
    }

    int get_level(int l, int field, void *out) override {
        if (l < 0 || l >= nlev || field < 0 || field > 7) return fail(MG_ERR_ARG, "level / field out of range");
        Level<T> &L = lv[l];
        if (field == 0) {
            dim3 grid((L.m + 31) / 32, (L.n + 7) / 8);
            k_phi_out<T><<<grid, dim3(32, 8), 0, st>>>(L.pn, L.u, L.n, L.m, L.pitch, (T *)out);
        } else {
            const T *src = field == 1 ? L.w : field == 2 ? L.z : field == 3 ? L.d : field == 4 ? L.F
                         : field == 5 ? L.rhs : field == 6 ? L.G : omega_buf[l];
            if (!src) return fail(MG_ERR_ARG, "field not stored on this level");
            launch_copy_out<T>(src, (T *)out, L.n, L.m, L.pitch, st);
        }
        CKL();
        CK(cudaStreamSynchronize(st));
        return MG_OK;
    }

    int rows() const override { return n; }
    int cols() const override { return m; }
    int steps_done() const override { return steps; }
    double last_eta() const override {
        if (eta_pending) {
            cudaStreamSynchronize(st);   // the copy of end_step's sums; an error here reaches the next call
            const double *e = eta_sums();
            eta = e[1] > 0 ? std::sqrt(e[0] / e[1]) : std::sqrt(e[0]);
            eta_pending = false;
        }
        return eta;
    }

    int stats(mg_stats *s) override {
        CK(cudaMemcpyAsync(hsc, dsc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        s->n = n; s->m = m; s->levels = nlev; s->precision = p.precision;
        s->steps = steps; s->cycles_step = cycles_step; s->cycles_total = cycles_total;
        s->picard_last = hsc->picard;
        s->rho = rho; s->res0 = res0; s->eta = last_eta();
        s->c1 = hsc->c1; s->c2 = hsc->c2; s->A1 = A1;
        s->device_bytes = pool_bytes;
        s->launches = launches;
        s->learned_accepted = learned_acc;
        s->learned_rejected = learned_rej;
        s->bottom_level = lc >= 0 ? -1 : lb;
        s->cluster_level = lc;
        s->tau = p.tau;
        s->attempts_rejected = rejected;
        return MG_OK;
    }

    int time_kernels(int l, int reps, double *ms) override {
        if (l < 0 || l >= nlev || reps < 1) return fail(MG_ERR_ARG, "level / reps");
        if (!in_step) return fail(MG_ERR_STATE, "mg_time_kernels outside a step");
        cudaEvent_t ev[7];
        for (auto &e : ev) CK(cudaEventCreate(&e));
        double acc[6] = {0, 0, 0, 0, 0, 0};
        LevelView<T> v = view(l);
        for (int r = 0; r < reps; ++r) {
            area_term(l, lv[l].u);
            cudaEventRecord(ev[0], st);
            snapshot(l, v);
            cudaEventRecord(ev[1], st);
            if (p.smoother == MG_SMOOTH_GSLINE || p.smoother == MG_SMOOTH_HS1) {
                relax(l, v, shape[l]);        // the whole smoother in the first slot
                for (int k = 0; k < 4; ++k) cudaEventRecord(ev[2 + k], st);
            } else {
                for (int k = 0; k < 4; ++k) {
                    sweep(l, v, k, shape[l]);
                    cudaEventRecord(ev[2 + k], st);
                }
            }
            if constexpr (std::is_same<T, float>::value)
                launch_residual_tma(v, 0, area_ptr(), lv[l].r, 0, partials, 0, nullptr, lv[l].smaps, lv[l].rmaps,
                                    &dsc->err, wait_limit, st);
            else launch_residual<T>(v, lv[l].u, area_ptr(), lv[l].r, 0, partials, 0, nullptr, st);
            cudaEventRecord(ev[6], st);
            launches += area_launches(l) + 2 + smoother_launches(l);
            CKL();
            CK(cudaEventSynchronize(ev[6]));
            for (int k = 0; k < 6; ++k) {
                float t = 0;
                cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
                acc[k] += t;
            }
        }
        for (auto &e : ev) cudaEventDestroy(e);
        for (int k = 0; k < 6; ++k) ms[k] = acc[k] / reps;
        return MG_OK;
    }

    // The sweeps of grid l as a V-cycle's graph replays them: one snapshot at the current state,
    // then the sweeps A..D of `reps` outer iterations captured back to back in one graph (the
    // snapshot's lagged coefficients and member masks serve every sweep), launched once
    // untimed and once between two events; ms[0] = mean ms per sweep, kernel boundaries of the
    // graph included.
    int time_sweeps_graph(int l, int reps, double *ms) override {
        if (l < 0 || l >= nlev || reps < 1 || reps > 256) return fail(MG_ERR_ARG, "level / reps");
        if (!in_step) return fail(MG_ERR_STATE, "mg_time_sweeps_graph outside a step");
        if (p.smoother == MG_SMOOTH_GSLINE || p.smoother == MG_SMOOTH_HS1)
            return fail(MG_ERR_ARG, "mg_time_sweeps_graph times the Hybrid Smoother 2 sweeps");
        const LevelView<T> v = view(l);
        area_term(l, lv[l].u);
        snapshot(l, v);
        launches += area_launches(l) + 1;
        CKL();
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int r = 0; r < reps; ++r)
            for (int k = 0; k < 4; ++k) sweep(l, v, k, shape[l]);
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t ge = nullptr;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        float t = 0;
        e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        for (int it = 0; it < 2 && e == cudaSuccess; ++it) {   // the first launch warms up
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaGraphExecDestroy(ge);
        if (e != cudaSuccess) return fail(MG_ERR_CUDA, cudaGetErrorString(e));
        launches += 2LL * reps * smoother_launches(l);
        ms[0] = (double)t / (4.0 * reps);
        return MG_OK;
    }

    // The residual kernels a V-cycle runs on grid l: [0] the residual norm (the tile kernel and
    // the final sum; the norm goes to a scratch slot), [1] the residual with full weighting into
    // grid l + 1 (-1 on the coarsest grid).  Writes grid l + 1's rhs, u and u0.
    int time_residuals(int l, int reps, double *ms) override {
        if (l < 0 || l >= nlev || reps < 1) return fail(MG_ERR_ARG, "level / reps");
        if (!in_step) return fail(MG_ERR_STATE, "mg_time_residuals outside a step");
        cudaEvent_t ev[3];
        for (auto &e : ev) CK(cudaEventCreate(&e));
        double acc[2] = {0, 0};
        const LevelView<T> v = view(l);
        const int np = num_partials(lv[l].n, lv[l].m);
        for (int r = 0; r < reps; ++r) {
            area_term(l, lv[l].u);
            cudaEventRecord(ev[0], st);
            if constexpr (std::is_same<T, float>::value)
                launch_residual_tma(v, 0, area_ptr(), nullptr, 0, partials, np, &dsc->sums[6], lv[l].smaps,
                                    lv[l].rmaps, &dsc->err, wait_limit, st);
            else launch_residual<T>(v, lv[l].u, area_ptr(), lv[l].r, 0, partials, np, &dsc->sums[6], st);
            cudaEventRecord(ev[1], st);
            launches += area_launches(l) + norm_launches(l);
            if (l + 1 < nlev) {
                Level<T> &L = lv[l], &C = lv[l + 1];
                if constexpr (std::is_same<T, float>::value) {
                    launch_residual_restrict_tma(v, view(l + 1), area_ptr(), L.rmaps, &dsc->err, wait_limit, st);
                    launches += 1;
                } else {
                    launch_residual<T>(v, L.u, area_ptr(), L.r, 0, partials, 0, nullptr, st);
                    launch_restrict<T>(L.r, L.n, L.m, L.pitch, C.rhs, nullptr, C.pitch, st);
                    launch_restrict<T>(L.u, L.n, L.m, L.pitch, C.u, C.u0, C.pitch, st);
                    launches += 3;
                }
            }
            cudaEventRecord(ev[2], st);
            CKL();
            CK(cudaEventSynchronize(ev[2]));
            float t0 = 0, t1 = 0;
            cudaEventElapsedTime(&t0, ev[0], ev[1]);
            cudaEventElapsedTime(&t1, ev[1], ev[2]);
            acc[0] += t0;
            acc[1] += t1;
        }
        for (auto &e : ev) cudaEventDestroy(e);
        ms[0] = acc[0] / reps;
        ms[1] = l + 1 < nlev ? acc[1] / reps : -1.0;
        return MG_OK;
    }
};

int check_params(const mg_params *p, int n, int m) {
    if (!p) return fail(MG_ERR_ARG, "params is NULL");
    if (n < 1 || m < 1) return fail(MG_ERR_ARG, "image size must be positive");
    if (p->model != MG_MODEL_SC && p->model != MG_MODEL_RC) return fail(MG_ERR_ARG, "model");
    if (p->precision != MG_F32 && p->precision != MG_F64 && p->precision != MG_MIXED)
        return fail(MG_ERR_ARG, "precision");
    if (p->smoother < MG_SMOOTH_FUSED || p->smoother > MG_SMOOTH_HS1) return fail(MG_ERR_ARG, "smoother");
    if (p->coarse_solver != MG_COARSE_PICARD && p->coarse_solver != MG_COARSE_AOS) return fail(MG_ERR_ARG, "coarse_solver");
    if (p->coarse_solver == MG_COARSE_AOS && !(p->aos_dt > 0)) return fail(MG_ERR_ARG, "aos_dt <= 0");
    const double pos[] = {p->mu, p->eps, p->beta, p->sigma_blur, p->sigma_d};
    for (double v : pos)
        if (!(v > 0) || !std::isfinite(v)) return fail(MG_ERR_ARG, "mu, eps, beta, sigma_blur, sigma_d must be > 0");
    const double nonneg[] = {p->lambda1, p->lambda2, p->theta, p->nu, p->beta_edge, p->tau};
    for (double v : nonneg)
        if (!(v >= 0) || !std::isfinite(v)) return fail(MG_ERR_ARG, "weights and tau must be finite and >= 0");
    if (!(p->Sigma > 1)) return fail(MG_ERR_ARG, "Sigma must exceed 1");
    if (p->sigma_blur > 5.0) return fail(MG_ERR_ARG, "sigma_blur above 5 px is not supported");
    if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 > 64) return fail(MG_ERR_ARG, "nu1, nu2");
    if (p->levels < 1 || p->levels > kMaxLevels) return fail(MG_ERR_ARG, "levels");
    int nc = n >> (p->levels - 1), mc = m >> (p->levels - 1);
    if (nc < 1 || mc < 1) return fail(MG_ERR_ARG, "too many levels for the image size");
    if ((long)nc * mc > kMaxCoarseCells || std::min(nc, mc) > kMaxCoarseBand)
        return fail(MG_ERR_ARG, "coarsest grid too large for the direct solve (use more levels)");
    if (p->coarse_maxit < 1 || !(p->coarse_tol >= 0)) return fail(MG_ERR_ARG, "coarse_maxit / coarse_tol");
    if (p->model == MG_MODEL_SC && p->tau == 0 && p->lambda1 == 0 && p->lambda2 == 0 && p->theta == 0)
        return fail(MG_ERR_ARG, "degenerate model");
    if (!(p->stall_ratio >= 0 && p->stall_ratio < 1) || p->max_halvings < 0 || p->max_halvings > 60)
        return fail(MG_ERR_ARG, "stall_ratio must be in [0, 1) and max_halvings in [0, 60]");
    return MG_OK;
}

// The step control's test on the residual history of one attempt (rho[0..j-1] after V-cycle j):
// reject from the 4th V-cycle on when two V-cycles gained less than a factor 1 / stall_ratio.
bool attempt_stalled(const std::vector<double> &rho, double stall_ratio) {
    const size_t j = rho.size();
    return stall_ratio > 0 && j >= 4 && rho[j - 1] > stall_ratio * rho[j - 3];
}

// One pseudo-time step under the step control (mg_solve_step): attempts from phi^n with tau,
// tau / 2, ... until one reaches tol.  A rejected attempt restores phi^n.
int solve_step_controlled(SolverBase *s, double tol, int max_cycles, int *cycles, double *rho) {
    Range range("pseudo-time step");
    const bool control = s->params().stall_ratio > 0;
    int total = 0, rc = MG_OK;
    double r = 1.0;
    bool ok = false;
    const int step0 = s->steps_done();
    for (int attempt = 0;; ++attempt) {
        if ((rc = s->begin_step_deferred())) return rc;
        std::vector<double> hist;
        bool bad = false;   // diverged or non-finite: the state is not kept
        // the attempt's V-cycles in one graph launch, the step control's tests on the device ...
        int stop = 0;
        const auto t0 = std::chrono::steady_clock::now();
        rc = s->loop_attempt(tol, max_cycles, hist, stop);
        if (int rb = s->finish_begin()) return rb;   // a non-finite reference norm ends the step
        if (rc != MG_ERR_STATE || !hist.empty()) {
            const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            for (size_t k = 0; k < hist.size(); ++k)
                log_cycle(step0, attempt, (int)k + 1, hist[k], s->params().tau, ms / (double)hist.size());
            total += (int)hist.size();
            if (!hist.empty()) r = hist.back();
            if (rc == MG_ERR_DIVERGED || rc == MG_ERR_NAN) {
                if (!control) return rc;
                bad = true;
            } else if (rc) {
                return rc;
            }
            ok = stop == 1;   // (without the step control the loop ends only at tol or the cap)
        } else {
            // ... or one V-cycle per launch with the tests on the host
            for (int j = 1; j <= max_cycles; ++j) {
                const auto t1 = std::chrono::steady_clock::now();
                rc = s->vcycle(&r);
                ++total;
                log_cycle(step0, attempt, j, r, s->params().tau,
                          std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t1).count());
                if (rc == MG_ERR_DIVERGED || rc == MG_ERR_NAN) {
                    if (!control) return rc;
                    bad = true;
                    break;
                }
                if (rc) return rc;
                hist.push_back(r);
                if (r <= tol) { ok = true; break; }
                if (control && attempt_stalled(hist, s->params().stall_ratio)) break;
            }
        }
        if (ok || !control) break;
        const double tau = s->params().tau;
        if (attempt >= s->params().max_halvings || !(tau > 0)) {
            if (bad && (rc = s->restart_step(tau))) return rc;   // keep phi^n, not a diverged state
            if (bad && (rc = s->begin_step(nullptr))) return rc;
            break;
        }
        if ((rc = s->restart_step(0.5 * tau))) return rc;
    }
    s->set_cycles_step(total);
    if (cycles) *cycles = total;
    if (rho) *rho = r;
    if ((rc = s->end_step(nullptr))) return rc;
    return ok ? MG_OK : fail(MG_ERR_TIMEOUT, "no attempt at the step reached the tolerance");
}

int check_markers(const double *mk, int k, int n, int m) {
    if (!mk || k < 1) return fail(MG_ERR_ARG, "at least one marker is required");
    for (int q = 0; q < k; ++q) {
        double x = mk[2 * q], y = mk[2 * q + 1];
        if (!std::isfinite(x) || !std::isfinite(y) || x < 0 || y < 0 || x > m - 1 || y > n - 1)
            return fail(MG_ERR_ARG, "marker outside the image");
    }
    return MG_OK;
}

}  // namespace

struct mg_handle_s {
    SolverBase *s;
};

namespace {

// ---------------------------------------------------------------------------------------
// Batched solves: many images, one CUDA graph per V-cycle whose branches are the images.
// Each branch is a conditional node: a one-thread kernel sets its condition from the image's
// last residual norm, so images that have reached the tolerance are skipped on the device.
// ---------------------------------------------------------------------------------------
__global__ void k_batch_cond(cudaGraphConditionalHandle h, const Scalars *sc, double tol2) {
    const double n2 = sc->norm2, n0 = sc->norm2_0;
    cudaGraphSetConditional(h, (n2 > tol2 * n0 && sc->halt == 0) ? 1u : 0u);
}

__global__ void k_batch_gather(Scalars *const *sc, int count, double *out) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        out[3 * i] = sc[i]->norm2;
        out[3 * i + 1] = sc[i]->norm2_0;
        out[3 * i + 2] = (double)sc[i]->err;
    }
}

struct Batch {
    std::vector<Solver<float> *> s;
    std::vector<mg_handle_s *> h;
    std::vector<long long> nodes;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    Scalars **d_sc = nullptr;
    double *d_out = nullptr, *h_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    double tol_baked = -1.0;
    std::vector<long long> epochs;   // each image's graph_epoch when the batch graph was built
    int tuned_shape = -2;            // mg_batch_autotune: -1 per-image shapes, 0..5 one shape, -2 not run

    ~Batch() {
        if (st) cudaStreamSynchronize(st);
        if (exec) cudaGraphExecDestroy(exec);
        for (auto *x : s) delete x;
        for (auto *x : h) delete x;
        if (d_sc) cudaFree(d_sc);
        if (d_out) cudaFree(d_out);
        if (h_out) cudaFreeHost(h_out);
        if (own_stream && st) cudaStreamDestroy(st);
    }

    int build(double tol) {
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        const int count = (int)s.size();
        cudaGraph_t B;
        CK(cudaGraphCreate(&B, 0));
        std::vector<cudaGraphNode_t> ends;
        nodes.assign(count, 0);
        int rc = MG_OK;
        double tol2 = tol * tol;
        for (int i = 0; i < count && rc == MG_OK; ++i) {
            cudaGraph_t gi;
            if ((rc = s[i]->capture_vcycle(&gi, &nodes[i]))) break;
            cudaGraphConditionalHandle hc;
            cudaError_t e = cudaGraphConditionalHandleCreate(&hc, B, 0, cudaGraphCondAssignDefault);
            cudaGraphNode_t kn = nullptr, cn = nullptr, child = nullptr;
            if (e == cudaSuccess) {
                const Scalars *sc = s[i]->dsc;
                void *args[] = {&hc, (void *)&sc, &tol2};
                cudaKernelNodeParams kp = {};
                kp.func = (void *)k_batch_cond;
                kp.gridDim = dim3(1);
                kp.blockDim = dim3(1);
                kp.kernelParams = args;
                e = cudaGraphAddKernelNode(&kn, B, nullptr, 0, &kp);
            }
            if (e == cudaSuccess) {
                cudaGraphNodeParams cp = {};
                cp.type = cudaGraphNodeTypeConditional;
                cp.conditional.handle = hc;
                cp.conditional.type = cudaGraphCondTypeIf;
                cp.conditional.size = 1;
                e = cudaGraphAddNode(&cn, B, &kn, nullptr, 1, &cp);
                if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&child, cp.conditional.phGraph_out[0], nullptr, 0, gi);
            }
            cudaGraphDestroy(gi);
            if (e != cudaSuccess) rc = fail(MG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
            else ends.push_back(cn);
        }
        if (rc == MG_OK) {
            cudaGraphNode_t gn, mn;
            int cnt = count;
            void *args[] = {(void *)&d_sc, &cnt, (void *)&d_out};
            cudaKernelNodeParams kp = {};
            kp.func = (void *)k_batch_gather;
            kp.gridDim = dim3(1);
            kp.blockDim = dim3(256);
            kp.kernelParams = args;
            cudaError_t e = cudaGraphAddKernelNode(&gn, B, ends.data(), ends.size(), &kp);
            if (e == cudaSuccess)
                e = cudaGraphAddMemcpyNode1D(&mn, B, &gn, 1, h_out, d_out, sizeof(double) * 3 * count, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, B, 0);
            if (e != cudaSuccess) { exec = nullptr; rc = fail(MG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e)); }
        }
        cudaGraphDestroy(B);
        if (rc == MG_OK) {
            tol_baked = tol;
            epochs.resize(count);
            for (int i = 0; i < count; ++i) epochs[i] = s[i]->graph_epoch;
        }
        return rc;
    }

    // Tile shapes for the batch as a whole: the per-image choices of mg_autotune, and each tile
    // shape on every grid of every image, each timed as `reps` launches of the batch graph (every
    // image running: tolerance 0) from the images' phi^n; keeps the fastest.  The images' state
    // is restored (phi = phi^n); a step is left begun, as after mg_autotune.
    int autotune(int reps) {
        const int count = (int)s.size();
        std::vector<std::vector<int>> own(count);
        for (int i = 0; i < count; ++i) {
            int rc = s[i]->begin_step(nullptr);
            if (!rc) rc = s[i]->autotune(reps, nullptr);
            if (rc) return rc;
            own[i].assign(s[i]->shape, s[i]->shape + kMaxLevels);
        }
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        float best = 1e30f;
        int best_c = -1;
        int rc = MG_OK;
        for (int c = -1; c < kTileShapes && rc == MG_OK; ++c) {   // -1: the per-image choices
            for (int i = 0; i < count && rc == MG_OK; ++i) {
                std::vector<int> sh(kMaxLevels, c);
                rc = s[i]->set_shapes(c < 0 ? own[i].data() : sh.data());
                if (!rc) rc = s[i]->begin_step(nullptr);
            }
            if (rc || (rc = build(0.0))) break;
            float t = 0;
            for (int warm = 0; warm < 2 && rc == MG_OK; ++warm) {
                if (cudaEventRecord(e0, st) != cudaSuccess) rc = fail(MG_ERR_CUDA, "event");
                for (int r = 0; r < reps && rc == MG_OK; ++r)
                    if (cudaGraphLaunch(exec, st) != cudaSuccess) rc = fail(MG_ERR_CUDA, "graph launch");
                if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                    rc = fail(MG_ERR_CUDA, "event");
                cudaEventElapsedTime(&t, e0, e1);
            }
            for (int i = 0; i < count && rc == MG_OK; ++i) rc = s[i]->zero_increment();
            if (rc == MG_OK && t < best) { best = t; best_c = c; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        for (int i = 0; i < count && rc == MG_OK; ++i) {
            std::vector<int> sh(kMaxLevels, best_c);
            rc = s[i]->set_shapes(best_c < 0 ? own[i].data() : sh.data());
            if (!rc) rc = s[i]->begin_step(nullptr);
        }
        tuned_shape = best_c;
        if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
        return rc;
    }

    // One pseudo-time step of every image.  Each graph launch runs one V-cycle of every image
    // that has not reached tol.  The step control of mg_solve_step applies per image, in rounds:
    // an image whose attempt stalls, diverges or reaches max_cycles V-cycles is halted on the
    // device; once no image is left running, the halted ones restart from their phi^n with
    // tau / 2 together (one rebuild of the batch graph per round).
    int solve_step(double tol, int max_cycles, int *cycles, double *rho) {
        const int count = (int)s.size();
        for (int i = 0; i < count; ++i) {
            int rc = s[i]->begin_step(nullptr);
            if (rc) return rc;
        }
        bool stale = !exec || tol != tol_baked || (int)epochs.size() != count;
        for (int i = 0; i < count && !stale; ++i) stale = s[i]->graph_epoch != epochs[i];
        if (stale) {
            int rc = build(tol);
            if (rc) return rc;
        }
        std::vector<int> cyc(count, 0), halvings(count, 0);
        std::vector<double> r(count, 1.0);
        std::vector<std::vector<double>> hist(count);
        std::vector<char> active(count, 1), failed(count, 0), restart(count, 0);
        int rc = MG_OK;
        for (;;) {
            bool any = true;
            while (any && rc == MG_OK) {
                CK(cudaGraphLaunch(exec, st));
                CK(cudaStreamSynchronize(st));
                any = false;
                for (int i = 0; i < count; ++i) {
                    if (!active[i]) continue;
                    const double n2 = h_out[3 * i], n0 = h_out[3 * i + 1];
                    ++cyc[i];
                    s[i]->cycles_step = cyc[i];
                    ++s[i]->cycles_total;
                    s[i]->launches += nodes[i] + 1;
                    r[i] = n0 > 0 ? std::sqrt(n2) / std::sqrt(n0) : std::sqrt(n2);   // as mg_vcycle
                    s[i]->rho = r[i];
                    const int err = (int)h_out[3 * i + 2];
                    if ((err & 1) && rc == MG_OK) rc = fail(MG_ERR_NOT_SPD, "coarsest Cholesky: non-positive pivot");
                    if ((err & 4) && rc == MG_OK) {
                        CK(cudaMemsetAsync(&s[i]->dsc->err, 0, sizeof(int), st));
                        rc = fail(MG_ERR_TIMEOUT, "a tile copy into shared memory did not complete within the wait limit");
                    }
                    hist[i].push_back(r[i]);
                    if (r[i] <= tol) { active[i] = 0; continue; }
                    const mg_params &pi = s[i]->p;
                    const bool control = pi.stall_ratio > 0;
                    const bool bad = !std::isfinite(r[i]) || r[i] > 1e3;
                    const bool capped = (int)hist[i].size() >= max_cycles;
                    if (!control) {
                        if (!std::isfinite(r[i]) && rc == MG_OK) rc = fail(MG_ERR_NAN, "non-finite residual");
                        if (capped) failed[i] = 1;
                    } else if (bad || capped || attempt_stalled(hist[i], pi.stall_ratio)) {
                        if (halvings[i] >= pi.max_halvings) failed[i] = 1;
                        else restart[i] = 1;
                    }
                    if (failed[i] || restart[i]) {
                        active[i] = 0;
                        if (bad && failed[i] && rc == MG_OK && !(rc = s[i]->restart_step(pi.tau)))
                            rc = s[i]->begin_step(nullptr);   // keep phi^n, not a diverged state
                        CK(cudaMemsetAsync(&s[i]->dsc->halt, 1, sizeof(int), st));   // after any begin_step
                        continue;
                    }
                    any = true;
                }
            }
            if (rc) break;
            bool again = false;
            for (int i = 0; i < count && rc == MG_OK; ++i) {
                if (!restart[i]) continue;
                restart[i] = 0;
                ++halvings[i];
                hist[i].clear();
                if (!(rc = s[i]->restart_step(0.5 * s[i]->p.tau))) rc = s[i]->begin_step(nullptr);
                active[i] = 1;
                again = true;
            }
            if (rc || !again) break;
            if ((rc = build(tol))) break;
        }
        if (cycles) for (int i = 0; i < count; ++i) cycles[i] = cyc[i];
        if (rho) for (int i = 0; i < count; ++i) rho[i] = r[i];
        if (rc) return rc;
        for (int i = 0; i < count; ++i) {
            int e = s[i]->end_step(nullptr);
            if (e) return e;
        }
        for (int i = 0; i < count; ++i)
            if (failed[i]) return fail(MG_ERR_TIMEOUT, "an image reached no tolerance within its attempts");
        return MG_OK;
    }
};

}  // namespace

struct mg_batch_s {
    Batch b;
};

extern "C" {

int mg_default_params(mg_params *p, int n, int m) {
    if (!p) return fail(MG_ERR_ARG, "params is NULL");
    std::memset(p, 0, sizeof(*p));
    p->model = MG_MODEL_SC;
    p->mu = 1.0; p->lambda1 = 10.0; p->lambda2 = 10.0; p->theta = 1.0; p->nu = 1.0;
    p->eps = 1.0; p->beta = 1e-6; p->beta_edge = 1.0; p->sigma_blur = 1.0;
    p->sigma_d = 0.05 * std::max(n, m);
    p->Sigma = 2.0; p->tau = 1.0;
    p->nu1 = 2; p->nu2 = 2;
    int lev = 1, s = std::min(n, m);
    while (s / 2 >= 4 && lev < 12) { s /= 2; ++lev; }
    p->levels = lev;
    p->precision = MG_F32; p->smoother = MG_SMOOTH_FUSED;
    p->coarse_maxit = 100; p->coarse_tol = 1e-13; p->use_graph = 1;
    p->coarse_solver = MG_COARSE_PICARD; p->aos_dt = 10.0;
    p->stall_ratio = 0.6; p->max_halvings = 10;
    return MG_OK;
}

int mg_setup(mg_handle *out, const void *image, int n, int m, const double *markers_xy, int k,
             const mg_params *p, const mg_allocator *alloc, void *stream) {
    if (!out) return fail(MG_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_params(p, n, m);
    if (rc) return rc;
    if (!image) return fail(MG_ERR_ARG, "image is NULL");
    if ((rc = check_markers(markers_xy, k, n, m))) return rc;
    prepare_smoother_kernels();
    prepare_coarse_kernels();
    prepare_bottom_kernel();
    prepare_sweep_tma();
    prepare_snapshot_tma();
    prepare_residual_tma();
    prepare_learned_kernels();
    SolverBase *s = nullptr;
    if (p->precision != MG_F64) {
        auto *t = new Solver<float>();
        rc = t->init(n, m, *p, alloc, (cudaStream_t)stream, k);
        s = t;
    } else {
        auto *t = new Solver<double>();
        rc = t->init(n, m, *p, alloc, (cudaStream_t)stream, k);
        s = t;
    }
    if (!rc) rc = s->reset(image, markers_xy, k);
    if (rc) {
        std::string keep = g_err;
        delete s;
        g_err = keep;
        return rc;
    }
    *out = new mg_handle_s{s};
    return MG_OK;
}

int mg_reset(mg_handle h, const void *image, const double *markers_xy, int k) {
    if (!h || !image) return fail(MG_ERR_ARG, "NULL argument");
    int rc = check_markers(markers_xy, k, h->s->rows(), h->s->cols());
    if (rc) return rc;
    return h->s->reset(image, markers_xy, k);
}

int mg_begin_step(mg_handle h, double *res0) { return h ? h->s->begin_step(res0) : fail(MG_ERR_ARG, "NULL handle"); }
int mg_vcycle(mg_handle h, double *rho) { return h ? h->s->vcycle(rho) : fail(MG_ERR_ARG, "NULL handle"); }
int mg_end_step(mg_handle h, double *eta) { return h ? h->s->end_step(eta) : fail(MG_ERR_ARG, "NULL handle"); }

int mg_solve_step(mg_handle h, double tol, int max_cycles, int *cycles, double *rho) {
    if (!h || max_cycles < 1) return fail(MG_ERR_ARG, "NULL handle or max_cycles < 1");
    return solve_step_controlled(h->s, tol, max_cycles, cycles, rho);
}

int mg_solve(mg_handle h, double tol, int max_cycles, double eta_stop, int max_steps, int *steps) {
    if (!h || max_steps < 1) return fail(MG_ERR_ARG, "NULL handle or max_steps < 1");
    int taken = 0;
    for (; taken < max_steps;) {
        int rc = mg_solve_step(h, tol, max_cycles, nullptr, nullptr);
        ++taken;
        if (rc && rc != MG_ERR_TIMEOUT) { if (steps) *steps = taken; return rc; }
        if (h->s->last_eta() < eta_stop) break;
    }
    if (steps) *steps = taken;
    return MG_OK;
}

int mg_mask(mg_handle h, unsigned char *mask) {
    if (!h || !mask) return fail(MG_ERR_ARG, "NULL argument");
    return h->s->mask(mask);
}
int mg_get_phi(mg_handle h, void *phi) { return (h && phi) ? h->s->get_phi(phi) : fail(MG_ERR_ARG, "NULL argument"); }
int mg_set_phi(mg_handle h, const void *phi) { return (h && phi) ? h->s->set_phi(phi) : fail(MG_ERR_ARG, "NULL argument"); }
int mg_set_regions(mg_handle h, double c1, double c2) {
    if (!h || !std::isfinite(c1) || !std::isfinite(c2)) return fail(MG_ERR_ARG, "bad argument");
    return h->s->set_regions(c1, c2);
}
int mg_get_level(mg_handle h, int level, int field, void *out) {
    return (h && out) ? h->s->get_level(level, field, out) : fail(MG_ERR_ARG, "NULL argument");
}
int mg_get_stats(mg_handle h, mg_stats *s) { return (h && s) ? h->s->stats(s) : fail(MG_ERR_ARG, "NULL argument"); }
int mg_inject_divergence(mg_handle h, int cycle) {
    return h ? h->s->inject_divergence(cycle) : fail(MG_ERR_ARG, "NULL handle");
}
int mg_set_wait_limit(mg_handle h, long long rounds) {
    return h ? h->s->set_wait_limit(rounds) : fail(MG_ERR_ARG, "NULL handle");
}

#ifdef MG_DEBUG
namespace {
__global__ void k_debug_selftest(long long lim) { (void)MG_DBG_OK(lim + 5, lim, kDbgOther); }
}  // namespace
#endif

int mg_debug_selftest(void) {
#ifdef MG_DEBUG
    k_debug_selftest<<<1, 1>>>(1000);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
#endif
    return MG_OK;
}

int mg_debug_status(mg_debug_info *out, int clear) {
    if (!out) return fail(MG_ERR_ARG, "NULL argument");
    *out = mg_debug_info{};
    out->first_site = -1;
#ifdef MG_DEBUG
    out->enabled = 1;
    CK(cudaDeviceSynchronize());
    for (auto rd : segmg::debug_readers()) {
        unsigned long long w[4] = {0, 0, 0, 0};
        if (rd(w, clear) != 0) return fail(MG_ERR_CUDA, "reading the debug words");
        out->sites |= w[0];
        if (out->first_site < 0 && w[2] != 0) {
            out->first_site = (int)w[2] - 1;
            out->first_index = (long long)w[1];
        }
        out->count += (long long)w[3];
    }
#else
    (void)clear;
#endif
    return MG_OK;
}

namespace {

// The context of mg_segment_host kept between calls: the handle, its device buffers and stream,
// for the size, parameters and device of the last call (one per process, under a lock).
struct HostContext {
    std::mutex mu;
    int dev = -1, n = 0, m = 0, kcap = 0;
    mg_params q{};
    mg_handle h = nullptr;
    float *dimg = nullptr, *dphi = nullptr;
    unsigned char *dmask = nullptr;
    cudaStream_t st = nullptr;
    void release() {
        if (h) mg_destroy(h);
        if (dimg) cudaFree(dimg);
        if (dmask) cudaFree(dmask);
        if (dphi) cudaFree(dphi);
        if (st) cudaStreamDestroy(st);
        h = nullptr; dimg = nullptr; dmask = nullptr; dphi = nullptr; st = nullptr;
        dev = -1; n = m = kcap = 0;
    }
};
HostContext &host_context() {
    static HostContext *c = new HostContext();   // never destroyed: no CUDA calls at process exit
    return *c;
}

}  // namespace

int mg_segment_host(const float *image_host, int n, int m, const double *markers_xy, int k,
                    const mg_params *p, double tol, int max_cycles, double eta_stop, int max_steps,
                    unsigned char *mask_host, float *phi_host, mg_stats *stats) {
    if (!image_host || !mask_host || !p) return fail(MG_ERR_ARG, "NULL argument");
    mg_params q = *p;
    if (q.precision == MG_F64) q.precision = MG_F32;
    int rc = check_params(&q, n, m);
    if (rc) return rc;
    if ((rc = check_markers(markers_xy, k, n, m))) return rc;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    HostContext &c = host_context();
    std::lock_guard<std::mutex> lock(c.mu);
    const size_t N = (size_t)n * m;
    const bool same = c.h && c.dev == dev && c.n == n && c.m == m && k <= c.kcap &&
                      std::memcmp(&c.q, &q, sizeof(mg_params)) == 0;
    if (!same) c.release();
    cudaError_t e = cudaSuccess;
    if (!c.st) e = cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking);
    if (e == cudaSuccess && !c.dimg) e = cudaMalloc(&c.dimg, N * sizeof(float));
    if (e == cudaSuccess && !c.dmask) e = cudaMalloc(&c.dmask, N);
    if (e == cudaSuccess && phi_host && !c.dphi) e = cudaMalloc(&c.dphi, N * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.dimg, image_host, N * sizeof(float), cudaMemcpyHostToDevice, c.st);
    if (e != cudaSuccess) {
        c.release();
        return fail(e == cudaErrorMemoryAllocation ? MG_ERR_NOMEM : MG_ERR_CUDA, cudaGetErrorString(e));
    }
    if (same) {
        rc = mg_reset(c.h, c.dimg, markers_xy, k);
    } else {
        rc = mg_setup(&c.h, c.dimg, n, m, markers_xy, k, &q, nullptr, c.st);
        if (!rc) {
            c.dev = dev; c.n = n; c.m = m; c.kcap = std::max(k, 16); c.q = q;
        }
    }
    if (!rc) rc = mg_solve(c.h, tol, max_cycles, eta_stop, max_steps, nullptr);
    if (!rc) rc = c.h->s->mask_async(c.dmask);   // on the handle's stream: ordered before the copies below
    if (!rc && phi_host) rc = mg_get_phi(c.h, c.dphi);
    if (!rc) {
        e = cudaMemcpyAsync(mask_host, c.dmask, N, cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess && phi_host)
            e = cudaMemcpyAsync(phi_host, c.dphi, N * sizeof(float), cudaMemcpyDeviceToHost, c.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
        if (e != cudaSuccess) rc = fail(MG_ERR_CUDA, cudaGetErrorString(e));
    }
    if (!rc && stats) rc = mg_get_stats(c.h, stats);   // after the copies: the stream is idle by now
    if (rc) {   // a failed call keeps nothing
        std::string keep = g_err;
        c.release();
        g_err = keep;
    }
    return rc;
}

void mg_segment_host_release(void) {
    HostContext &c = host_context();
    std::lock_guard<std::mutex> lock(c.mu);
    c.release();
}

int mg_autotune(mg_handle h, int reps, int *shapes) {
    if (!h || reps < 1) return fail(MG_ERR_ARG, "NULL handle or reps < 1");
    return h->s->autotune(reps, shapes);
}

int mg_set_tile_shapes(mg_handle h, const int *shapes) {
    if (!h || !shapes) return fail(MG_ERR_ARG, "NULL argument");
    return h->s->set_shapes(shapes);
}

int mg_aos(mg_handle h, double dt, int max_iter, double eta, int *iters, double *rho) {
    if (!h) return fail(MG_ERR_ARG, "NULL handle");
    return h->s->aos(dt, max_iter, eta, iters, rho);
}

int mg_set_learned(mg_handle h, const float *theta, int mode, int refresh) {
    if (!h) return fail(MG_ERR_ARG, "NULL handle");
    return h->s->set_learned(theta, mode, refresh);
}

int mg_set_omega(mg_handle h, int level, const void *omega) {
    if (!h) return fail(MG_ERR_ARG, "NULL handle");
    return h->s->set_omega(level, omega);
}

int mg_learned_nparam(void) { return learned_nparam(); }

}  // extern "C"

struct mg_trainer_s {
    int cap = 0, count = 0, batch_max = 0, step = 0;
    int loss_kind = 0;   // mg_trainer_set_loss
    unsigned long long seed = 0;
    cudaStream_t st = nullptr;
    float *data = nullptr, *theta = nullptr, *mom = nullptr, *vel = nullptr, *grad = nullptr, *loss = nullptr;
    float *gmean = nullptr, *lmean = nullptr;
    int *idx = nullptr;
    std::mt19937_64 rng;
    ~mg_trainer_s() {
        if (st) cudaStreamSynchronize(st);
        for (void *q : {(void *)data, (void *)theta, (void *)mom, (void *)vel, (void *)grad, (void *)loss,
                        (void *)gmean, (void *)lmean, (void *)idx})
            if (q) cudaFree(q);
        if (st) cudaStreamDestroy(st);
    }
};

extern "C" {

int mg_trainer_create(mg_trainer *out, int capacity, int batch_max, unsigned long long seed, const float *theta0) {
    if (!out || capacity < 1 || batch_max < 1) return fail(MG_ERR_ARG, "NULL out, capacity < 1 or batch_max < 1");
    *out = nullptr;
    prepare_learned_kernels();
    auto *t = new mg_trainer_s();
    t->cap = capacity; t->batch_max = batch_max; t->seed = seed; t->rng.seed(seed);
    const int np = learned_nparam();
    const size_t rec = learned_record_floats();
    cudaError_t e = cudaStreamCreateWithFlags(&t->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&t->data, sizeof(float) * rec * capacity);
    if (e == cudaSuccess) e = cudaMalloc(&t->theta, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&t->mom, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&t->vel, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&t->grad, sizeof(float) * np * (size_t)batch_max);
    if (e == cudaSuccess) e = cudaMalloc(&t->loss, sizeof(float) * batch_max);
    if (e == cudaSuccess) e = cudaMalloc(&t->gmean, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMalloc(&t->lmean, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&t->idx, sizeof(int) * batch_max);
    if (e == cudaSuccess) e = cudaMemset(t->mom, 0, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaMemset(t->vel, 0, sizeof(float) * np);
    if (e != cudaSuccess) {
        delete t;
        return fail(e == cudaErrorMemoryAllocation ? MG_ERR_NOMEM : MG_ERR_CUDA, cudaGetErrorString(e));
    }
    std::vector<float> th(np, 0.f);
    if (theta0) {
        std::copy(theta0, theta0 + np, th.begin());
    } else {
        // He-normal hidden layers, zero output layer and biases: omega = 2 sigmoid(0) = 1 at the
        // start, the plain smoother
        std::normal_distribution<float> nd(0.f, 1.f);
        const float s1 = std::sqrt(2.f / 45.f), s2 = std::sqrt(2.f / 144.f);
        for (int k = 0; k < 720; ++k) th[k] = s1 * nd(t->rng);
        for (int k = 736; k < 3040; ++k) th[k] = s2 * nd(t->rng);
    }
    if (cudaMemcpy(t->theta, th.data(), sizeof(float) * np, cudaMemcpyHostToDevice) != cudaSuccess) {
        delete t;
        return fail(MG_ERR_CUDA, "parameter upload");
    }
    *out = t;
    return MG_OK;
}

int mg_trainer_record(mg_trainer t, mg_handle h, int count) {
    if (!t || !h || count < 1) return fail(MG_ERR_ARG, "NULL argument or count < 1");
    count = std::min(count, t->cap - t->count);
    if (count <= 0) return MG_OK;
    int rc = h->s->record_crops(t->data, t->count, count, t->rng());
    if (!rc) t->count += count;
    return rc;
}

int mg_trainer_load(mg_trainer t, const float *records, int count) {
    if (!t || !records || count < 1 || t->count + count > t->cap) return fail(MG_ERR_ARG, "NULL argument or capacity");
    const size_t rec = learned_record_floats();
    cudaError_t e = cudaMemcpy(t->data + rec * t->count, records, sizeof(float) * rec * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, cudaGetErrorString(e));
    t->count += count;
    return MG_OK;
}

int mg_trainer_count(mg_trainer t) { return t ? t->count : 0; }

int mg_trainer_set_loss(mg_trainer t, int kind) {
    if (!t || kind < 0 || kind > 1) return fail(MG_ERR_ARG, "NULL trainer or loss kind not 0 / 1");
    t->loss_kind = kind;
    return MG_OK;
}

// One batch: mean loss and gradient over the given crops; with lr > 0 also the Adam step.
static int trainer_batch(mg_trainer t, const int *idx, int batch, double lr, double *loss_out, float *grad_out) {
    if (cudaMemcpyAsync(t->idx, idx, sizeof(int) * batch, cudaMemcpyHostToDevice, t->st) != cudaSuccess)
        return fail(MG_ERR_CUDA, "index upload");
    if (lr > 0) ++t->step;
    launch_train_step(t->theta, t->mom, t->vel, t->data, t->idx, batch, t->grad, t->loss, t->gmean, t->lmean,
                      (float)lr, lr > 0 ? t->step : 0, t->loss_kind, t->st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, cudaGetErrorString(e));
    float l = 0.f;
    e = cudaMemcpyAsync(&l, t->lmean, sizeof(float), cudaMemcpyDeviceToHost, t->st);
    if (e == cudaSuccess && grad_out)
        e = cudaMemcpyAsync(grad_out, t->gmean, sizeof(float) * learned_nparam(), cudaMemcpyDeviceToHost, t->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(t->st);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, cudaGetErrorString(e));
    if (loss_out) *loss_out = l;
    return MG_OK;
}

int mg_trainer_grad(mg_trainer t, const int *idx, int batch, float *grad, double *loss) {
    if (!t || !idx || batch < 1 || batch > t->batch_max) return fail(MG_ERR_ARG, "NULL argument or batch");
    for (int k = 0; k < batch; ++k)
        if (idx[k] < 0 || idx[k] >= t->count) return fail(MG_ERR_ARG, "crop index out of range");
    return trainer_batch(t, idx, batch, 0.0, loss, grad);
}

int mg_trainer_train(mg_trainer t, int iters, int batch, double lr, double *loss) {
    if (!t || iters < 1 || batch < 1 || batch > t->batch_max || !(lr > 0) || t->count < 1)
        return fail(MG_ERR_ARG, "NULL trainer, iters / batch / lr out of range or no crops");
    std::vector<int> idx(batch);
    double l = 0.0;
    for (int it = 0; it < iters; ++it) {
        for (int k = 0; k < batch; ++k) idx[k] = (int)(t->rng() % (unsigned long long)t->count);
        int rc = trainer_batch(t, idx.data(), batch, lr, &l, nullptr);
        if (rc) return rc;
    }
    if (loss) *loss = l;
    return MG_OK;
}

int mg_trainer_get(mg_trainer t, float *theta) {
    if (!t || !theta) return fail(MG_ERR_ARG, "NULL argument");
    cudaError_t e = cudaMemcpy(theta, t->theta, sizeof(float) * learned_nparam(), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MG_OK : fail(MG_ERR_CUDA, cudaGetErrorString(e));
}

void mg_trainer_destroy(mg_trainer t) { delete t; }

int mg_energy(mg_handle h, double *E) {
    if (!h || !E) return fail(MG_ERR_ARG, "NULL argument");
    return h->s->energy(E);
}

int mg_set_bottom_kernel(mg_handle h, int enable, int *first_level) {
    if (!h || (enable != 0 && enable != 1)) return fail(MG_ERR_ARG, "NULL handle or enable not 0/1");
    int lb = h->s->set_bottom(enable);
    if (first_level) *first_level = lb;
    return MG_OK;
}

int mg_set_bottom_level(mg_handle h, int level) {
    if (!h) return fail(MG_ERR_ARG, "NULL handle");
    return h->s->set_bottom_level(level);
}

int mg_set_cluster_level(mg_handle h, int level) {
    if (!h) return fail(MG_ERR_ARG, "NULL handle");
    return h->s->set_cluster_level(level);
}

int mg_batch_setup(mg_batch *out, int count, const void *const *images, const int *n, const int *m,
                   const double *const *markers, const int *k, const mg_params *params, void *stream) {
    if (!out) return fail(MG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (count < 1 || !images || !n || !m || !markers || !k || !params) return fail(MG_ERR_ARG, "NULL argument or count < 1");
    for (int i = 0; i < count; ++i) {
        int rc = check_params(&params[i], n[i], m[i]);
        if (rc) return rc;
        if (params[i].precision == MG_F64) return fail(MG_ERR_ARG, "batches take MG_F32 or MG_MIXED images");
        if (!images[i]) return fail(MG_ERR_ARG, "image is NULL");
        if ((rc = check_markers(markers[i], k[i], n[i], m[i]))) return rc;
    }
    prepare_smoother_kernels();
    prepare_coarse_kernels();
    prepare_bottom_kernel();
    prepare_sweep_tma();
    prepare_snapshot_tma();
    prepare_residual_tma();
    prepare_learned_kernels();
    auto *B = new mg_batch_s();
    Batch &b = B->b;
    int rc = MG_OK;
    if (stream) b.st = (cudaStream_t)stream;
    else if (cudaStreamCreateWithFlags(&b.st, cudaStreamNonBlocking) == cudaSuccess) b.own_stream = true;
    else rc = fail(MG_ERR_CUDA, "stream creation failed");
    for (int i = 0; i < count && rc == MG_OK; ++i) {
        auto *sv = new Solver<float>();
        b.s.push_back(sv);
        b.h.push_back(new mg_handle_s{sv});
        rc = sv->init(n[i], m[i], params[i], nullptr, b.st, k[i]);
        if (!rc) rc = sv->reset(images[i], markers[i], k[i]);
    }
    if (rc == MG_OK) {
        std::vector<Scalars *> ptrs;
        for (auto *x : b.s) ptrs.push_back(x->dsc);
        cudaError_t e = cudaMalloc(&b.d_sc, sizeof(Scalars *) * count);
        if (e == cudaSuccess) e = cudaMalloc(&b.d_out, sizeof(double) * 3 * count);
        if (e == cudaSuccess) e = cudaMallocHost(&b.h_out, sizeof(double) * 3 * count);
        if (e == cudaSuccess) e = cudaMemcpy(b.d_sc, ptrs.data(), sizeof(Scalars *) * count, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = fail(MG_ERR_CUDA, cudaGetErrorString(e));
    }
    if (rc) {
        std::string keep = g_err;
        delete B;
        g_err = keep;
        return rc;
    }
    *out = B;
    return MG_OK;
}

int mg_batch_solve_step(mg_batch b, double tol, int max_cycles, int *cycles, double *rho) {
    if (!b || max_cycles < 1) return fail(MG_ERR_ARG, "NULL batch or max_cycles < 1");
    return b->b.solve_step(tol, max_cycles, cycles, rho);
}

int mg_batch_autotune(mg_batch b, int reps) {
    if (!b || reps < 1) return fail(MG_ERR_ARG, "NULL batch or reps < 1");
    return b->b.autotune(reps);
}

mg_handle mg_batch_handle(mg_batch b, int i) {
    if (!b || i < 0 || i >= (int)b->b.h.size()) return nullptr;
    return b->b.h[i];
}

void mg_batch_destroy(mg_batch b) { delete b; }

void mg_destroy(mg_handle h) {
    if (!h) return;
    delete h->s;
    delete h;
}

void *mg_get_stream(mg_handle h) { return h ? (void *)h->s->stream() : nullptr; }

int mg_time_kernels(mg_handle h, int level, int reps, double *ms) {
    return (h && ms) ? h->s->time_kernels(level, reps, ms) : fail(MG_ERR_ARG, "NULL argument");
}

int mg_time_residuals(mg_handle h, int level, int reps, double *ms) {
    return (h && ms) ? h->s->time_residuals(level, reps, ms) : fail(MG_ERR_ARG, "NULL argument");
}

int mg_time_sweeps_graph(mg_handle h, int level, int reps, double *ms) {
    return (h && ms) ? h->s->time_sweeps_graph(level, reps, ms) : fail(MG_ERR_ARG, "NULL argument");
}

const char *mg_strerror(int code) {
    switch (code) {
        case MG_OK: return "ok";
        case MG_ERR_ARG: return "invalid argument";
        case MG_ERR_NAN: return "non-finite value";
        case MG_ERR_CUDA: return "CUDA error";
        case MG_ERR_DIVERGED: return "diverged";
        case MG_ERR_TIMEOUT: return "iteration cap reached";
        case MG_ERR_NOT_SPD: return "coarsest system not positive definite";
        case MG_ERR_NOMEM: return "out of device memory";
        case MG_ERR_STATE: return "call out of order";
        default: return "unknown error";
    }
}

const char *mg_last_error(void) { return g_err.c_str(); }

}  // extern "C"
