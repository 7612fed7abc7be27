// sweep_tma.cu -- the fused Hybrid Smoother 2 sweep (Sec. 4.3) for FP32 storage, with the tiles
// staged into shared memory by the Tensor Memory Accelerator.
//
// Same sweep, same tiles and the same per-cell operations as k_sweep in smooth_kernels.cu (the
// results are bitwise identical); what changes is how tiles reach shared memory:
//   - persistent blocks: each block walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...;
//   - the u, G and f boxes of a tile (output tile plus a 4-cell halo, zero outside the grid)
//     are copied by three cp.async.bulk.tensor loads issued by one thread, completing on an
//     mbarrier;
//   - two stages: while a block smooths one tile, the next tile's boxes are in flight.
// Shared memory holds the boxes dense (row-major, as TMA writes them).  The checkerboard phases
// interleave two rows across the lanes of a warp (lane 2k: row a, lane 2k+1: row a+1), so the
// 32 cells a warp updates fall in 32 different banks without the colour-split layout the
// vector-load kernel uses.
//
// Every wait on an mbarrier is bounded (wait_limit try_wait rounds, a launch argument: the
// handle's mg_set_wait_limit, default kDefaultWaitLimit).  On time-out the block records bit 4 in
// the handle's error word, waits (bounded by kDrainLimit) for its copies still in flight and
// returns; the host reports it.
#include <cuda.h>

#include <algorithm>

#include "arith.cuh"
#include "line_phase.cuh"
#include "tma.cuh"

namespace segmg {

namespace {

constexpr int kH = 4;
constexpr long long kDrainLimit = 1LL << 22;   // try_wait rounds of the last wait for copies in flight

template <int OH_, int OW_, int NT_, int MINB_ = 1, bool ONE_ = false>
struct TShape {
    static constexpr int OH = OH_, OW = OW_, NT = NT_;
    static constexpr int MinBlocks = MINB_;   // resident blocks per SM asked of the compiler
    static constexpr bool OneTile = ONE_;     // always one tile per block (one stage), any grid size
    static constexpr int RH = OH + 2 * kH, RW = OW + 2 * kH;
    static constexpr int RowPieces = OW / 32 + 2, ColPieces = OH / 32 + 2;
    static constexpr int MkLines = RH > RW ? RH : RW, MkPieces = RowPieces > ColPieces ? RowPieces : ColPieces;
    static constexpr int BoxBytes = RH * RW * 4;
};
// 6 blocks of 256 threads per SM (at most 42 registers), one tile and one stage per block: the
// register limit, not shared memory, is what bounds the resident blocks, and six blocks each
// waiting on their own copies hide more latency than three double-buffered persistent ones
// (8192^2: 0.28 -> 0.24 ms per sweep)
using TT0 = TShape<32, 64, 256, 6, true>;
using TT1 = TShape<32, 32, 128>;
using TT2 = TShape<64, 64, 512, 2>;   // 512-thread shapes: at most 64 registers, two blocks per SM
using TT3 = TShape<32, 64, 512, 2>;
// 8 blocks of 256 threads per SM (at most 32 registers): every 32 x 32 tile of a 1024^2 grid
// then has its own resident block, one stage and no persistent loop
using TT4 = TShape<32, 32, 256, 8>;
// at most 64 registers: two blocks per SM for every sweep direction, so that every tile of a 512^2
// grid gets its own block (sweep D's code otherwise took more registers than A to C, fitting
// one block per SM and running persistent: 7.0 against 5.4 us per launch)
using TT5 = TShape<32, 32, 512, 2>;

template <typename TS, int STAGES>
struct TmaSmem {
    float box[STAGES][3][TS::RH][TS::RW];      // [stage][u, G, f][row][column]
    uint32_t mk[TS::MkLines][TS::MkPieces];    // member masks of the tile (as k_sweep)
    unsigned long long bar[STAGES];            // one mbarrier per stage
};


template <typename TS, int STAGES, bool ROWWISE>
__device__ __forceinline__ bool member(const TmaSmem<TS, STAGES> &S, int a, int b) {
    if (ROWWISE) return (S.mk[a][(b + 28) >> 5] >> ((b - kH) & 31)) & 1u;
    return (S.mk[b][(a + 28) >> 5] >> ((a - kH) & 31)) & 1u;
}

// One checkerboard phase over the box cells within distance 3 - ph of the output tile (the
// cells and the operations of rb_phase in smooth_kernels.cu).
// MEMBERS = false: no line piece that crosses the box has a member cell, so no cell is skipped.
template <typename TS, int STAGES, int SWEEP, bool INTERIOR, bool WEIGHTED, bool MEMBERS = true>
__device__ __forceinline__ void rb_phase(TmaSmem<TS, STAGES> &S, int st, const LevelView<float> &L, int ph, int i0,
                                         int j0) {
    constexpr int kRH = TS::RH, kRW = TS::RW;
    constexpr bool rev = (SWEEP & 1) != 0;
    float (*u)[kRW] = S.box[st][0];
    const float (*G)[kRW] = S.box[st][1];
    const float (*f)[kRW] = S.box[st][2];
    const int colour = rev ? 1 - ph : ph, lo = 1 + ph;
    const int n = L.n, m = L.m;
    const float c2 = L.cdiff * 0.5f;   // with face2 (see arith.cuh)
    for (int q = threadIdx.x; q < (kRH / 2) * kRW; q += TS::NT) {
        const int pr = q / kRW, e = q - pr * kRW;
        const int a = 2 * pr + (e & 1), b = (e & ~1) + ((a + colour) & 1);
        if (a < lo || a >= kRH - lo || b < lo || b >= kRW - lo) continue;
        bool hS = true, hN = true, hE = true, hW = true;
        if (!INTERIOR) {
            const int gi = i0 - kH + a, gj = j0 - kH + b;
            if (gi < 0 || gi >= n || gj < 0 || gj >= m) continue;
            hS = gi + 1 < n; hN = gi > 0; hE = gj + 1 < m; hW = gj > 0;
        }
        if (MEMBERS && member<TS, STAGES, (SWEEP < 2)>(S, a, b)) continue;
        const float gc = G[a][b];
        const float sS = face2(gc, G[a + 1][b], hS), sN = face2(gc, G[a - 1][b], hN);
        const float sE = face2(gc, G[a][b + 1], hE), sW = face2(gc, G[a][b - 1], hW);
        float v = point_relax(c2, L.inv_tau, sS, sN, sE, sW, u[a + 1][b], u[a - 1][b], u[a][b + 1], u[a][b - 1],
                              f[a][b]);
        if (WEIGHTED) {
            const size_t o = (size_t)(i0 - kH + a) * L.pitch + (j0 - kH + b);
            v = relax_weighted(ldc(L.omega, o, (size_t)L.n * L.pitch, kDbgSweep), v, u[a][b]);
        }
        u[a][b] = v;
    }
}

// STAGES = 2: persistent blocks, the next tile's copies in flight while a tile is smoothed;
// STAGES = 1: one box set per block (half the shared memory, more blocks per SM), used when every
// tile of the grid gets its own resident block.
template <int SWEEP, typename TS, int STAGES>
__global__ void __launch_bounds__(TS::NT, TS::MinBlocks) k_sweep_tma(LevelView<float> L, const __grid_constant__ CUtensorMap tin,
                                                      const __grid_constant__ CUtensorMap tG,
                                                      const __grid_constant__ CUtensorMap tf, int *err,
                                                      long long wait_limit) {
    constexpr int kOH = TS::OH, kOW = TS::OW, kRH = TS::RH, kRW = TS::RW;
    constexpr int kRowPieces = TS::RowPieces, kColPieces = TS::ColPieces;
    constexpr bool rowwise = SWEEP < 2, rev = (SWEEP & 1) != 0;
    extern __shared__ unsigned char smem_raw[];
    TmaSmem<TS, STAGES> &S = *reinterpret_cast<TmaSmem<TS, STAGES> *>(
        smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127));   // boxes 128-byte aligned
    const int n = L.n, m = L.m, p = L.pitch;
    const int tid = threadIdx.x;
    const int ntx = (m + kOW - 1) / kOW, ntiles = ntx * ((n + kOH - 1) / kOH);
    float *uout = (SWEEP & 1) ? L.u : L.t;   // ping-pong (see k_sweep)
    // the member masks of every line piece that touches a tile's box (zero outside the grid):
    // loaded into registers ahead of use (the first tile's before the block's set-up, the next
    // tile's while a tile is smoothed), stored to shared memory when the tile starts
    constexpr int kMaskWords = rowwise ? kRH * kRowPieces : kRW * kColPieces;
    constexpr int kMaskPer = (kMaskWords + TS::NT - 1) / TS::NT;
    auto load_masks = [&](int t, uint32_t (&w)[kMaskPer]) {
        const int ty = t / ntx, tx = t - ty * ntx;
        const int i0 = ty * kOH, j0 = tx * kOW;
#pragma unroll
        for (int r = 0; r < kMaskPer; ++r) {
            const int q = tid + r * TS::NT;
            w[r] = 0;
            if (q >= kMaskWords || t >= ntiles) continue;
            if (rowwise) {
                const int a = q / kRowPieces, pc = q % kRowPieces;
                const int gi = i0 - kH + a, piece = (j0 >> 5) - 1 + pc;
                if (gi >= 0 && gi < n && piece >= 0 && piece < L.npm &&
                    MG_DBG_OK(((size_t)SWEEP * n + gi) * L.npm + piece, (size_t)2 * n * L.npm, kDbgMaskLoad))
                    w[r] = __ldg(L.mrow + ((size_t)SWEEP * n + gi) * L.npm + piece);
            } else {
                const int b = q / kColPieces, pc = q % kColPieces;
                const int gj = j0 - kH + b, piece = (i0 >> 5) - 1 + pc;
                if (gj >= 0 && gj < m && piece >= 0 && piece < L.npn &&
                    MG_DBG_OK(((size_t)(SWEEP - 2) * m + gj) * L.npn + piece, (size_t)2 * m * L.npn, kDbgMaskLoad))
                    w[r] = __ldg(L.mcol + ((size_t)(SWEEP - 2) * m + gj) * L.npn + piece);
            }
        }
    };
    // true: a piece the line phases solve has a member; anym: some staged piece has one
    auto store_masks = [&](const uint32_t (&w)[kMaskPer], bool &anym) {
        bool lm = false;
#pragma unroll
        for (int r = 0; r < kMaskPer; ++r) {
            const int q = tid + r * TS::NT;
            if (q >= kMaskWords) continue;
            anym |= w[r] != 0u;
            if (rowwise) {
                const int a = q / kRowPieces, pc = q % kRowPieces;
                S.mk[a][pc] = w[r];
                lm |= solves_word<kH, kOH, kOW, true>(a, pc, w[r]);
            } else {
                const int b = q / kColPieces, pc = q % kColPieces;
                S.mk[b][pc] = w[r];
                lm |= solves_word<kH, kOH, kOW, false>(b, pc, w[r]);
            }
        }
        return lm;
    };
    auto issue = [&](int tile, int stage) {   // one thread
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int x = tx * kOW - kH, y = ty * kOH - kH;
        fence_proxy_async();
        mbar_expect_tx(&S.bar[stage], 3u * TS::BoxBytes);
        tma_load(&S.box[stage][0][0][0], &tin, x, y, &S.bar[stage]);
        tma_load(&S.box[stage][1][0][0], &tG, x, y, &S.bar[stage]);
        tma_load(&S.box[stage][2][0][0], &tf, x, y, &S.bar[stage]);
    };
    int tile = blockIdx.x;
    uint32_t mw[kMaskPer];
    load_masks(tile, mw);
    if (tid == 0) {   // the thread that initialises the barriers issues the first tile's copies
        for (int k = 0; k < STAGES; ++k) mbar_init(&S.bar[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        if (tile < ntiles) issue(tile, 0);
    }
    __syncthreads();
    for (int k = 0; tile < ntiles; ++k, tile += gridDim.x) {
        const int st = STAGES == 2 ? (k & 1) : 0;
        const unsigned parity = STAGES == 2 ? (unsigned)((k >> 1) & 1) : (unsigned)(k & 1);
        const int next = tile + gridDim.x;
        if (STAGES == 2 && tid == 0 && next < ntiles) issue(next, st ^ 1);
        const int ty = tile / ntx, tx = tile - ty * ntx;
        const int i0 = ty * kOH, j0 = tx * kOW;
        bool anym = false;
        const bool lm = store_masks(mw, anym);
        load_masks(next, mw);   // in flight while this tile is smoothed (zeros past the last tile)
        const bool ok = mbar_wait(&S.bar[st], parity, wait_limit);
        if (__syncthreads_or(!ok)) {
            // a copy did not complete within wait_limit rounds: report, give the copies in flight a
            // last bounded wait (kDrainLimit rounds, so that none still writes into shared memory
            // once the block has ended), stop
            if (tid == 0) {
                atomicOr(err, 4);
                mbar_wait(&S.bar[st], parity, kDrainLimit);
                if (STAGES == 2 && next < ntiles) mbar_wait(&S.bar[st ^ 1], (unsigned)(((k + 1) >> 1) & 1), kDrainLimit);
            }
            __syncthreads();
            return;
        }
        const bool lines = __syncthreads_or(lm);
        const bool members = __syncthreads_or(anym);   // else the checkerboard skips no cell
        float (*u)[kRW] = S.box[st][0];
        const float (*G)[kRW] = S.box[st][1];
        const float (*f)[kRW] = S.box[st][2];
        // ---- checkerboard phases (distance 3 then 2 from the output tile)
        const bool interior = i0 - kH >= 0 && i0 - kH + kRH <= n && j0 - kH >= 0 && j0 - kH + kRW <= m;
#pragma unroll
        for (int ph = 0; ph < 2; ++ph) {
            if (L.omega) {
                if (interior) rb_phase<TS, STAGES, SWEEP, true, true>(S, st, L, ph, i0, j0);
                else rb_phase<TS, STAGES, SWEEP, false, true>(S, st, L, ph, i0, j0);
            } else {
                if (interior) {
                    if (members) rb_phase<TS, STAGES, SWEEP, true, false>(S, st, L, ph, i0, j0);
                    else rb_phase<TS, STAGES, SWEEP, true, false, false>(S, st, L, ph, i0, j0);
                } else {
                    rb_phase<TS, STAGES, SWEEP, false, false>(S, st, L, ph, i0, j0);
                }
            }
            __syncthreads();
        }
        // ---- partial-line phases (line_phase.cuh), skipped when no piece of the tile has a member
        if (lines)
            tile_line_phases<float, kH, kOH, kOW, TS::NT, rowwise, rev>(
                [&](int a, int b) -> float & { return u[a][b]; }, [&](int a, int b) { return G[a][b]; },
                [&](int a, int b) { return f[a][b]; }, [&](int li, int pc) { return S.mk[li][1 + pc]; }, i0, j0, n,
                m, L.cdiff, L.inv_tau);
        // ---- the output tile to uout (16-byte vectors; padding columns keep their box values)
        constexpr int NVO = kOW / 4;
        for (int q = tid; q < kOH * NVO; q += TS::NT) {
            const int a = kH + q / NVO, b0 = kH + (q % NVO) * 4;
            const int gi = i0 + q / NVO, gj = j0 + (q % NVO) * 4;
            if (gi >= n || gj >= p) continue;
            if (!MG_DBG_OK((size_t)gi * p + gj + 3, (size_t)n * p, kDbgSweep)) continue;
            *reinterpret_cast<float4 *>(uout + (size_t)gi * p + gj) = *reinterpret_cast<const float4 *>(&u[a][b0]);
        }
        __syncthreads();   // the stage is free for the next copy into it
        if (STAGES == 1 && tid == 0 && next < ntiles) issue(next, 0);
    }
}

template <int SW, typename TS, int STAGES>
size_t tma_smem() { return sizeof(TmaSmem<TS, STAGES>) + 128; }

// Resident blocks per SM of each instantiation (measured once at set-up, outside any capture).
template <int SW, typename TS, int STAGES>
int &tma_blocks_per_sm() {
    static int b = 1;
    return b;
}

template <int SW, typename TS, int STAGES>
void set_attr() {
    cudaFuncSetAttribute(k_sweep_tma<SW, TS, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tma_smem<SW, TS, STAGES>());
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_sweep_tma<SW, TS, STAGES>, TS::NT,
                                                      tma_smem<SW, TS, STAGES>()) != cudaSuccess || v < 1)
        v = 1;
    tma_blocks_per_sm<SW, TS, STAGES>() = v;
}

template <typename TS>
void set_attrs() {
    set_attr<0, TS, 1>(); set_attr<1, TS, 1>(); set_attr<2, TS, 1>(); set_attr<3, TS, 1>();
    set_attr<0, TS, 2>(); set_attr<1, TS, 2>(); set_attr<2, TS, 2>(); set_attr<3, TS, 2>();
}

// One tile per block (one stage) when the shape asks for it or when every tile gets a resident
// block with one stage; else persistent double-buffered blocks, as many as fit.
template <int SW, typename TS>
void launch_one(const LevelView<float> &L, const SweepMaps &M, int sms, int *err, long long wl, cudaStream_t st) {
    const int ntiles = ((L.m + TS::OW - 1) / TS::OW) * ((L.n + TS::OH - 1) / TS::OH);
    const CUtensorMap *in = reinterpret_cast<const CUtensorMap *>((SW & 1) ? M.t : M.u);
    const CUtensorMap &mG = *reinterpret_cast<const CUtensorMap *>(M.G);
    const CUtensorMap &mf = *reinterpret_cast<const CUtensorMap *>(M.f);
    if (TS::OneTile || ntiles <= sms * tma_blocks_per_sm<SW, TS, 1>()) {
        k_sweep_tma<SW, TS, 1><<<ntiles, TS::NT, tma_smem<SW, TS, 1>(), st>>>(L, *in, mG, mf, err, wl);
    } else {
        const int grid = std::min(ntiles, sms * tma_blocks_per_sm<SW, TS, 2>());
        k_sweep_tma<SW, TS, 2><<<grid, TS::NT, tma_smem<SW, TS, 2>(), st>>>(L, *in, mG, mf, err, wl);
    }
}

template <typename TS>
void launch_shape(const LevelView<float> &L, int sweep, const SweepMaps &M, int sms, int *err, long long wl,
                  cudaStream_t st) {
    switch (sweep) {
        case 0: launch_one<0, TS>(L, M, sms, err, wl, st); break;
        case 1: launch_one<1, TS>(L, M, sms, err, wl, st); break;
        case 2: launch_one<2, TS>(L, M, sms, err, wl, st); break;
        default: launch_one<3, TS>(L, M, sms, err, wl, st); break;
    }
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder() {
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

bool encode(void *out, float *base, int n, int m, int pitch, int RH, int RW) {
    return encode_map_2d(out, base, 4, n, m, pitch, RH, RW);
}

template <typename TS>
bool encode_shape(const LevelView<float> &L, SweepMaps &M) {
    return encode(M.u, L.u, L.n, L.m, L.pitch, TS::RH, TS::RW) && encode(M.t, L.t, L.n, L.m, L.pitch, TS::RH, TS::RW) &&
           encode(M.G, L.G, L.n, L.m, L.pitch, TS::RH, TS::RW) && encode(M.f, L.f, L.n, L.m, L.pitch, TS::RH, TS::RW);
}

int g_sms = 0;

}  // namespace

// One n x m grid function (FP32, elem = 4, or BF16, elem = 2) with row pitch `pitch` (elements) as
// a 2-D tensor, box RW x RH, zero fill outside.
bool encode_map_2d(void *out, void *base, int elem, int n, int m, int pitch, int RH, int RW) {
    EncodeFn fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * (cuuint64_t)elem};
    cuuint32_t box[2] = {(cuuint32_t)RW, (cuuint32_t)RH};
    cuuint32_t estr[2] = {1, 1};
    return fn(reinterpret_cast<CUtensorMap *>(out),
              elem == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides,
              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void prepare_sweep_tma() {
    set_attrs<TT0>(); set_attrs<TT1>(); set_attrs<TT2>(); set_attrs<TT3>(); set_attrs<TT4>(); set_attrs<TT5>();
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms < 1) g_sms = 1;
}

bool encode_sweep_maps(const LevelView<float> &L, int shape, SweepMaps *M) {
    if (shape == 1) return encode_shape<TT1>(L, *M);
    if (shape == 2) return encode_shape<TT2>(L, *M);
    if (shape == 3) return encode_shape<TT3>(L, *M);
    if (shape == 4) return encode_shape<TT4>(L, *M);
    if (shape == 5) return encode_shape<TT5>(L, *M);
    return encode_shape<TT0>(L, *M);
}

void launch_sweep_tma(const LevelView<float> &L, int sweep, int shape, const SweepMaps &M, int *err,
                      long long wait_limit, cudaStream_t st) {
    const long long wl = wait_limit;
    if (shape == 1) launch_shape<TT1>(L, sweep, M, g_sms, err, wl, st);
    else if (shape == 2) launch_shape<TT2>(L, sweep, M, g_sms, err, wl, st);
    else if (shape == 3) launch_shape<TT3>(L, sweep, M, g_sms, err, wl, st);
    else if (shape == 4) launch_shape<TT4>(L, sweep, M, g_sms, err, wl, st);
    else if (shape == 5) launch_shape<TT5>(L, sweep, M, g_sms, err, wl, st);
    else launch_shape<TT0>(L, sweep, M, g_sms, err, wl, st);
}

}  // namespace segmg
