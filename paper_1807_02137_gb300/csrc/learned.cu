// learned.cu -- learned per-cell relaxation weights for the point updates of Hybrid Smoother 2:
// inference (BF16 weights and activations on the tensor cores, FP32 accumulation) and training
// (FP32).
//
// The paper chooses its smoother cell by cell from the local coefficients (Sec. 4).  This
// extension learns a weight omega in (0, 2) for the point update phi += omega (g - phi) of every
// non-member cell from the same local stencil:
//   input, per cell, from its four face values a_X of G (X = S, N, E, W; zero on a boundary
//   face; the ratios equal those of the row-scaled coefficients):
//       x_k = a_X / sum_X a_X (k = 0..3),  x_4 = log(max a / min a over existing faces) / 8
//   three 3x3 convolutions, zero padding at the grid boundary: 5 -> 16 (ReLU) -> 16 (ReLU) -> 1,
//   omega = 2 sigmoid(z).
// Parameters (3201 floats): W1 (16,5,3,3), b1 (16), W2 (16,16,3,3), b2 (16), W3 (1,16,3,3), b3.
//
// Training: crops of 24 x 24 cells recorded from plain solves (row-scaled coefficients c_X,
// right-hand side f, state u, 1/tau, colour parity of the crop's origin).  Loss of a crop: one
// red and one black damped point update on the cells at least one cell inside, then 1/2 the
// mean of v^2 over the cells at least two inside, with v = r = f - (sum_X c_X u_X - S u),
// S = sum_X c_X + 1/tau (loss 0), or v = 4 r - (the sum of r at the four neighbours), the
// residual's high-frequency part, which the smoother of a multigrid cycle must remove (loss 1).  One block per crop computes the loss and its gradient by reverse mode;
// a second kernel averages the gradients over the batch in a fixed order and a third applies
// Adam.
#include <cuda_bf16.h>

#include "arith.cuh"
#include "reduce.cuh"

namespace segmg {

namespace {

constexpr int kCin = 5, kCh = 16;
constexpr int oW1 = 0, oB1 = 720, oW2 = 736, oB2 = 3040, oW3 = 3056, oB3 = 3200, kNP = 3201;

__device__ __forceinline__ void cell_features(float aS, float aN, float aE, float aW, float *x) {
    const float s = aS + aN + aE + aW;
    const float inv = s > 0.f ? 1.f / s : 0.f;
    x[0] = aS * inv; x[1] = aN * inv; x[2] = aE * inv; x[3] = aW * inv;
    float mx = 0.f, mn = 3.0e38f;
    const float a[4] = {aS, aN, aE, aW};
    for (int t = 0; t < 4; ++t)
        if (a[t] > 0.f) { mx = fmaxf(mx, a[t]); mn = fminf(mn, a[t]); }
    x[4] = (mx > 0.f && mn < 3.0e38f) ? logf(mx / mn) * 0.125f : 0.f;
}

// ---------------------------------------------------------------------------------------
// Inference: one 16 x 16 tile of omega per block (256 threads), all three layers in shared
// memory (features on the tile + 3 cells, layer 1 on + 2, layer 2 on + 1).  The two hidden
// convolutions run on the tensor cores as implicit GEMMs (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation): rows = the window's pixels (16 per MMA), columns = the 16 output
// channels (two n8 blocks), K = 9 taps x 16 input channels (one k16 step per tap; layer 1's
// 5 input channels padded with zeros).  Activations are stored channel-minor (16 BF16 = 32 bytes
// per pixel), so a fragment's pair of channels is one 32-bit word.  The output convolution
// (16 -> 1) runs on the CUDA cores.
// ---------------------------------------------------------------------------------------
struct InferSmem {
    float G[24][25];
    __nv_bfloat16 X[22][22][kCh];   // features, channels 5..15 zero
    __nv_bfloat16 A1[20][20][kCh];
    __nv_bfloat16 A2[18][18][kCh];
    float W[kNP];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t l = __bfloat16_as_ushort(__float2bfloat16(lo));
    const uint32_t h = __bfloat16_as_ushort(__float2bfloat16(hi));
    return l | (h << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// One hidden 3x3 convolution of the tile on the tensor cores: input IN (an IW x IW window of
// pixels, 16 channels each), output OUT (the (IW-2) x (IW-2) window inside it), weights Wt
// (o, cin, 3, 3) at S.W + wofs with cin input channels, bias at S.W + bofs, ReLU; pixels outside
// the grid (window origin gi0, gj0) get 0.  One warp per M-tile of 16 pixels.
template <int IW>
__device__ __forceinline__ void conv_tc(const InferSmem &S, const __nv_bfloat16 (*IN)[IW][kCh],
                                        __nv_bfloat16 (*OUT)[IW - 2][kCh], int wofs, int bofs, int cin,
                                        int gi0, int gj0, int n, int m) {
    constexpr int OW = IW - 2, NPIX = OW * OW, MT = (NPIX + 15) / 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
    // B fragments of the 9 taps and the two n8 blocks: k = input channel, n = output channel
    uint32_t bf[9][2][2];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int nb = 0; nb < 2; ++nb) {
            const int o = g + 8 * nb;
            float w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = 2 * t4 + (e & 1) + 8 * (e >> 1);
                w[e] = i < cin ? S.W[wofs + (o * cin + i) * 9 + tap] : 0.f;
            }
            bf[tap][nb][0] = pack_bf16(w[0], w[1]);
            bf[tap][nb][1] = pack_bf16(w[2], w[3]);
        }
    const uint32_t *in32 = reinterpret_cast<const uint32_t *>(&IN[0][0][0]);   // 8 words per pixel
    for (int mt = warp; mt < MT; mt += 8) {
        const int p0 = min(mt * 16 + g, NPIX - 1), p1 = min(mt * 16 + g + 8, NPIX - 1);
        const int r0 = p0 / OW, c0 = p0 - r0 * OW, r1 = p1 / OW, c1 = p1 - r1 * OW;
        float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int dr = tap / 3, dc = tap % 3;
            const int q0 = ((r0 + dr) * IW + c0 + dc) * 8, q1 = ((r1 + dr) * IW + c1 + dc) * 8;
            const uint32_t a0 = in32[q0 + t4], a1 = in32[q1 + t4], a2 = in32[q0 + t4 + 4], a3 = in32[q1 + t4 + 4];
            mma_bf16(acc[0], a0, a1, a2, a3, bf[tap][0][0], bf[tap][0][1]);
            mma_bf16(acc[1], a0, a1, a2, a3, bf[tap][1][0], bf[tap][1][1]);
        }
        // epilogue: bias, ReLU, zero outside the grid, BF16
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int pp = mt * 16 + g + 8 * half;
            if (pp >= NPIX) continue;
            const int r = pp / OW, c = pp - r * OW, gi = gi0 + r, gj = gj0 + c;
            const bool in = gi >= 0 && gi < n && gj >= 0 && gj < m;
#pragma unroll
            for (int nb = 0; nb < 2; ++nb)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int o = 8 * nb + 2 * t4 + e;
                    const float v = in ? fmaxf(acc[nb][2 * half + e] + S.W[bofs + o], 0.f) : 0.f;
                    OUT[r][c][o] = __float2bfloat16(v);
                }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_omega_infer(LevelView<T> L, const __nv_bfloat16 *net, T *omega) {
    extern __shared__ __align__(16) unsigned char smem_inf[];
    InferSmem &S = *reinterpret_cast<InferSmem *>(smem_inf);
    const int tid = threadIdx.x, i0 = blockIdx.y * 16, j0 = blockIdx.x * 16;
    const int n = L.n, m = L.m, p = L.pitch;
    for (int q = tid; q < kNP; q += 256) S.W[q] = __bfloat162float(net[q]);
    for (int q = tid; q < 24 * 24; q += 256) {
        const int r = q / 24, c = q % 24, gi = i0 - 4 + r, gj = j0 - 4 + c;
        S.G[r][c] = (gi >= 0 && gi < n && gj >= 0 && gj < m) ? (float)L.G[(size_t)gi * p + gj] : 0.f;
    }
    __syncthreads();
    for (int q = tid; q < 22 * 22; q += 256) {
        const int r = q / 22, c = q % 22, gi = i0 - 3 + r, gj = j0 - 3 + c;
        float x[kCin] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (gi >= 0 && gi < n && gj >= 0 && gj < m) {
            const int a = r + 1, b = c + 1;
            const float gc = S.G[a][b];
            cell_features(face(gc, S.G[a + 1][b], gi + 1 < n), face(gc, S.G[a - 1][b], gi > 0),
                          face(gc, S.G[a][b + 1], gj + 1 < m), face(gc, S.G[a][b - 1], gj > 0), x);
        }
        for (int k = 0; k < kCh; ++k) S.X[r][c][k] = __float2bfloat16(k < kCin ? x[k] : 0.f);
    }
    __syncthreads();
    conv_tc<22>(S, S.X, S.A1, oW1, oB1, kCin, i0 - 2, j0 - 2, n, m);
    __syncthreads();
    conv_tc<20>(S, S.A1, S.A2, oW2, oB2, kCh, i0 - 1, j0 - 1, n, m);
    __syncthreads();
    {
        const int r = tid / 16, c = tid % 16, gi = i0 + r, gj = j0 + c;
        if (gi < n && gj < m) {
            float z = S.W[oB3];
            for (int i = 0; i < kCh; ++i)
                for (int di = 0; di < 3; ++di)
                    for (int dj = 0; dj < 3; ++dj)
                        z = fmaf(S.W[oW3 + (i * 3 + di) * 3 + dj], __bfloat162float(S.A2[r + di][c + dj][i]), z);
            stc(omega, (size_t)gi * p + gj, (size_t)n * p, kDbgOther, T(2.f / (1.f + expf(-z))));
        }
    }
}

// ---------------------------------------------------------------------------------------
// Training.  Crop record: 7 planes of 24 x 24 floats (cS, cN, cE, cW, f, u, and in plane 6 at
// [0] = 1/tau, [1] = colour parity of the origin).
// ---------------------------------------------------------------------------------------
constexpr int kCrop = 24, kCC = kCrop * kCrop, kRec = 7 * kCC;

template <typename T>
__global__ void k_record_crops(LevelView<T> L, const int *origins, int count, float *data, int first) {
    const int k = blockIdx.x;
    if (k >= count) return;
    const int i0 = origins[2 * k], j0 = origins[2 * k + 1];
    float *rec = data + (size_t)(first + k) * kRec;
    const int n = L.n, m = L.m, p = L.pitch;
    for (int q = threadIdx.x; q < kCC; q += blockDim.x) {
        const int gi = i0 + q / kCrop, gj = j0 + q % kCrop;
        const size_t o = (size_t)gi * p + gj;
        const T gc = L.G[o];
        const bool hS = gi + 1 < n, hN = gi > 0, hE = gj + 1 < m, hW = gj > 0;
        rec[0 * kCC + q] = (float)(L.cdiff * face(gc, L.G[hS ? o + p : o], hS));
        rec[1 * kCC + q] = (float)(L.cdiff * face(gc, L.G[hN ? o - p : o], hN));
        rec[2 * kCC + q] = (float)(L.cdiff * face(gc, L.G[hE ? o + 1 : o], hE));
        rec[3 * kCC + q] = (float)(L.cdiff * face(gc, L.G[hW ? o - 1 : o], hW));
        rec[4 * kCC + q] = (float)L.f[o];
        rec[5 * kCC + q] = (float)L.u[o];
    }
    if (threadIdx.x == 0) {
        rec[6 * kCC + 0] = (float)L.inv_tau;
        rec[6 * kCC + 1] = (float)((i0 + j0) & 1);
    }
}

struct TrainSmem {
    float c[4][kCC], S[kCC], f[kCC], u0[kCC], u1[kCC], u2[kCC], g0[kCC], g1[kCC], x[kCin][kCC];
    float om[kCC], sig[kCC], r[kCC], du[kCC], dom[kCC], t[kCC];
    float a1[kCh][kCC], a2[kCh][kCC], d[kCh][kCC];
    float W[kNP];
    double red[33];
};

// y[o] at cell q of a 24 x 24 plane: 3x3 cross-correlation with zero padding.
__device__ __forceinline__ float conv_at(const float *W, int o, int cin, const float *in, int r, int c,
                                         float bias) {
    float acc = bias;
    for (int i = 0; i < cin; ++i)
        for (int di = 0; di < 3; ++di) {
            const int rr = r + di - 1;
            if (rr < 0 || rr >= kCrop) continue;
            for (int dj = 0; dj < 3; ++dj) {
                const int cc = c + dj - 1;
                if (cc < 0 || cc >= kCrop) continue;
                acc = fmaf(W[((o * cin + i) * 3 + di) * 3 + dj], in[i * kCC + rr * kCrop + cc], acc);
            }
        }
    return acc;
}

__global__ void __launch_bounds__(256) k_train_crop(const float *theta, const float *data, const int *idx,
                                                    float *grad, float *loss, int hf) {
    extern __shared__ __align__(16) unsigned char smem_tr[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_tr);
    const int tid = threadIdx.x, nt = blockDim.x;
    const float *rec = data + (size_t)idx[blockIdx.x] * kRec;
    for (int q = tid; q < kNP; q += nt) S.W[q] = theta[q];
    const float inv_tau = rec[6 * kCC], par = rec[6 * kCC + 1];
    const int parity0 = par > 0.5f ? 1 : 0;
    for (int q = tid; q < kCC; q += nt) {
        for (int k = 0; k < 4; ++k) S.c[k][q] = rec[k * kCC + q];
        S.f[q] = rec[4 * kCC + q];
        S.u0[q] = rec[5 * kCC + q];
        S.S[q] = S.c[0][q] + S.c[1][q] + S.c[2][q] + S.c[3][q] + inv_tau;
        float x[kCin];
        cell_features(S.c[0][q], S.c[1][q], S.c[2][q], S.c[3][q], x);
        for (int k = 0; k < kCin; ++k) S.x[k][q] = x[k];
    }
    __syncthreads();
    // forward: two convolutions with ReLU, the output convolution, omega = 2 sigmoid
    for (int q = tid; q < kCh * kCC; q += nt) {
        const int o = q / kCC, cell = q % kCC;
        S.a1[o][cell] = fmaxf(conv_at(S.W + oW1, o, kCin, &S.x[0][0], cell / kCrop, cell % kCrop, S.W[oB1 + o]), 0.f);
    }
    __syncthreads();
    for (int q = tid; q < kCh * kCC; q += nt) {
        const int o = q / kCC, cell = q % kCC;
        S.a2[o][cell] = fmaxf(conv_at(S.W + oW2, o, kCh, &S.a1[0][0], cell / kCrop, cell % kCrop, S.W[oB2 + o]), 0.f);
    }
    __syncthreads();
    for (int q = tid; q < kCC; q += nt) {
        const float z = conv_at(S.W + oW3, 0, kCh, &S.a2[0][0], q / kCrop, q % kCrop, S.W[oB3]);
        const float sg = 1.f / (1.f + expf(-z));
        S.sig[q] = sg;
        S.om[q] = 2.f * sg;
    }
    __syncthreads();
    // the two damped colour phases on the cells at least one inside
    auto inner = [&](int q) { const int r = q / kCrop, c = q % kCrop; return r >= 1 && r < kCrop - 1 && c >= 1 && c < kCrop - 1; };
    auto gval = [&](const float *u, int q) {
        return (S.c[0][q] * u[q + kCrop] + S.c[1][q] * u[q - kCrop] + S.c[2][q] * u[q + 1] + S.c[3][q] * u[q - 1] - S.f[q]) / S.S[q];
    };
    for (int ph = 0; ph < 2; ++ph) {
        const float *prev = ph == 0 ? S.u0 : S.u1;
        float *nxt = ph == 0 ? S.u1 : S.u2;
        float *gv = ph == 0 ? S.g0 : S.g1;
        for (int q = tid; q < kCC; q += nt) {
            const bool sel = inner(q) && (((q / kCrop + q % kCrop + parity0) & 1) == ph);
            const float g = inner(q) ? gval(prev, q) : 0.f;
            gv[q] = g;
            nxt[q] = sel ? prev[q] + S.om[q] * (g - prev[q]) : prev[q];
        }
        __syncthreads();
    }
    // residual (in t), the loss over the cells at least two inside
    const int cnt = (kCrop - 4) * (kCrop - 4);
    for (int q = tid; q < kCC; q += nt) {
        float r = 0.f;
        if (inner(q))
            r = S.f[q] - (S.c[0][q] * S.u2[q + kCrop] + S.c[1][q] * S.u2[q - kCrop] + S.c[2][q] * S.u2[q + 1] +
                          S.c[3][q] * S.u2[q - 1] - S.S[q] * S.u2[q]);
        S.t[q] = r;
    }
    __syncthreads();
    double ls = 0.0;
    for (int q = tid; q < kCC; q += nt) {
        const int rr = q / kCrop, cc = q % kCrop;
        const bool lc = rr >= 2 && rr < kCrop - 2 && cc >= 2 && cc < kCrop - 2;
        float v = 0.f;
        if (lc) {
            v = hf ? 4.f * S.t[q] - (S.t[q + kCrop] + S.t[q - kCrop] + S.t[q + 1] + S.t[q - 1]) : S.t[q];
            ls += 0.5 * (double)v * v;
        }
        S.du[q] = lc ? v / cnt : 0.f;           // dL/dv
    }
    ls = block_sum(ls, S.red);
    if (tid == 0) loss[blockIdx.x] = (float)(ls / cnt);
    __syncthreads();
    for (int q = tid; q < kCC; q += nt) {      // dL/dr (the high-pass stencil is symmetric)
        float d = S.du[q];
        if (hf) d = inner(q) ? 4.f * S.du[q] - (S.du[q + kCrop] + S.du[q - kCrop] + S.du[q + 1] + S.du[q - 1]) : 0.f;
        S.r[q] = d;
    }
    __syncthreads();
    // dL/du2 through r = f - (sum c u_X - S u)
    for (int q = tid; q < kCC; q += nt) {
        const int rr = q / kCrop, cc = q % kCrop;
        float v = inner(q) ? S.S[q] * S.r[q] : 0.f;
        if (rr >= 1 && inner(q - kCrop)) v -= S.c[0][q - kCrop] * S.r[q - kCrop];
        if (rr + 1 < kCrop && inner(q + kCrop)) v -= S.c[1][q + kCrop] * S.r[q + kCrop];
        if (cc >= 1 && inner(q - 1)) v -= S.c[2][q - 1] * S.r[q - 1];
        if (cc + 1 < kCrop && inner(q + 1)) v -= S.c[3][q + 1] * S.r[q + 1];
        S.du[q] = v;
        S.dom[q] = 0.f;
    }
    __syncthreads();
    for (int ph = 1; ph >= 0; --ph) {
        const float *prev = ph == 0 ? S.u0 : S.u1;
        const float *gv = ph == 0 ? S.g0 : S.g1;
        for (int q = tid; q < kCC; q += nt) {
            const bool sel = inner(q) && (((q / kCrop + q % kCrop + parity0) & 1) == ph);
            S.t[q] = sel ? S.du[q] * S.om[q] / S.S[q] : 0.f;      // dL/dg at updated cells
            if (sel) S.dom[q] += S.du[q] * (gv[q] - prev[q]);
        }
        __syncthreads();
        for (int q = tid; q < kCC; q += nt) {
            const int rr = q / kCrop, cc = q % kCrop;
            const bool sel = inner(q) && (((rr + cc + parity0) & 1) == ph);
            float v = sel ? S.du[q] * (1.f - S.om[q]) : S.du[q];
            // the updated cells whose g reads cell q
            if (rr >= 1) v += S.c[0][q - kCrop] * S.t[q - kCrop];
            if (rr + 1 < kCrop) v += S.c[1][q + kCrop] * S.t[q + kCrop];
            if (cc >= 1) v += S.c[2][q - 1] * S.t[q - 1];
            if (cc + 1 < kCrop) v += S.c[3][q + 1] * S.t[q + 1];
            S.g1[q] = v;   // new dL/du (g1 no longer needed after this phase's use above)
        }
        __syncthreads();
        for (int q = tid; q < kCC; q += nt) S.du[q] = S.g1[q];
        __syncthreads();
    }
    // dz3 into r
    for (int q = tid; q < kCC; q += nt) S.r[q] = S.dom[q] * 2.f * S.sig[q] * (1.f - S.sig[q]);
    __syncthreads();
    float *g = grad + (size_t)blockIdx.x * kNP;
    // layer 3: dW3, db3; da2 into d (masked by a2 > 0)
    for (int k = tid; k < 144 + 1; k += nt) {
        float acc = 0.f;
        if (k < 144) {
            const int i = k / 9, di = (k / 3) % 3, dj = k % 3;
            for (int q = 0; q < kCC; ++q) {
                const int rr = q / kCrop + di - 1, cc = q % kCrop + dj - 1;
                if (rr >= 0 && rr < kCrop && cc >= 0 && cc < kCrop) acc = fmaf(S.r[q], S.a2[i][rr * kCrop + cc], acc);
            }
            g[oW3 + k] = acc;
        } else {
            for (int q = 0; q < kCC; ++q) acc += S.r[q];
            g[oB3] = acc;
        }
    }
    for (int q = tid; q < kCh * kCC; q += nt) {
        const int i = q / kCC, cell = q % kCC, r0 = cell / kCrop, c0 = cell % kCrop;
        float acc = 0.f;
        for (int di = 0; di < 3; ++di)
            for (int dj = 0; dj < 3; ++dj) {
                const int rr = r0 - di + 1, cc = c0 - dj + 1;     // outputs whose window holds this cell
                if (rr >= 0 && rr < kCrop && cc >= 0 && cc < kCrop)
                    acc = fmaf(S.W[oW3 + (i * 3 + di) * 3 + dj], S.r[rr * kCrop + cc], acc);
            }
        S.d[i][cell] = S.a2[i][cell] > 0.f ? acc : 0.f;
    }
    __syncthreads();
    // layer 2: dW2, db2 (dz2 in d); da1 into a2 (masked by a1 > 0)
    for (int k = tid; k < 2304 + 16; k += nt) {
        float acc = 0.f;
        if (k < 2304) {
            const int o = k / 144, i = (k / 9) % 16, di = (k / 3) % 3, dj = k % 3;
            for (int q = 0; q < kCC; ++q) {
                const int rr = q / kCrop + di - 1, cc = q % kCrop + dj - 1;
                if (rr >= 0 && rr < kCrop && cc >= 0 && cc < kCrop) acc = fmaf(S.d[o][q], S.a1[i][rr * kCrop + cc], acc);
            }
            g[oW2 + k] = acc;
        } else {
            const int o = k - 2304;
            for (int q = 0; q < kCC; ++q) acc += S.d[o][q];
            g[oB2 + o] = acc;
        }
    }
    __syncthreads();
    for (int q = tid; q < kCh * kCC; q += nt) {
        const int i = q / kCC, cell = q % kCC, r0 = cell / kCrop, c0 = cell % kCrop;
        float acc = 0.f;
        for (int o = 0; o < kCh; ++o)
            for (int di = 0; di < 3; ++di)
                for (int dj = 0; dj < 3; ++dj) {
                    const int rr = r0 - di + 1, cc = c0 - dj + 1;
                    if (rr >= 0 && rr < kCrop && cc >= 0 && cc < kCrop)
                        acc = fmaf(S.W[oW2 + ((o * kCh + i) * 3 + di) * 3 + dj], S.d[o][rr * kCrop + cc], acc);
                }
        S.a2[i][cell] = S.a1[i][cell] > 0.f ? acc : 0.f;          // dz1
    }
    __syncthreads();
    // layer 1: dW1, db1 (dz1 in a2)
    for (int k = tid; k < 720 + 16; k += nt) {
        float acc = 0.f;
        if (k < 720) {
            const int o = k / 45, i = (k / 9) % 5, di = (k / 3) % 3, dj = k % 3;
            for (int q = 0; q < kCC; ++q) {
                const int rr = q / kCrop + di - 1, cc = q % kCrop + dj - 1;
                if (rr >= 0 && rr < kCrop && cc >= 0 && cc < kCrop) acc = fmaf(S.a2[o][q], S.x[i][rr * kCrop + cc], acc);
            }
            g[oW1 + k] = acc;
        } else {
            const int o = k - 720;
            for (int q = 0; q < kCC; ++q) acc += S.a2[o][q];
            g[oB1 + o] = acc;
        }
    }
}

// Mean of the per-crop gradients and losses, in crop order.
__global__ void k_train_reduce(const float *grad, const float *loss, int batch, float *gmean, float *lmean) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < kNP) {
        double s = 0.0;
        for (int b = 0; b < batch; ++b) s += grad[(size_t)b * kNP + k];
        gmean[k] = (float)(s / batch);
    }
    if (k == 0) {
        double s = 0.0;
        for (int b = 0; b < batch; ++b) s += loss[b];
        *lmean = (float)(s / batch);
    }
}

// One Adam step (Kingma and Ba, 2015) on every parameter.
__global__ void k_adam(float *theta, float *mom, float *vel, const float *g, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNP) return;
    const float gk = g[k];
    const float mk = b1 * mom[k] + (1.f - b1) * gk;
    const float vk = b2 * vel[k] + (1.f - b2) * gk * gk;
    mom[k] = mk;
    vel[k] = vk;
    theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

}  // namespace

int learned_nparam() { return kNP; }
int learned_crop() { return kCrop; }
size_t learned_record_floats() { return kRec; }

void prepare_learned_kernels() {
    cudaFuncSetAttribute(k_omega_infer<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(InferSmem));
    cudaFuncSetAttribute(k_omega_infer<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(InferSmem));
    cudaFuncSetAttribute(k_train_crop, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem));
}

template <typename T>
void launch_omega_infer(const LevelView<T> &L, const __nv_bfloat16 *net, T *omega, cudaStream_t st) {
    dim3 grid((L.m + 15) / 16, (L.n + 15) / 16);
    k_omega_infer<T><<<grid, 256, sizeof(InferSmem), st>>>(L, net, omega);
}

template <typename T>
void launch_record_crops(const LevelView<T> &L, const int *origins, int count, float *data, int first,
                         cudaStream_t st) {
    k_record_crops<T><<<count, 256, 0, st>>>(L, origins, count, data, first);
}

void launch_train_step(float *theta, float *mom, float *vel, const float *data, const int *idx, int batch,
                       float *grad, float *loss, float *gmean, float *lmean, float lr, int step, int loss_kind,
                       cudaStream_t st) {
    k_train_crop<<<batch, 256, sizeof(TrainSmem), st>>>(theta, data, idx, grad, loss, loss_kind);
    k_train_reduce<<<(kNP + 255) / 256, 256, 0, st>>>(grad, loss, batch, gmean, lmean);
    if (!(lr > 0.f)) return;   // gradient only
    const float b1 = 0.9f, b2 = 0.999f;
    k_adam<<<(kNP + 255) / 256, 256, 0, st>>>(theta, mom, vel, gmean, lr, b1, b2,
                                              1.f - powf(b1, (float)step), 1.f - powf(b2, (float)step), 1e-8f);
}

template void launch_omega_infer<float>(const LevelView<float> &, const __nv_bfloat16 *, float *, cudaStream_t);
template void launch_omega_infer<double>(const LevelView<double> &, const __nv_bfloat16 *, double *, cudaStream_t);
template void launch_record_crops<float>(const LevelView<float> &, const int *, int, float *, int, cudaStream_t);
template void launch_record_crops<double>(const LevelView<double> &, const int *, int, float *, int, cudaStream_t);

}  // namespace segmg
