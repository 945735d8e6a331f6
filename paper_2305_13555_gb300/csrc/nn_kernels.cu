// 1-D convolutional network over cells (learned initial guess / corrector of
// the OCI iteration): forward, backward, Adam, feature and target builders.
//
// Network: 5 convolution layers along the cell index, kernel width 5, zero
// padding of 2 cells at the slab ends, channels 13 -> 32 -> 32 -> 32 -> 32 -> 4,
// ReLU after layers 1-4.  Weights are used in BF16 (rounded from FP32 master
// copies), activations and all accumulations are FP32.  Parameter layout: per
// layer W[co][ci][5] then b[co] (flat FP32).  Activations: [B][C][J] FP32.
// Reductions over cells (weight gradients, loss) are per-tile partials summed
// in a fixed order, so results are deterministic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/oci_nn.h"

namespace ocinn {

constexpr int KW = 5, PAD = 2, NL = 5;
constexpr int CH[NL + 1] = {13, 32, 32, 32, 32, 4};
constexpr int TX = 128;      // cells per tile
constexpr int MAXC = 32;

constexpr int layer_w(int l) { return CH[l + 1] * CH[l] * KW; }
constexpr int layer_off(int l)
{
    int o = 0;
    for (int i = 0; i < l; ++i) o += layer_w(i) + CH[i + 1];
    return o;
}
constexpr int NPARAM = layer_off(NL);

// ------------------------------------------------------------- forward conv
// out[b][co][x] = bias[co] + sum_ci sum_k W[co][ci][k] in[b][ci][x+k-2]; one
// thread per cell x computes every output channel.  If FLIP, the kernel runs
// the data gradient instead: W is read as W'[ci'][co'][k] = W[co'][ci'][4-k]
// (input channels = the layer's outputs), no bias, and the incoming gradient is
// masked by the ReLU derivative of `mask` (the layer's own output) on load.
template <int CI, int CO, bool RELU, bool FLIP>
__global__ void __launch_bounds__(TX) k_conv(const float *__restrict__ in, const float *__restrict__ mask,
                                             const __nv_bfloat16 *__restrict__ W, const float *__restrict__ bias,
                                             float *__restrict__ out, int J)
{
    __shared__ float s_in[CI][TX + 2 * PAD];
    __shared__ __align__(16) float s_w[CI][KW][CO];   // [ci][k][co] for vector loads over co
    const int b = blockIdx.y, x0 = blockIdx.x * TX, t = threadIdx.x;
    // weights: natural layout W[o][i][k] (o = CO or CI of the forward layer)
    for (int e = t; e < CI * KW * CO; e += TX) {
        const int co = e % CO, k = (e / CO) % KW, ci = e / (CO * KW);
        float w;
        if (!FLIP) w = __bfloat162float(W[(co * CI + ci) * KW + k]);
        else w = __bfloat162float(W[(ci * CO + co) * KW + (KW - 1 - k)]);  // forward layer had CO' = CI inputs
        s_w[ci][k][co] = w;
    }
    for (int e = t; e < CI * (TX + 2 * PAD); e += TX) {
        const int ci = e / (TX + 2 * PAD), xx = e % (TX + 2 * PAD);
        const int x = x0 + xx - PAD;
        float v = 0.f;
        if (x >= 0 && x < J) {
            v = in[((size_t)b * CI + ci) * J + x];
            if (FLIP && mask) v = mask[((size_t)b * CI + ci) * J + x] > 0.f ? v : 0.f;
        }
        s_in[ci][xx] = v;
    }
    __syncthreads();
    const int x = x0 + t;
    if (x >= J) return;
    float acc[CO];
#pragma unroll
    for (int co = 0; co < CO; ++co) acc[co] = (!FLIP && bias) ? bias[co] : 0.f;
    for (int ci = 0; ci < CI; ++ci) {
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const float v = s_in[ci][t + k];
            if constexpr (CO % 4 == 0) {
#pragma unroll
                for (int c4 = 0; c4 < CO / 4; ++c4) {
                    const float4 w = *reinterpret_cast<const float4 *>(&s_w[ci][k][4 * c4]);
                    acc[4 * c4 + 0] = __fmaf_rn(w.x, v, acc[4 * c4 + 0]);
                    acc[4 * c4 + 1] = __fmaf_rn(w.y, v, acc[4 * c4 + 1]);
                    acc[4 * c4 + 2] = __fmaf_rn(w.z, v, acc[4 * c4 + 2]);
                    acc[4 * c4 + 3] = __fmaf_rn(w.w, v, acc[4 * c4 + 3]);
                }
            } else {
#pragma unroll
                for (int co = 0; co < CO; ++co) acc[co] = __fmaf_rn(s_w[ci][k][co], v, acc[co]);
            }
        }
    }
#pragma unroll
    for (int co = 0; co < CO; ++co) {
        float r = acc[co];
        if (RELU) r = fmaxf(r, 0.f);
        out[((size_t)b * CO + co) * J + x] = r;
    }
}

// ------------------------------------------------- forward conv, tensor cores
// Inference form of the layer: the same contraction as a GEMM per tile of TX
// cells, out[x][co] = sum_{k, ci} in[x + k - 2][ci] W[co][ci][k], on the BF16
// tensor-core MMA (m16n8k16, FP32 accumulate): the layer's input rounded to
// BF16 (the weights already are), bias and ReLU in FP32.  Shared memory holds
// the input tile transposed to [x][ci] and the weights as [k][co][ci], both
// with the channel index contiguous so that every fragment register is one
// 32-bit load of two adjacent channels; row strides padded by 8 elements keep
// the eight rows of a fragment in distinct banks.  Each of the four warps owns
// 32 cells (two 16-row tiles) and every output channel (CO / 8 8-column tiles).
template <int CI, int CO, bool RELU>
__global__ void __launch_bounds__(TX) k_conv_mma(const float *__restrict__ in, const __nv_bfloat16 *__restrict__ W,
                                                 const float *__restrict__ bias, float *__restrict__ out, int J)
{
    constexpr int KC = (CI + 15) / 16, CIP = KC * 16;  // 16-channel K chunks, padded input channels
    constexpr int NT = (CO + 7) / 8, COP = NT * 8;     // 8-channel N tiles, padded output channels
    constexpr int RS = CIP + 8;                        // row stride of both tiles (bf16 elements)
    constexpr int XR = TX + 2 * PAD;                   // input rows of a tile
    static_assert(TX == 128, "four warps of 32 cells");
    __shared__ __align__(16) __nv_bfloat16 s_in[XR * RS];
    __shared__ __align__(16) __nv_bfloat16 s_w[KW * COP * RS];
    const int b = blockIdx.y, x0 = blockIdx.x * TX, t = threadIdx.x;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int e = t; e < KW * COP * CIP; e += TX) {
        const int ci = e % CIP, co = (e / CIP) % COP, k = e / (CIP * COP);
        s_w[(k * COP + co) * RS + ci] = (ci < CI && co < CO) ? W[(co * CI + ci) * KW + k] : zero;
    }
    for (int e = t; e < CIP * XR; e += TX) {
        const int ci = e / XR, xx = e % XR;
        const int x = x0 + xx - PAD;
        const float v = (ci < CI && x >= 0 && x < J) ? in[((size_t)b * CI + ci) * J + x] : 0.f;
        s_in[xx * RS + ci] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    const int warp = t >> 5, lane = t & 31, g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = warp * 32 + mt * 16 + g;  // this lane's two rows: r0 and r0 + 8
        float acc[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
        for (int k = 0; k < KW; ++k) {
#pragma unroll
            for (int kc = 0; kc < KC; ++kc) {
                const int c = kc * 16 + 2 * tq;
                const unsigned a0 = *reinterpret_cast<const unsigned *>(&s_in[(r0 + k) * RS + c]);
                const unsigned a1 = *reinterpret_cast<const unsigned *>(&s_in[(r0 + 8 + k) * RS + c]);
                const unsigned a2 = *reinterpret_cast<const unsigned *>(&s_in[(r0 + k) * RS + c + 8]);
                const unsigned a3 = *reinterpret_cast<const unsigned *>(&s_in[(r0 + 8 + k) * RS + c + 8]);
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const __nv_bfloat16 *wr = &s_w[(k * COP + n * 8 + g) * RS + c];
                    const unsigned b0 = *reinterpret_cast<const unsigned *>(wr);
                    const unsigned b1 = *reinterpret_cast<const unsigned *>(wr + 8);
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                        "{%8, %9}, {%0, %1, %2, %3};\n"
                        : "+f"(acc[n][0]), "+f"(acc[n][1]), "+f"(acc[n][2]), "+f"(acc[n][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                }
            }
        }
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int co = n * 8 + 2 * tq + (h & 1);
                const int x = x0 + r0 + (h >> 1) * 8;
                if (co < CO && x < J) {
                    float r = acc[n][h] + bias[co];
                    if (RELU) r = fmaxf(r, 0.f);
                    out[((size_t)b * CO + co) * J + x] = r;
                }
            }
    }
}

// ------------------------------------------------------------- fused inference
// All five layers of one tile of cells in one CTA, the activations kept in
// shared memory.  Output cell x of the network depends on input cells x - 10 ..
// x + 10 (five layers of half-width 2), so a tile of FOUT = 240 output cells
// reads FB = 260 input rows; every layer computes FR = 256 rows (16 m-tiles of
// the m16n8k16 MMA, two per warp) of which the valid region shrinks by two
// rows per side and layer, ending on the tile's 240 cells.  Rows whose cell is
// outside the slab are stored as zero after every layer (the zero padding of
// each layer's input).  Arithmetic per output element is that of k_conv_mma
// (same MMA sequence, FP32 bias and ReLU, the next layer's input rounded to
// BF16), so the result is bit-identical to the per-layer kernels.
// Shared image of the parameters (packed once per call by k_pack_fused): per
// layer [k][co][ci] BF16 with row stride ci_padded + 8, then the FP32 biases.
constexpr int FWARPS = 8, FTHREADS = FWARPS * 32;
constexpr int FR = 16 * 2 * FWARPS;          // rows computed per layer
constexpr int FB = FR + 2 * PAD;             // rows of each activation buffer
constexpr int FOUT = FB - 2 * PAD * NL;      // valid output cells per tile
constexpr int fcip(int l) { return ((CH[l] + 15) / 16) * 16; }
constexpr int fcop(int l) { return ((CH[l + 1] + 7) / 8) * 8; }
constexpr int frs(int l) { return fcip(l) + 8; }
constexpr int fw_off(int l)
{
    int o = 0;
    for (int i = 0; i < l; ++i) o += KW * fcop(i) * frs(i);
    return o;
}
constexpr int FW_ELEMS = fw_off(NL);                      // BF16 weight elements
constexpr int FBIAS = 4 * 32 + 8;                         // FP32 biases, layer by layer (last padded to 8)
constexpr int fb_off(int l) { return l * 32; }
constexpr int FPACK_BYTES = FW_ELEMS * 2 + FBIAS * 4;     // the packed image
constexpr int FCI = CH[0], FCO = CH[NL];                  // network input and output channels
constexpr int FRS_ACT = 32 + 8;                           // row stride of the 32-channel buffers
constexpr int FSMEM = FPACK_BYTES + FB * frs(0) * 2 + 2 * FB * FRS_ACT * 2;
static_assert(FPACK_BYTES % 16 == 0 && (FB * frs(0) * 2) % 16 == 0, "16-byte aligned regions");
static_assert(4 * FOUT * 4 <= FB * frs(0) * 2, "output staging fits in the input buffer");

template <int L>
__device__ __forceinline__ void pack_layer(const float *__restrict__ params, __nv_bfloat16 *__restrict__ w,
                                           float *__restrict__ bias, int r)
{
    constexpr int CI = CH[L], CO = CH[L + 1], RS = frs(L), COP = fcop(L), WOFF = layer_off(L);
    constexpr int N = KW * COP * RS;
    if (r < N) {
        const int ci = r % RS, co = (r / RS) % COP, k = r / (RS * COP);
        const float v = (ci < CI && co < CO) ? params[WOFF + (co * CI + ci) * KW + k] : 0.f;
        w[fw_off(L) + r] = __float2bfloat16_rn(v);
    } else if (r < N + 32) {
        const int co = r - N;
        if (L < NL - 1 || co < 8) bias[fb_off(L) + co] = co < CO ? params[WOFF + CI * CO * KW + co] : 0.f;
    }
}

// one thread per element of a layer's weight image (and its biases): grid (blocks, NL)
__global__ void k_pack_fused(const float *__restrict__ params, unsigned char *__restrict__ pack)
{
    __nv_bfloat16 *w = reinterpret_cast<__nv_bfloat16 *>(pack);
    float *bias = reinterpret_cast<float *>(pack + FW_ELEMS * 2);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    switch (blockIdx.y) {
    case 0: pack_layer<0>(params, w, bias, r); break;
    case 1: pack_layer<1>(params, w, bias, r); break;
    case 2: pack_layer<2>(params, w, bias, r); break;
    case 3: pack_layer<3>(params, w, bias, r); break;
    default: pack_layer<4>(params, w, bias, r); break;
    }
}
constexpr int FPACK_MAX_LAYER = KW * 32 * (32 + 8) + 32;  // elements of the largest layer image + biases

// One layer over the tile: src rows [0, FB) (stride frs(L)) -> rows [2, FB - 2)
// of dst (stride FRS_ACT, BF16, zero outside the slab), or, for the last layer,
// the FP32 outputs of the tile's valid rows into dout[co][row - 2 PAD NL].
template <int L>
__device__ __forceinline__ void fused_layer(const __nv_bfloat16 *src, const __nv_bfloat16 *w, const float *bias,
                                            __nv_bfloat16 *dst, float *dout, int xrow0, int J, int warp, int lane)
{
    constexpr int CO = CH[L + 1];
    constexpr int KC = fcip(L) / 16, RS = frs(L);
    constexpr int NT = fcop(L) / 8, COP = NT * 8;
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int i0 = 16 * (warp + FWARPS * mi) + g;  // input row of tap 0 for this lane's first output row
        float acc[NT][4];
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
#pragma unroll
        for (int k = 0; k < KW; ++k) {
#pragma unroll
            for (int kc = 0; kc < KC; ++kc) {
                const int c = kc * 16 + 2 * tq;
                const unsigned a0 = *reinterpret_cast<const unsigned *>(&src[(i0 + k) * RS + c]);
                const unsigned a1 = *reinterpret_cast<const unsigned *>(&src[(i0 + 8 + k) * RS + c]);
                const unsigned a2 = *reinterpret_cast<const unsigned *>(&src[(i0 + k) * RS + c + 8]);
                const unsigned a3 = *reinterpret_cast<const unsigned *>(&src[(i0 + 8 + k) * RS + c + 8]);
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const __nv_bfloat16 *wr = &w[(k * COP + n * 8 + g) * RS + c];
                    const unsigned b0 = *reinterpret_cast<const unsigned *>(wr);
                    const unsigned b1 = *reinterpret_cast<const unsigned *>(wr + 8);
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                        "{%8, %9}, {%0, %1, %2, %3};\n"
                        : "+f"(acc[n][0]), "+f"(acc[n][1]), "+f"(acc[n][2]), "+f"(acc[n][3])
                        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
                }
            }
        }
#pragma unroll
        for (int hr = 0; hr < 2; ++hr) {  // this lane's output rows i0 + 2 and i0 + 10
            const int o = i0 + PAD + 8 * hr;
            const int x = xrow0 + o;
            const bool inside = x >= 0 && x < J;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int co = n * 8 + 2 * tq;
                float v0 = acc[n][2 * hr] + bias[co], v1 = acc[n][2 * hr + 1] + bias[co + 1];
                if (L < NL - 1) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                    if (!inside) v0 = v1 = 0.f;
                    *reinterpret_cast<__nv_bfloat162 *>(&dst[o * FRS_ACT + co]) = __floats2bfloat162_rn(v0, v1);
                } else {
                    const int r = o - PAD * NL;
                    if (r >= 0 && r < FOUT && co < CO) {
                        dout[co * FOUT + r] = v0;
                        dout[(co + 1) * FOUT + r] = v1;
                    }
                }
            }
        }
    }
}

// Persistent over tiles (b, tile), two CTAs per SM; tile t of sample b covers
// output cells [t FOUT, (t + 1) FOUT).
__global__ void __launch_bounds__(FTHREADS, 2) k_forward_fused(const unsigned char *__restrict__ pack,
                                                                const float *__restrict__ in, float *__restrict__ out,
                                                                int B, int J)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    const __nv_bfloat16 *s_w = reinterpret_cast<const __nv_bfloat16 *>(fsm);
    const float *s_bias = reinterpret_cast<const float *>(fsm + FW_ELEMS * 2);
    __nv_bfloat16 *s_x = reinterpret_cast<__nv_bfloat16 *>(fsm + FPACK_BYTES);
    __nv_bfloat16 *s_a = s_x + FB * frs(0);
    __nv_bfloat16 *s_b = s_a + FB * FRS_ACT;
    float *s_out = reinterpret_cast<float *>(s_x);  // free once layer 0 has read it
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int per = (J + FOUT - 1) / FOUT;
    // the tile's input rows, FP32 in registers: loaded for the next tile while the
    // current one's layers run, rounded and transposed into s_x afterwards
    constexpr int NST = (fcip(0) * FB + FTHREADS - 1) / FTHREADS;
    float stage[NST];
    auto load_tile = [&](int tile) {
        const int b = tile / per, xrow0 = (tile % per) * FOUT - PAD * NL;
#pragma unroll
        for (int u = 0; u < NST; ++u) {
            const int e = t + u * FTHREADS;
            const int ci = e / FB, r = e % FB, x = xrow0 + r;
            stage[u] = (e < fcip(0) * FB && ci < FCI && x >= 0 && x < J) ? __ldg(in + ((size_t)b * FCI + ci) * J + x)
                                                                        : 0.f;
        }
    };
    auto store_tile = [&]() {
#pragma unroll
        for (int u = 0; u < NST; ++u) {
            const int e = t + u * FTHREADS;
            if (e < fcip(0) * FB) s_x[(e % FB) * frs(0) + e / FB] = __float2bfloat16_rn(stage[u]);
        }
    };
    if (blockIdx.x < B * per) load_tile(blockIdx.x);
    {
        // the parameter image: every thread's 16-byte loads issued before any is stored
        constexpr int NW = (FPACK_BYTES / 16 + FTHREADS - 1) / FTHREADS;
        const uint4 *src = reinterpret_cast<const uint4 *>(pack);
        uint4 *dst = reinterpret_cast<uint4 *>(fsm);
        uint4 wv[NW];
#pragma unroll
        for (int u = 0; u < NW; ++u) {
            const int e = t + u * FTHREADS;
            if (e < FPACK_BYTES / 16) wv[u] = __ldg(src + e);
        }
#pragma unroll
        for (int u = 0; u < NW; ++u) {
            const int e = t + u * FTHREADS;
            if (e < FPACK_BYTES / 16) dst[e] = wv[u];
        }
        const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
        for (int e = t; e < 2 * PAD * FRS_ACT; e += FTHREADS) {  // edge rows no layer writes
            const int r = e / FRS_ACT, c = e % FRS_ACT, row = r < PAD ? r : FB - 2 * PAD + r;
            s_a[row * FRS_ACT + c] = zero;
            s_b[row * FRS_ACT + c] = zero;
        }
    }
    for (int tile = blockIdx.x; tile < B * per; tile += gridDim.x) {
        const int b = tile / per, x0 = (tile % per) * FOUT;
        const int xrow0 = x0 - PAD * NL;  // cell of buffer row 0
        store_tile();
        __syncthreads();
        if (tile + (int)gridDim.x < B * per) load_tile(tile + gridDim.x);  // lands while the layers run
        fused_layer<0>(s_x, s_w + fw_off(0), s_bias + fb_off(0), s_a, nullptr, xrow0, J, warp, lane);
        __syncthreads();
        fused_layer<1>(s_a, s_w + fw_off(1), s_bias + fb_off(1), s_b, nullptr, xrow0, J, warp, lane);
        __syncthreads();
        fused_layer<2>(s_b, s_w + fw_off(2), s_bias + fb_off(2), s_a, nullptr, xrow0, J, warp, lane);
        __syncthreads();
        fused_layer<3>(s_a, s_w + fw_off(3), s_bias + fb_off(3), s_b, nullptr, xrow0, J, warp, lane);
        __syncthreads();
        fused_layer<4>(s_b, s_w + fw_off(4), s_bias + fb_off(4), nullptr, s_out, xrow0, J, warp, lane);
        __syncthreads();
        const int nx = J - x0 < FOUT ? J - x0 : FOUT;
        for (int e = t; e < FCO * FOUT; e += FTHREADS) {
            const int co = e / FOUT, r = e % FOUT;
            if (r < nx) out[((size_t)b * FCO + co) * J + x0 + r] = s_out[e];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- weight grad
// Per tile of TX cells of one sample: partial dW[co][ci][k] = sum_x g[co][x]
// in[ci][x+k-2] and db[co] = sum_x g[co][x], where g is the output gradient
// masked by the ReLU derivative (when the layer has one).
template <int CI, int CO, bool RELU>
__global__ void __launch_bounds__(256) k_wgrad(const float *__restrict__ in, const float *__restrict__ g,
                                               const float *__restrict__ outv, float *__restrict__ partial, int J)
{
    __shared__ float s_in[CI][TX + 2 * PAD];
    __shared__ float s_g[CO][TX];
    const int b = blockIdx.y, x0 = blockIdx.x * TX, t = threadIdx.x;
    for (int e = t; e < CI * (TX + 2 * PAD); e += blockDim.x) {
        const int ci = e / (TX + 2 * PAD), xx = e % (TX + 2 * PAD);
        const int x = x0 + xx - PAD;
        s_in[ci][xx] = (x >= 0 && x < J) ? in[((size_t)b * CI + ci) * J + x] : 0.f;
    }
    for (int e = t; e < CO * TX; e += blockDim.x) {
        const int co = e / TX, xx = e % TX;
        const int x = x0 + xx;
        float v = 0.f;
        if (x < J) {
            v = g[((size_t)b * CO + co) * J + x];
            if (RELU) v = outv[((size_t)b * CO + co) * J + x] > 0.f ? v : 0.f;
        }
        s_g[co][xx] = v;
    }
    __syncthreads();
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    float *part = partial + (size_t)tile * (CO * CI * KW + CO);
    const int nx = J - x0 < TX ? J - x0 : TX;
    for (int pr = t; pr < CO * CI; pr += blockDim.x) {
        const int co = pr / CI, ci = pr % CI;
        float a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0;
        for (int xx = 0; xx < nx; ++xx) {
            const float gv = s_g[co][xx];
            a0 = __fmaf_rn(gv, s_in[ci][xx + 0], a0);
            a1 = __fmaf_rn(gv, s_in[ci][xx + 1], a1);
            a2 = __fmaf_rn(gv, s_in[ci][xx + 2], a2);
            a3 = __fmaf_rn(gv, s_in[ci][xx + 3], a3);
            a4 = __fmaf_rn(gv, s_in[ci][xx + 4], a4);
        }
        float *w = part + (co * CI + ci) * KW;
        w[0] = a0; w[1] = a1; w[2] = a2; w[3] = a3; w[4] = a4;
    }
    for (int co = t; co < CO; co += blockDim.x) {
        float a = 0.f;
        for (int xx = 0; xx < nx; ++xx) a += s_g[co][xx];
        part[CO * CI * KW + co] = a;
    }
}

// Sum the per-tile partials (fixed order) into grad[off .. off + n).
__global__ void k_reduce_partials(const float *__restrict__ partial, int ntiles, int n, float *__restrict__ grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float a = 0.f;
    for (int tile = 0; tile < ntiles; ++tile) a += partial[(size_t)tile * n + i];
    grad[i] = a;
}

// Mean squared error: per-tile partial sums of (out - t)^2 and the output
// gradient 2 (out - t) / count.
__global__ void __launch_bounds__(256) k_mse(const float *__restrict__ out, const float *__restrict__ tgt, size_t n,
                                             float *__restrict__ g, double *__restrict__ partial)
{
    __shared__ double sh[8];
    double acc = 0.0;
    const float scale = 2.f / (float)n;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = out[i] - tgt[i];
        acc += (double)d * d;
        if (g) g[i] = scale * d;
    }
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void k_sum_doubles(const double *__restrict__ v, int n, double denom, double *__restrict__ out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += v[i];
        *out = s / denom;
    }
}

// Adam (Kingma & Ba) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ grad, int n, float lr, float b1, float b2, float eps, float c1,
                       float c2, __nv_bfloat16 *__restrict__ pb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gr = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gr;
    const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float *__restrict__ p, int n, __nv_bfloat16 *__restrict__ pb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

// ------------------------------------------------------------- features
// Per-sample scale S = sqrt(mean over cells and moments of phi1^2), floored by
// the source scale, so that the network sees O(1) inputs at every flux level.
// Two kernels, no workspace: k_scale_part spreads each sample over many blocks
// (block i sums the squares of a fixed contiguous slice of phi1 and of qfeat in
// FP64) and parks the two partial sums as 32-bit word pairs at the head of the
// sample's block of `in`, which k_features overwrites afterwards; k_scale_final
// adds the partials of each sample in a fixed order.  Deterministic.
constexpr int SC_T = 256;          // threads of the scale kernels
constexpr int SC_PER_BLOCK = 2048; // phi1 elements per partial-sum block

inline int scale_blocks(int J)
{
    const long long n = (4LL * J + SC_PER_BLOCK - 1) / SC_PER_BLOCK;
    return (int)(n < 1 ? 1 : (n > 1024 ? 1024 : n));  // 4 words per block fit in 13 J floats
}

// fixed-order sum of one double per thread over a block of SC_T threads (thread 0 gets it)
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < SC_T / 32; ++w) r += sh[w];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SC_T) k_scale_part(const double *__restrict__ phi1, const float *__restrict__ qfeat,
                                                     int J, int nblk, float *__restrict__ in)
{
    __shared__ double sh[SC_T / 32];
    const int b = blockIdx.y, i = blockIdx.x;
    const long long n1 = 4LL * J;
    const long long lo1 = n1 * i / nblk, hi1 = n1 * (i + 1) / nblk;
    const long long lo2 = (long long)J * i / nblk, hi2 = (long long)J * (i + 1) / nblk;
    const double *p = phi1 + (size_t)b * n1;
    const float *q = qfeat + (size_t)b * J;
    double a = 0.0, c = 0.0;
#pragma unroll 4
    for (long long e = lo1 + threadIdx.x; e < hi1; e += SC_T) {
        const double v = p[e];
        a += v * v;
    }
    for (long long e = lo2 + threadIdx.x; e < hi2; e += SC_T) {
        const double v = q[e];
        c += v * v;
    }
    a = block_sum(a, sh);
    c = block_sum(c, sh);
    if (threadIdx.x == 0) {
        unsigned *wd = reinterpret_cast<unsigned *>(in + (size_t)b * 13 * J) + 4 * i;
        const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
        const unsigned long long uc = (unsigned long long)__double_as_longlong(c);
        wd[0] = (unsigned)ua;
        wd[1] = (unsigned)(ua >> 32);
        wd[2] = (unsigned)uc;
        wd[3] = (unsigned)(uc >> 32);
    }
}

__global__ void __launch_bounds__(SC_T) k_scale_final(const float *__restrict__ in, int J, int nblk,
                                                      float *__restrict__ scale)
{
    __shared__ double sh[SC_T / 32];
    const int b = blockIdx.x;
    const unsigned *wd = reinterpret_cast<const unsigned *>(in + (size_t)b * 13 * J);
    double a = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nblk; i += SC_T) {
        a += __longlong_as_double((long long)(((unsigned long long)wd[4 * i + 1] << 32) | wd[4 * i]));
        c += __longlong_as_double((long long)(((unsigned long long)wd[4 * i + 3] << 32) | wd[4 * i + 2]));
    }
    a = block_sum(a, sh);
    c = block_sum(c, sh);
    if (threadIdx.x == 0) {
        double s = sqrt(a / (4.0 * J));
        const double sqv = sqrt(c / J);
        if (s < sqv) s = sqv;
        if (!(s > 1e-30)) s = 1.0;
        scale[b] = (float)s;
    }
}

__global__ void k_features(const double *__restrict__ phi1, const double *__restrict__ phi2,
                           const float *__restrict__ stat, const float *__restrict__ qfeat,
                           const float *__restrict__ scale, int J, float *__restrict__ in)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (j >= J) return;
    const float inv = 1.f / scale[b];
    float *o = in + (size_t)b * 13 * J + j;
    const double *p1 = phi1 + ((size_t)b * J + j) * 4, *p2 = phi2 + ((size_t)b * J + j) * 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        o[(size_t)c * J] = (float)p1[c] * inv;
        o[(size_t)(4 + c) * J] = (float)(p1[c] - p2[c]) * inv;
    }
    const float *s = stat + ((size_t)b * J + j) * 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) o[(size_t)(8 + c) * J] = s[c];
    o[(size_t)12 * J] = qfeat[(size_t)b * J + j] * inv;
}

__global__ void k_targets(const double *__restrict__ phin, const double *__restrict__ phi1,
                          const float *__restrict__ scale, int J, float *__restrict__ tgt)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (j >= J) return;
    const float inv = 1.f / scale[b];
#pragma unroll
    for (int c = 0; c < 4; ++c)
        tgt[((size_t)b * 4 + c) * J + j] = (float)(phin[((size_t)b * J + j) * 4 + c] - phi1[((size_t)b * J + j) * 4 + c]) * inv;
}

// prediction phi_hat = phi1 + S * out, as double [B][J][4]
__global__ void k_predict(const double *__restrict__ phi1, const float *__restrict__ out,
                          const float *__restrict__ scale, int J, double *__restrict__ phat)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (j >= J) return;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        phat[((size_t)b * J + j) * 4 + c] =
            phi1[((size_t)b * J + j) * 4 + c] + (double)scale[b] * (double)out[((size_t)b * 4 + c) * J + j];
}

// ------------------------------------------------------------- workspace
struct Work {
    __nv_bfloat16 *wb;     // BF16 weights [NPARAM]
    unsigned char *pack;   // the fused inference kernel's parameter image [FPACK_BYTES]
    float *act[NL + 1];    // act[0] = input (caller's), act[l] = output of layer l
    float *g[2];           // gradient ping-pong [B][32][J]
    float *grad;           // [NPARAM]
    float *partial;        // [tiles][max layer params]
    double *lpart;         // loss partials
    double *loss;          // [1]
};

size_t workspace_layout(int B, int J, Work *w, char *base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += (bytes + 255) & ~(size_t)255;
        return p;
    };
    const size_t cells = (size_t)B * J;
    const int tiles = B * ((J + TX - 1) / TX);
    int maxp = 0;
    for (int l = 0; l < NL; ++l) maxp = layer_w(l) + CH[l + 1] > maxp ? layer_w(l) + CH[l + 1] : maxp;
    Work tmp{};
    Work &o = w ? *w : tmp;
    o.wb = (__nv_bfloat16 *)take(sizeof(__nv_bfloat16) * NPARAM);
    o.pack = (unsigned char *)take(FPACK_BYTES);
    o.act[0] = nullptr;
    for (int l = 1; l <= NL; ++l) o.act[l] = (float *)take(sizeof(float) * cells * CH[l]);
    o.g[0] = (float *)take(sizeof(float) * cells * MAXC);
    o.g[1] = (float *)take(sizeof(float) * cells * MAXC);
    o.grad = (float *)take(sizeof(float) * NPARAM);
    o.partial = (float *)take(sizeof(float) * (size_t)tiles * maxp);
    o.lpart = (double *)take(sizeof(double) * 1024);
    o.loss = (double *)take(sizeof(double));
    return off;
}

template <int L>
void launch_fwd(const Work &w, const float *bias, int B, int J, cudaStream_t s)
{
    constexpr int CI = CH[L], CO = CH[L + 1];
    const dim3 grid((J + TX - 1) / TX, B);
    k_conv<CI, CO, (L < NL - 1), false><<<grid, TX, 0, s>>>(w.act[L], nullptr, w.wb + layer_off(L), bias, w.act[L + 1], J);
}

void forward_all(const Work &w, const float *params, int B, int J, cudaStream_t s)
{
    launch_fwd<0>(w, params + layer_off(0) + layer_w(0), B, J, s);
    launch_fwd<1>(w, params + layer_off(1) + layer_w(1), B, J, s);
    launch_fwd<2>(w, params + layer_off(2) + layer_w(2), B, J, s);
    launch_fwd<3>(w, params + layer_off(3) + layer_w(3), B, J, s);
    launch_fwd<4>(w, params + layer_off(4) + layer_w(4), B, J, s);
}

// Inference: the five layers on the tensor cores, activations ping-ponging
// between two buffers a and b (layer 0 reads in, the last layer writes out).
void forward_mma(const __nv_bfloat16 *wb, const float *params, const float *in, float *a, float *b, float *out, int B,
                 int J, cudaStream_t s)
{
    const dim3 grid((J + TX - 1) / TX, B);
    k_conv_mma<13, 32, true><<<grid, TX, 0, s>>>(in, wb + layer_off(0), params + layer_off(0) + layer_w(0), a, J);
    k_conv_mma<32, 32, true><<<grid, TX, 0, s>>>(a, wb + layer_off(1), params + layer_off(1) + layer_w(1), b, J);
    k_conv_mma<32, 32, true><<<grid, TX, 0, s>>>(b, wb + layer_off(2), params + layer_off(2) + layer_w(2), a, J);
    k_conv_mma<32, 32, true><<<grid, TX, 0, s>>>(a, wb + layer_off(3), params + layer_off(3) + layer_w(3), b, J);
    k_conv_mma<32, 4, false><<<grid, TX, 0, s>>>(b, wb + layer_off(4), params + layer_off(4) + layer_w(4), out, J);
}

// Inference in one kernel: the parameter image, then the fused layers on a
// persistent grid of two CTAs per SM.
int forward_fused(unsigned char *pack, const float *params, const float *in, float *out, int B, int J, cudaStream_t s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(k_forward_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, FSMEM) != cudaSuccess)
        return 3;
    k_pack_fused<<<dim3((FPACK_MAX_LAYER + 255) / 256, NL), 256, 0, s>>>(params, pack);
    const long long tiles = (long long)B * ((J + FOUT - 1) / FOUT);
    const int grid = (int)(tiles < 2LL * sms ? tiles : 2LL * sms);
    k_forward_fused<<<grid, FTHREADS, FSMEM, s>>>(pack, in, out, B, J);
    return 0;
}

// Backward of layer L: gin = gradient w.r.t. the layer's output (before the
// ReLU mask), produces the parameter gradient and (L > 0) the gradient w.r.t.
// the layer's input in gout.
template <int L>
void launch_bwd(const Work &w, const float *gin, float *gout, int B, int J, cudaStream_t s)
{
    constexpr int CI = CH[L], CO = CH[L + 1];
    constexpr bool RELU = L < NL - 1;
    const dim3 grid((J + TX - 1) / TX, B);
    const int tiles = grid.x * grid.y;
    k_wgrad<CI, CO, RELU><<<grid, 256, 0, s>>>(w.act[L], gin, w.act[L + 1], w.partial, J);
    const int n = CO * CI * KW + CO;
    k_reduce_partials<<<(n + 255) / 256, 256, 0, s>>>(w.partial, tiles, n, w.grad + layer_off(L));
    if constexpr (L > 0)  // data gradient: transposed, flipped conv of the masked gradient
        k_conv<CO, CI, false, true><<<grid, TX, 0, s>>>(gin, RELU ? w.act[L + 1] : nullptr, w.wb + layer_off(L),
                                                         nullptr, gout, J);
}

int loss_grad(const float *params, const float *in, const float *tgt, int B, int J, void *ws, size_t ws_bytes,
              double *loss_host, float *grad_out, cudaStream_t s)
{
    Work w{};
    if (workspace_layout(B, J, nullptr, nullptr) > ws_bytes) return 1;
    workspace_layout(B, J, &w, (char *)ws);
    w.act[0] = const_cast<float *>(in);
    k_to_bf16<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, NPARAM, w.wb);
    forward_all(w, params, B, J, s);
    const size_t n = (size_t)B * 4 * J;
    const int nb = 256;
    k_mse<<<nb, 256, 0, s>>>(w.act[NL], tgt, n, w.g[0], w.lpart);
    k_sum_doubles<<<1, 32, 0, s>>>(w.lpart, nb, 1.0 * n, w.loss);
    launch_bwd<4>(w, w.g[0], w.g[1], B, J, s);
    launch_bwd<3>(w, w.g[1], w.g[0], B, J, s);
    launch_bwd<2>(w, w.g[0], w.g[1], B, J, s);
    launch_bwd<1>(w, w.g[1], w.g[0], B, J, s);
    launch_bwd<0>(w, w.g[0], w.g[1], B, J, s);
    if (grad_out) cudaMemcpyAsync(grad_out, w.grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, s);
    if (loss_host) {
        cudaMemcpyAsync(loss_host, w.loss, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// ------------------------------------------------- allocation-free inference
// Scratch of oci_nn_forward_noalloc: BF16 weights and two activation buffers
// of 32 channels x OCI_NN_NOALLOC_MAX_CELLS cells, in one file-scope device
// array that every GPU loading this library keeps until the process exits.
constexpr size_t kStaticWeightBytes = ((size_t)NPARAM * 2 + 255) & ~(size_t)255;
constexpr size_t kStaticActFloats = (size_t)MAXC * OCI_NN_NOALLOC_MAX_CELLS;
static __device__ __align__(256) unsigned char g_nn_scratch[kStaticWeightBytes + 2 * kStaticActFloats * 4];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
struct ScratchSlot {
    unsigned long long ctx_id;  // context the address belongs to (0: none yet)
    void *addr;
};
ScratchSlot g_scratch[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (driver entry points
// resolved through the runtime, so the library does not link libcuda).
int current_context_id(unsigned long long *id)
{
    typedef int (*get_current_t)(void **);
    typedef int (*get_id_t)(void *, unsigned long long *);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
            qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return 3;
        get_current = (get_current_t)a;
        get_id = (get_id_t)b;
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, id) != 0) return 3;
    return 0;
}

// Device address of g_nn_scratch on the current device (the host-side symbol
// is only a stand-in).  Looked up with that device current, once per device
// and context: a reset of the device's primary context (cudaDeviceReset)
// reloads the module, and the next call looks the address up again.
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 3;
    if (dev < 0 || dev >= kMaxDevices) return 1;
    if (cudaSetDevice(dev) != cudaSuccess) return 3;  // makes the device's primary context current
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long ctx = 0;
    if (current_context_id(&ctx)) return 3;
    ScratchSlot &s = g_scratch[dev];
    if (!s.addr || s.ctx_id != ctx) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_nn_scratch) != cudaSuccess || !p) return 3;
        s.addr = p;
        s.ctx_id = ctx;
    }
    *out = s.addr;
    return 0;
}

// ------------------------------------------------------------ training driver
// Minibatch gather of oci_nn_train: sample k = t S + (n - 1) of the list idx
// (entries [b0, b0 + B)) -> phi_n, phi_{n-1}, phi_{max(n-2, 0)} [B][J][4]
// (double), stat [B][J][4] and qfeat [B][J].
__global__ void k_gather(const double *__restrict__ phi, const float *__restrict__ stat,
                         const float *__restrict__ qfeat, const int *__restrict__ idx, int b0, int S, int J,
                         double *__restrict__ phin, double *__restrict__ phi1, double *__restrict__ phi2,
                         float *__restrict__ st_b, float *__restrict__ qf_b)
{
    const int b = blockIdx.y;
    const int k = idx[b0 + b];
    const int t = k / S, n = k % S + 1;
    const size_t JB = (size_t)J * 4;
    const double *base = phi + (size_t)t * (S + 1) * JB;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < J * 4; e += gridDim.x * blockDim.x) {
        phin[b * JB + e] = base[(size_t)n * JB + e];
        phi1[b * JB + e] = base[(size_t)(n - 1) * JB + e];
        phi2[b * JB + e] = base[(size_t)(n >= 2 ? n - 2 : 0) * JB + e];
        st_b[b * JB + e] = stat[(size_t)t * JB + e];
        if (e < J) qf_b[(size_t)b * J + e] = qfeat[(size_t)t * J + e];
    }
}

// Vigna's splitmix64 finaliser (the generator the training order is defined by).
inline uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void shuffle_round(std::vector<int> &a, uint64_t seed, uint64_t r)
{
    for (size_t i = a.size(); i-- > 1;) {
        const uint64_t j = splitmix64(seed + (r << 32) + i) % (uint64_t)(i + 1);
        std::swap(a[i], a[j]);
    }
}

}  // namespace ocinn

using namespace ocinn;

extern "C" {

int32_t oci_nn_param_count(void) { return NPARAM; }

size_t oci_nn_workspace_bytes(int32_t batch, int32_t n_cells)
{
    if (batch < 1 || n_cells < 1) return 0;
    return workspace_layout(batch, n_cells, nullptr, nullptr);
}

int oci_nn_features(const double *phi1, const double *phi2, const float *stat, const float *qfeat, int32_t batch,
                    int32_t n_cells, float *in, float *scale, void *stream)
{
    if (!phi1 || !phi2 || !stat || !qfeat || !in || !scale || batch < 1 || n_cells < 1) return 1;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = scale_blocks(n_cells);
    k_scale_part<<<dim3(nblk, batch), SC_T, 0, s>>>(phi1, qfeat, n_cells, nblk, in);
    k_scale_final<<<batch, SC_T, 0, s>>>(in, n_cells, nblk, scale);
    k_features<<<dim3((n_cells + 255) / 256, batch), 256, 0, s>>>(phi1, phi2, stat, qfeat, scale, n_cells, in);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int oci_nn_targets(const double *phin, const double *phi1, const float *scale, int32_t batch, int32_t n_cells,
                   float *tgt, void *stream)
{
    if (!phin || !phi1 || !scale || !tgt || batch < 1 || n_cells < 1) return 1;
    k_targets<<<dim3((n_cells + 255) / 256, batch), 256, 0, (cudaStream_t)stream>>>(phin, phi1, scale, n_cells, tgt);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int oci_nn_forward(const float *params, const float *in, int32_t batch, int32_t n_cells, float *out, void *ws,
                   size_t ws_bytes, void *stream)
{
    if (!params || !in || !out || !ws || batch < 1 || n_cells < 1) return 1;
    Work w{};
    if (workspace_layout(batch, n_cells, nullptr, nullptr) > ws_bytes) return 1;
    workspace_layout(batch, n_cells, &w, (char *)ws);
    if (forward_fused(w.pack, params, in, out, batch, n_cells, (cudaStream_t)stream)) return 3;
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int oci_nn_predict(const double *phi1, const float *out, const float *scale, int32_t batch, int32_t n_cells,
                   double *phat, void *stream)
{
    if (!phi1 || !out || !scale || !phat || batch < 1 || n_cells < 1) return 1;
    k_predict<<<dim3((n_cells + 255) / 256, batch), 256, 0, (cudaStream_t)stream>>>(phi1, out, scale, n_cells, phat);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int oci_nn_loss_grad(const float *params, const float *in, const float *tgt, int32_t batch, int32_t n_cells,
                     float *grad, double *loss, void *ws, size_t ws_bytes, void *stream)
{
    if (!params || !in || !tgt || batch < 1 || n_cells < 1 || !ws) return 1;
    return loss_grad(params, in, tgt, batch, n_cells, ws, ws_bytes, loss, grad, (cudaStream_t)stream);
}

int oci_nn_train_step(float *params, float *adam_m, float *adam_v, int32_t step, float lr, const float *in,
                      const float *tgt, int32_t batch, int32_t n_cells, double *loss, void *ws, size_t ws_bytes,
                      void *stream)
{
    if (!params || !adam_m || !adam_v || step < 1 || !in || !tgt || batch < 1 || n_cells < 1 || !ws) return 1;
    cudaStream_t s = (cudaStream_t)stream;
    const int rc = loss_grad(params, in, tgt, batch, n_cells, ws, ws_bytes, loss, nullptr, s);
    if (rc) return rc;
    Work w{};
    workspace_layout(batch, n_cells, &w, (char *)ws);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, adam_m, adam_v, w.grad, NPARAM, lr, b1, b2, 1e-8f, c1, c2,
                                                 w.wb);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int oci_nn_train(const oci_nn_train_cfg *cfg, float *weights_out, oci_nn_train_stats *stats)
{
    if (!cfg || !weights_out || !cfg->phi || !cfg->stat || !cfg->qfeat) return 1;
    const int T = cfg->n_traj, S = cfg->n_steps, J = cfg->n_cells, B = cfg->batch;
    if (T < 1 || S < 1 || J < 1 || B < 1 || cfg->epochs < 1 || !(cfg->val_frac >= 0.f && cfg->val_frac < 1.f) ||
        (int64_t)T * S > (int64_t)1 << 30)
        return 1;
    cudaStream_t s = (cudaStream_t)cfg->stream;
    const int n_all = T * S;
    const int n_val = (int)std::floor((double)n_all * cfg->val_frac);
    const int n_tr = n_all - n_val;
    if (n_tr < B) return 1;  // not one full minibatch
    std::vector<int> all(n_all);
    for (int k = 0; k < n_all; ++k) all[k] = k;
    shuffle_round(all, cfg->seed, 0);
    std::vector<int> val(all.begin(), all.begin() + n_val), tr(all.begin() + n_val, all.end());
    // device buffers: one allocation
    const size_t cells = (size_t)B * J;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) & ~(size_t)255; return o; };
    const size_t o_p = take(4 * (size_t)NPARAM), o_m = take(4 * (size_t)NPARAM), o_v = take(4 * (size_t)NPARAM);
    const size_t o_idx = take(4 * (size_t)n_all);
    const size_t o_phin = take(8 * cells * 4), o_phi1 = take(8 * cells * 4), o_phi2 = take(8 * cells * 4);
    const size_t o_st = take(4 * cells * 4), o_qf = take(4 * cells), o_in = take(4 * cells * 13),
                 o_tgt = take(4 * cells * 4), o_sc = take(4 * (size_t)B);
    const size_t ws_bytes = workspace_layout(B, J, nullptr, nullptr);
    const size_t o_ws = take(ws_bytes);
    char *mem = nullptr;
    if (cudaMalloc(&mem, off) != cudaSuccess) return 2;
    float *p = (float *)(mem + o_p), *m = (float *)(mem + o_m), *v = (float *)(mem + o_v);
    int *d_idx = (int *)(mem + o_idx);
    double *phin = (double *)(mem + o_phin), *phi1 = (double *)(mem + o_phi1), *phi2 = (double *)(mem + o_phi2);
    float *st_b = (float *)(mem + o_st), *qf_b = (float *)(mem + o_qf), *inp = (float *)(mem + o_in),
          *tgt = (float *)(mem + o_tgt), *sc = (float *)(mem + o_sc);
    void *ws = mem + o_ws;
    int rc = 0;
    auto cuda_ok = [&](cudaError_t e) { if (e != cudaSuccess && !rc) rc = 3; return rc == 0; };
    if (cfg->init_params) {
        cuda_ok(cudaMemcpyAsync(p, cfg->init_params, 4 * (size_t)NPARAM, cudaMemcpyDeviceToDevice, s));
    } else {
        std::vector<float> h(NPARAM, 0.f);
        for (int l = 0; l < NL; ++l) {
            const double bound = std::sqrt(6.0 / (KW * CH[l]));
            for (int i = layer_off(l); i < layer_off(l) + layer_w(l); ++i) {
                const double u = (double)(splitmix64((cfg->seed ^ 0x5DEECE66Dull) + (uint64_t)i) >> 11) *
                                 (1.0 / 9007199254740992.0);
                h[i] = (float)(bound * (2.0 * u - 1.0));
            }
        }
        cuda_ok(cudaMemcpy(p, h.data(), 4 * (size_t)NPARAM, cudaMemcpyHostToDevice));
    }
    cuda_ok(cudaMemsetAsync(m, 0, 4 * (size_t)NPARAM, s));
    cuda_ok(cudaMemsetAsync(v, 0, 4 * (size_t)NPARAM, s));
    const dim3 ggrid((J * 4 + 255) / 256 < 64 ? (J * 4 + 255) / 256 : 64, 1);
    auto batch_inputs = [&](int b0, int nb) {
        k_gather<<<dim3(ggrid.x, nb), 256, 0, s>>>(cfg->phi, cfg->stat, cfg->qfeat, d_idx, b0, S, J, phin, phi1, phi2,
                                                    st_b, qf_b);
        if (!cuda_ok(cudaGetLastError())) return false;
        if (oci_nn_features(phi1, phi2, st_b, qf_b, nb, J, inp, sc, s) || oci_nn_targets(phin, phi1, sc, nb, J, tgt, s)) {
            if (!rc) rc = 3;
            return false;
        }
        return true;
    };
    int step = 0, ep = 0;
    double train_loss = NAN, val_loss = NAN;
    for (ep = 0; ep < cfg->epochs && !rc; ++ep) {
        shuffle_round(tr, cfg->seed, (uint64_t)ep + 1);
        if (!cuda_ok(cudaMemcpyAsync(d_idx, tr.data(), 4 * (size_t)n_tr, cudaMemcpyHostToDevice, s))) break;
        const float lr_ep = (float)(cfg->lr * 0.5 * (1.0 + std::cos(3.14159265358979323846 * ep / cfg->epochs)));
        double lsum = 0.0;
        int lcnt = 0;
        for (int b0 = 0, bi = 0; b0 + B <= n_tr && !rc; b0 += B, ++bi) {
            if (!batch_inputs(b0, B)) break;
            ++step;
            double l = 0.0;
            const bool want = bi % 50 == 0;
            if (oci_nn_train_step(p, m, v, step, lr_ep, inp, tgt, B, J, want ? &l : nullptr, ws, ws_bytes, s)) {
                rc = 3;
                break;
            }
            if (want) { lsum += l; ++lcnt; }
        }
        train_loss = lcnt ? lsum / lcnt : NAN;
        if (rc) break;
        // validation: the held-out samples in minibatches of min(batch, n_val)
        if (n_val > 0) {
            const int vb = n_val < B ? n_val : B;
            if (!cuda_ok(cudaMemcpyAsync(d_idx, val.data(), 4 * (size_t)n_val, cudaMemcpyHostToDevice, s))) break;
            double vs = 0.0;
            int vc = 0;
            for (int b0 = 0; b0 + vb <= n_val && !rc; b0 += vb) {
                if (!batch_inputs(b0, vb)) break;
                double l = 0.0;
                if (oci_nn_loss_grad(p, inp, tgt, vb, J, nullptr, &l, ws, ws_bytes, s)) { rc = 3; break; }
                vs += l;
                ++vc;
            }
            val_loss = vc ? vs / vc : NAN;
        }
    }
    if (!rc) cuda_ok(cudaMemcpyAsync(weights_out, p, 4 * (size_t)NPARAM, cudaMemcpyDeviceToDevice, s));
    if (!rc) cuda_ok(cudaStreamSynchronize(s));
    cudaStreamSynchronize(s);
    cudaFree(mem);
    if (stats) {
        stats->epochs_done = ep;
        stats->steps_done = step;
        stats->n_train = n_tr;
        stats->n_val = n_val;
        stats->train_loss = train_loss;
        stats->val_loss = val_loss;
    }
    return rc;
}

int oci_nn_forward_noalloc(const float *params, const float *in, int32_t n_cells, float *out, void *stream)
{
    if (!params || !in || !out || n_cells < 1) return 1;
    if (n_cells > OCI_NN_NOALLOC_MAX_CELLS) return 1;  // beyond the static scratch
    void *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc) return rc;
    __nv_bfloat16 *wb = (__nv_bfloat16 *)scratch;
    float *a = (float *)((char *)scratch + kStaticWeightBytes);
    float *b = a + kStaticActFloats;
    cudaStream_t s = (cudaStream_t)stream;
    k_to_bf16<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, NPARAM, wb);
    forward_mma(wb, params, in, a, b, out, 1, n_cells, s);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // extern "C"
