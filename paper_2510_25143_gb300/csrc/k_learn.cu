// Learned predictor (an extension; the paper has none): whole-slice inference
// with the compressor's own tile code, and training on the GPU (forward,
// backward and Adam kernels).
//
// Training layout: every activation is a float32 [n][C][H][W] plane stack.
// The forward convolutions use the parameters rounded to bfloat16 and form
// each output as the same fused multiply-add chain as inference (bias, then
// input channel, ky, kx), so the training forward pass and the codec agree
// bit for bit.  Gradients run through the rounding as through the identity
// and are accumulated in float32: per-block partial sums over fixed tile
// sets, then a fixed-order reduction, so a step is deterministic.
#include <cmath>

#include "cpt_dev.cuh"
#include "cpt_internal.h"

namespace cpt {

// ---------------------------------------------------------------------------
// inference over a whole slice: one warp per 8 x 8 tile
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) net_predict_kernel(NetDev nd, const int2* __restrict__ prev, int H, int W,
                                                         int2* __restrict__ out) {
    __shared__ NetScratch<8> s;
    const int r0 = blockIdx.y * 8, c0 = blockIdx.x * 8;
    auto pv = [&](int i, int j) -> int2 {
        return (i >= 0 && i < H && j >= 0 && j < W) ? prev[(size_t)i * W + j] : make_int2(0, 0);
    };
    auto o = [&](int li, int lj, int2 p) { out[(size_t)(r0 + li) * W + c0 + lj] = p; };
    net_tile<8>(nd, s, r0, c0, H, W, pv, o);
}

void launch_net_predict(const NetDev& nd, const int32_t* prev, int H, int W, int32_t* out, cudaStream_t s) {
    dim3 grid((W + 7) / 8, (H + 7) / 8);
    net_predict_kernel<<<grid, 32, 0, s>>>(nd, reinterpret_cast<const int2*>(prev), H, W,
                                           reinterpret_cast<int2*>(out));
}

// ---------------------------------------------------------------------------
// training
// ---------------------------------------------------------------------------
constexpr int kTile = 16;             // output tile side of the convolution kernels
constexpr int kHalo = kTile + 2;      // input tile side

__device__ __forceinline__ float bf16_round(float x) {
    // round to nearest even on the upper 16 bits (NaN stays NaN)
    const unsigned b = __float_as_uint(x);
    if ((b & 0x7F800000u) == 0x7F800000u && (b & 0x007FFFFFu)) return x;
    const unsigned r = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    return __uint_as_float(r);
}

// x0 = prev * 2^-23 and the target d = clamp((next - prev) * 2^-23, -2, 2),
// both [n][2][H][W].
__global__ void __launch_bounds__(256) net_inputs_kernel(const int2* __restrict__ prev, const int2* __restrict__ next,
                                                         size_t n, size_t HW, float* __restrict__ x0,
                                                         float* __restrict__ d) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n * HW; v += (size_t)gridDim.x * blockDim.x) {
        const size_t b = v / HW, p = v - b * HW;
        const int2 a = prev[v], c = next[v];
        const int av[2] = {a.x, a.y}, cv[2] = {c.x, c.y};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            x0[(b * 2 + k) * HW + p] = __fmul_rn(__int2float_rn(av[k]), 1.1920928955078125e-07f);
            float t = __fmul_rn(__ll2float_rn((long long)cv[k] - (long long)av[k]), 1.1920928955078125e-07f);
            d[(b * 2 + k) * HW + p] = t < -2.0f ? -2.0f : (t > 2.0f ? 2.0f : t);
        }
    }
}

// Master parameters (model layout) -> the bfloat16-rounded device layouts:
// forward weights transposed to [ci][k][co] (NetDev), backward-input weights
// wb[co][k'][ci] = w[co][ci][8 - k'] (the transposed, flipped kernel), the
// bfloat16 bits of the model.
__global__ void __launch_bounds__(256) net_prep_weights_kernel(const float* __restrict__ P, NetTrainPtrs o) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kNetParams) return;
    const float r = bf16_round(P[j]);
    o.bits[j] = (uint16_t)(__float_as_uint(r) >> 16);
    // locate j in the model layout: w1 b1 w2 b2 w3 b3
    int base = 0, cin = 2, cout = kNetC, layer = 0;
    int rel = j;
    const int wsz[3] = {kNetW1, kNetW2, kNetW3}, cins[3] = {2, kNetC, kNetC}, couts[3] = {kNetC, kNetC, 2};
    for (layer = 0; layer < 3; ++layer) {
        cin = cins[layer];
        cout = couts[layer];
        if (rel < wsz[layer] + cout) break;
        rel -= wsz[layer] + cout;
        base += wsz[layer] + cout;
    }
    if (rel >= wsz[layer]) {  // bias
        o.fwd[base + wsz[layer] + (rel - wsz[layer])] = r;
        return;
    }
    const int co = rel / (cin * 9), ci = (rel / 9) % cin, k = rel % 9;
    o.fwd[base + (ci * 9 + k) * cout + co] = r;
    if (layer == 1) o.bwd2[(co * 9 + (8 - k)) * cin + ci] = r;
    if (layer == 2) o.bwd3[(co * 9 + (8 - k)) * cin + ci] = r;
}

// 3x3 'same' convolution with zero padding, one thread per output position of
// a 16 x 16 tile, all COUT outputs in registers:
//   out[co][p] = epi(bias[co] + sum over (ci, ky, kx) of w * in[ci][p + (ky-1, kx-1)])
// wt: [CIN][9][COUT]; bias may be null (0).  EPI 0: none, 1: ReLU, 2: keep where
// mask[co][p] > 0 else 0 (the ReLU derivative of the layer below).
template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(256) conv3x3_kernel(const float* __restrict__ in, const float* __restrict__ wt,
                                                      const float* __restrict__ bias, const float* __restrict__ mask,
                                                      float* __restrict__ out, int H, int W) {
    extern __shared__ __align__(16) float sh[];
    float* s_w = sh;                       // CIN * 9 * COUT
    float* s_in = sh + CIN * 9 * COUT;     // CIN * 18 * 18
    const int tid = threadIdx.x;
    const int b = blockIdx.z, i0 = blockIdx.y * kTile, j0 = blockIdx.x * kTile;
    const size_t HW = (size_t)H * W;
    for (int k = tid; k < CIN * 9 * COUT; k += 256) s_w[k] = wt[k];
    for (int k = tid; k < CIN * kHalo * kHalo; k += 256) {
        const int ci = k / (kHalo * kHalo), r = (k / kHalo) % kHalo, c = k % kHalo;
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        s_in[k] = (i >= 0 && i < H && j >= 0 && j < W) ? in[((size_t)b * CIN + ci) * HW + (size_t)i * W + j] : 0.0f;
    }
    __syncthreads();
    const int ty = tid / kTile, tx = tid % kTile;
    const int i = i0 + ty, j = j0 + tx;
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bias ? bias[co] : 0.0f;
#pragma unroll 1
    for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float v = s_in[(ci * kHalo + ty + k / 3) * kHalo + tx + k % 3];
            const float* wp = s_w + (ci * 9 + k) * COUT;
            if constexpr (COUT % 4 == 0) {
#pragma unroll
                for (int co = 0; co < COUT; co += 4) {
                    const float4 w4 = *reinterpret_cast<const float4*>(wp + co);
                    acc[co] = __fmaf_rn(w4.x, v, acc[co]);
                    acc[co + 1] = __fmaf_rn(w4.y, v, acc[co + 1]);
                    acc[co + 2] = __fmaf_rn(w4.z, v, acc[co + 2]);
                    acc[co + 3] = __fmaf_rn(w4.w, v, acc[co + 3]);
                }
            } else {
#pragma unroll
                for (int co = 0; co < COUT; ++co) acc[co] = __fmaf_rn(wp[co], v, acc[co]);
            }
        }
    }
    if (i >= H || j >= W) return;
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
        const size_t o = ((size_t)b * COUT + co) * HW + (size_t)i * W + j;
        float r = acc[co];
        if (EPI == 1) r = r > 0.0f ? r : 0.0f;
        if (EPI == 2) r = mask[o] > 0.0f ? r : 0.0f;
        out[o] = r;
    }
}

// Loss and its gradient: with m = n * H * W * 2 terms,
//   loss = (1/m) sum (y - d)^2,  gy = 2 (y - d) / m   (written over y).
// Per-block partial sums of the loss (double) go to part[blockIdx.x].
__global__ void __launch_bounds__(256) net_loss_kernel(float* __restrict__ y, const float* __restrict__ d, size_t m,
                                                       float inv_m, double* __restrict__ part) {
    __shared__ double red[8];
    double acc = 0.0;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < m; v += (size_t)gridDim.x * blockDim.x) {
        const float e = __fsub_rn(y[v], d[v]);
        acc += (double)e * (double)e;
        y[v] = __fmul_rn(__fmul_rn(2.0f, e), inv_m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void net_loss_finish_kernel(const double* __restrict__ part, int nb, double inv_m, float* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += part[k];
    *out = (float)(s * inv_m);
}

// Weight and bias gradients of one layer:
//   gw[co][ci][ky][kx] = sum over (b, p) of gout[b][co][p] * in[b][ci][p + (ky-1, kx-1)]
//   gb[co]             = sum over (b, p) of gout[b][co][p]
// Each block walks a fixed set of 16 x 16 tiles (tile = blockIdx.x + k *
// gridDim.x) and writes its sums to part[blockIdx.x][COUT*CIN*9 + COUT] (the
// layer's model layout).  A thread owns CP output channels x 9 taps of one
// input channel; G groups of threads split a tile's positions.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) wgrad_kernel(const float* __restrict__ in, const float* __restrict__ gout, int n,
                                                    int H, int W, float* __restrict__ part) {
    constexpr int CP = COUT < 4 ? COUT : 4;
    constexpr int NQ = COUT / CP;
    constexpr int NW = CIN * NQ;
    constexpr int G = 256 / NW;
    static_assert(NW * G == 256, "thread split");
    constexpr int REC = COUT * CIN * 9 + COUT;
    extern __shared__ __align__(16) float sh[];
    float* s_in = sh;                              // CIN * 18 * 18
    float* s_g = sh + CIN * kHalo * kHalo;         // [256][COUT]
    const int tid = threadIdx.x;
    const int item = tid % NW, g = tid / NW;
    const int ci = item / NQ, cq = item % NQ;
    const size_t HW = (size_t)H * W;
    const int tx_n = (W + kTile - 1) / kTile, ty_n = (H + kTile - 1) / kTile;
    const long long ntiles = (long long)tx_n * ty_n * n;
    float acc[CP][9], bacc[CP];
#pragma unroll
    for (int c = 0; c < CP; ++c) {
        bacc[c] = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[c][k] = 0.0f;
    }
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = (int)(tile / ((long long)tx_n * ty_n));
        const int rem = (int)(tile % ((long long)tx_n * ty_n));
        const int i0 = (rem / tx_n) * kTile, j0 = (rem % tx_n) * kTile;
        __syncthreads();
        for (int k = tid; k < CIN * kHalo * kHalo; k += 256) {
            const int c = k / (kHalo * kHalo), r = (k / kHalo) % kHalo, cc = k % kHalo;
            const int i = i0 - 1 + r, j = j0 - 1 + cc;
            s_in[k] = (i >= 0 && i < H && j >= 0 && j < W) ? in[((size_t)b * CIN + c) * HW + (size_t)i * W + j] : 0.0f;
        }
        for (int k = tid; k < COUT * 256; k += 256) {
            const int co = k / 256, p = k % 256;
            const int i = i0 + p / kTile, j = j0 + p % kTile;
            s_g[p * COUT + co] = (i < H && j < W) ? gout[((size_t)b * COUT + co) * HW + (size_t)i * W + j] : 0.0f;
        }
        __syncthreads();
        for (int p = g; p < 256; p += G) {
            const int py = p / kTile, px = p % kTile;
            float gv[CP];
#pragma unroll
            for (int c = 0; c < CP; ++c) gv[c] = s_g[p * COUT + cq * CP + c];
            const float* ip = s_in + (ci * kHalo + py) * kHalo + px;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float v = ip[(k / 3) * kHalo + k % 3];
#pragma unroll
                for (int c = 0; c < CP; ++c) acc[c][k] = __fmaf_rn(gv[c], v, acc[c][k]);
            }
            if (ci == 0) {
#pragma unroll
                for (int c = 0; c < CP; ++c) bacc[c] = __fadd_rn(bacc[c], gv[c]);
            }
        }
    }
    // reduce the G groups in shared memory (fixed order), then write the record
    __syncthreads();
    float* s_r = sh;  // [G][REC]
    for (int k = tid; k < G * REC; k += 256) s_r[k] = 0.0f;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < CP; ++c) {
        const int co = cq * CP + c;
#pragma unroll
        for (int k = 0; k < 9; ++k) s_r[g * REC + (co * CIN + ci) * 9 + k] = acc[c][k];
        if (ci == 0) s_r[g * REC + COUT * CIN * 9 + co] = bacc[c];
    }
    __syncthreads();
    for (int k = tid; k < REC; k += 256) {
        float s = s_r[k];
        for (int q = 1; q < G; ++q) s = __fadd_rn(s, s_r[q * REC + k]);
        part[(size_t)blockIdx.x * REC + k] = s;
    }
}

// out[k] = sum over blocks (in order) of part[blk][k]
__global__ void __launch_bounds__(256) part_reduce_kernel(const float* __restrict__ part, int nblk, int rec,
                                                          float* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rec) return;
    float s = 0.0f;
    for (int b = 0; b < nblk; ++b) s = __fadd_rn(s, part[(size_t)b * rec + k]);
    out[k] = s;
}

// Adam (bias-corrected): c1 = 1 - beta1^t, c2 = 1 - beta2^t.
__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ P, float* __restrict__ m, float* __restrict__ v,
                                                   const float* __restrict__ g, int np, float lr, float b1, float b2,
                                                   float c1, float c2, float eps) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= np) return;
    const float gj = g[j];
    const float mj = __fadd_rn(__fmul_rn(b1, m[j]), __fmul_rn(__fsub_rn(1.0f, b1), gj));
    const float vj = __fadd_rn(__fmul_rn(b2, v[j]), __fmul_rn(__fsub_rn(1.0f, b2), __fmul_rn(gj, gj)));
    m[j] = mj;
    v[j] = vj;
    const float mh = __fdiv_rn(mj, c1), vh = __fdiv_rn(vj, c2);
    P[j] = __fsub_rn(P[j], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(__fsqrt_rn(vh), eps)));
}

// ---------------------------------------------------------------------------
// host side of one training step
// ---------------------------------------------------------------------------
template <typename K>
static cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int CIN, int COUT, int EPI>
static cudaError_t conv(const float* in, const float* wt, const float* bias, const float* mask, float* out, int n,
                        int H, int W, cudaStream_t s) {
    const size_t smem = sizeof(float) * (CIN * 9 * COUT + CIN * kHalo * kHalo);
    cudaError_t e = set_smem(conv3x3_kernel<CIN, COUT, EPI>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile, n);
    conv3x3_kernel<CIN, COUT, EPI><<<grid, 256, smem, s>>>(in, wt, bias, mask, out, H, W);
    return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t wgrad(const float* in, const float* gout, int n, int H, int W, int nblk, float* part,
                         float* out, cudaStream_t s) {
    constexpr int CP = COUT < 4 ? COUT : 4;
    constexpr int G = 256 / (CIN * (COUT / CP));
    constexpr int REC = COUT * CIN * 9 + COUT;
    const size_t tiles = sizeof(float) * (CIN * kHalo * kHalo + 256 * COUT);
    const size_t red = sizeof(float) * G * REC;
    const size_t smem = tiles > red ? tiles : red;
    cudaError_t e = set_smem(wgrad_kernel<CIN, COUT>, smem);
    if (e != cudaSuccess) return e;
    wgrad_kernel<CIN, COUT><<<nblk, 256, smem, s>>>(in, gout, n, H, W, part);
    part_reduce_kernel<<<(REC + 255) / 256, 256, 0, s>>>(part, nblk, REC, out);
    return cudaGetLastError();
}

size_t net_train_floats(int n, int H, int W) {
    const size_t P = (size_t)n * H * W;
    return P * (2 + 2 + kNetC + kNetC + 2 + kNetC);  // x0, d, h1, h2, y/gy, gh2 (gh1 reuses h2)
}

int net_wgrad_blocks(int n, int H, int W, int nsm) {
    const long long tiles = (long long)n * ((H + kTile - 1) / kTile) * ((W + kTile - 1) / kTile);
    const long long b = 2ll * nsm;
    return (int)(tiles < b ? tiles : b);
}

cudaError_t launch_net_inputs(const int32_t* prev, const int32_t* next, int n, int H, int W, float* x0, float* d,
                              cudaStream_t s) {
    net_inputs_kernel<<<1216, 256, 0, s>>>(reinterpret_cast<const int2*>(prev), reinterpret_cast<const int2*>(next),
                                           (size_t)n, (size_t)H * W, x0, d);
    return cudaGetLastError();
}

// One forward/backward pass at the master parameters P: writes the loss to
// *loss_dev and the gradient (model layout) to grad.  ws: net_train_floats()
// floats; part: nblk * (32*32*9 + 32) floats; lpart: 1216 doubles; w: the
// prepared weights.
cudaError_t net_train_pass(const float* P, float* ws, int n, int H, int W, int nblk, float* part, double* lpart,
                           const NetTrainPtrs& w, float* grad, float* loss_dev, cudaStream_t s) {
    const size_t HW = (size_t)H * W, Pn = (size_t)n * HW;
    float* x0 = ws;
    float* d = x0 + 2 * Pn;
    float* h1 = d + 2 * Pn;
    float* h2 = h1 + kNetC * Pn;
    float* y = h2 + kNetC * Pn;
    float* gh2 = y + 2 * Pn;
    float* gh1 = h2;  // h2 is dead once gh2 is formed
    net_prep_weights_kernel<<<(kNetParams + 255) / 256, 256, 0, s>>>(P, w);
    const float* w1t = w.fwd;
    const float* b1 = w1t + kNetW1;
    const float* w2t = b1 + kNetC;
    const float* b2 = w2t + kNetW2;
    const float* w3t = b2 + kNetC;
    const float* b3 = w3t + kNetW3;
    cudaError_t e;
    if ((e = conv<2, kNetC, 1>(x0, w1t, b1, nullptr, h1, n, H, W, s)) != cudaSuccess) return e;
    if ((e = conv<kNetC, kNetC, 1>(h1, w2t, b2, nullptr, h2, n, H, W, s)) != cudaSuccess) return e;
    if ((e = conv<kNetC, 2, 0>(h2, w3t, b3, nullptr, y, n, H, W, s)) != cudaSuccess) return e;
    const size_t m = 2 * Pn;
    net_loss_kernel<<<1216, 256, 0, s>>>(y, d, m, (float)(1.0 / (double)m), lpart);
    net_loss_finish_kernel<<<1, 32, 0, s>>>(lpart, 1216, 1.0 / (double)m, loss_dev);
    float* g1 = grad;
    float* g2 = g1 + kNetW1 + kNetC;
    float* g3 = g2 + kNetW2 + kNetC;
    if ((e = wgrad<kNetC, 2>(h2, y, n, H, W, nblk, part, g3, s)) != cudaSuccess) return e;
    if ((e = conv<2, kNetC, 2>(y, w.bwd3, nullptr, h2, gh2, n, H, W, s)) != cudaSuccess) return e;
    if ((e = wgrad<kNetC, kNetC>(h1, gh2, n, H, W, nblk, part, g2, s)) != cudaSuccess) return e;
    if ((e = conv<kNetC, kNetC, 2>(gh2, w.bwd2, nullptr, h1, gh1, n, H, W, s)) != cudaSuccess) return e;
    if ((e = wgrad<2, kNetC>(x0, gh1, n, H, W, nblk, part, g1, s)) != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_adam(float* P, float* m, float* v, const float* g, float lr, int step, cudaStream_t s) {
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, step)), c2 = (float)(1.0 - std::pow(b2, step));
    adam_kernel<<<(kNetParams + 255) / 256, 256, 0, s>>>(P, m, v, g, kNetParams, lr, 0.9f, 0.999f, c1, c2, 1e-8f);
    return cudaGetLastError();
}

cudaError_t launch_net_prep_weights(const float* P, const NetTrainPtrs& w, cudaStream_t s) {
    net_prep_weights_kernel<<<(kNetParams + 255) / 256, 256, 0, s>>>(P, w);
    return cudaGetLastError();
}

NetDev net_dev_view(const float* fwd) {
    NetDev nd;
    nd.w1t = fwd;
    nd.b1 = nd.w1t + kNetW1;
    nd.w2t = nd.b1 + kNetC;
    nd.b2 = nd.w2t + kNetW2;
    nd.w3t = nd.b2 + kNetC;
    nd.b3 = nd.w3t + kNetW3;
    return nd;
}

}  // namespace cpt
