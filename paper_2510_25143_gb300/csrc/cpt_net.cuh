// Learned predictor (an extension; the paper has none): a 3-layer 3x3
// convolutional net, 2 -> 32 -> 32 -> 2 channels, ReLU after the first two
// layers, zero padding at the field boundary.  Input: the reconstructed slice
// t-1 scaled by 2^-23; output y; prediction qhat(t-1) + rint(clamp(y, -2, 2)
// * 2^23).  Every output is a chain of float32 fused multiply-adds from the
// bias over (input channel, ky, kx) in that order, padding included as zero
// inputs, so the encoder, the decoder and any IEEE reimplementation agree.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cpt {

constexpr int kNetC = 32;
constexpr int kNetW1 = kNetC * 2 * 9, kNetW2 = kNetC * kNetC * 9, kNetW3 = 2 * kNetC * 9;
constexpr int kNetParams = kNetW1 + kNetC + kNetW2 + kNetC + kNetW3 + 2;  // 10434
constexpr int kNetReach = 3;  // rows/columns of slice t-1 beyond a vertex that its prediction reads

// Device copy of the parameters as float, each layer's weights transposed so
// that the output channels of one (input channel, ky, kx) are contiguous (and
// every weight block starts on a 16-byte boundary):
// wt[((ci * 3 + ky) * 3 + kx) * COUT + co] = w[co][ci][ky][kx].
struct NetDev {
    const float* w1t;  // [2][3][3][32]
    const float* b1;   // [32]
    const float* w2t;  // [32][3][3][32]
    const float* b2;
    const float* w3t;  // [32][3][3][2]
    const float* b3;   // [2]
};
constexpr int kNetDevFloats = kNetParams;  // same count, transposed weights then biases per layer

// One layer over an OH x OW output region whose (0, 0) sits at global
// (gy0, gx0); in is the CIN x (OH+2) x (OW+2) window around it.  The weights
// and biases may sit in global or shared memory (plain loads).  Outputs at
// positions outside the H x W field are 0 (the next layer's padding).  Each
// lane computes two positions (p and p + 32) for a group of up to 16 output
// channels at a time, so that every weight it loads (four channels at a
// time, contiguous in the transposed layout) feeds two fused multiply-adds
// per channel; each output's chain keeps the order bias, then (input
// channel, ky, kx).
template <int CIN, int COUT, bool RELU>
__device__ __forceinline__ void net_layer(const float* __restrict__ in, const float* __restrict__ wt,
                                          const float* __restrict__ b, float* __restrict__ out, int OH, int OW,
                                          int gy0, int gx0, int H, int W) {
    constexpr int G = COUT < 16 ? COUT : 16;  // output channels per pass
    static_assert(COUT % G == 0 && G % 2 == 0, "output channels in groups of pairs or quads");
    const int lane = (int)(threadIdx.x & 31u);
    const int IH = OH + 2, IW = OW + 2, NP = OH * OW;
    for (int p0 = lane; p0 < NP; p0 += 64) {
        const int p1 = p0 + 32;
        const bool has1 = p1 < NP;
        const int q1 = has1 ? p1 : p0;  // the second slot reads a valid position either way
        const int oy0 = p0 / OW, ox0 = p0 - oy0 * OW;
        const int oy1 = q1 / OW, ox1 = q1 - oy1 * OW;
        const int g0y = gy0 + oy0, g0x = gx0 + ox0, g1y = gy0 + oy1, g1x = gx0 + ox1;
        const bool in0 = g0y >= 0 && g0y < H && g0x >= 0 && g0x < W;
        const bool in1 = g1y >= 0 && g1y < H && g1x >= 0 && g1x < W;
#pragma unroll 1
        for (int cg = 0; cg < COUT; cg += G) {
            float acc0[G], acc1[G];
#pragma unroll
            for (int c = 0; c < G; ++c) acc0[c] = acc1[c] = b[cg + c];
            for (int ci = 0; ci < CIN; ++ci)
#pragma unroll
                for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx) {
                        const float v0 = in[(ci * IH + oy0 + ky) * IW + ox0 + kx];
                        const float v1 = in[(ci * IH + oy1 + ky) * IW + ox1 + kx];
                        const float* wp = wt + ((ci * 3 + ky) * 3 + kx) * COUT + cg;
                        if constexpr (G % 4 == 0) {
#pragma unroll
                            for (int c = 0; c < G; c += 4) {
                                const float4 w = *reinterpret_cast<const float4*>(wp + c);
                                acc0[c] = __fmaf_rn(w.x, v0, acc0[c]);
                                acc0[c + 1] = __fmaf_rn(w.y, v0, acc0[c + 1]);
                                acc0[c + 2] = __fmaf_rn(w.z, v0, acc0[c + 2]);
                                acc0[c + 3] = __fmaf_rn(w.w, v0, acc0[c + 3]);
                                acc1[c] = __fmaf_rn(w.x, v1, acc1[c]);
                                acc1[c + 1] = __fmaf_rn(w.y, v1, acc1[c + 1]);
                                acc1[c + 2] = __fmaf_rn(w.z, v1, acc1[c + 2]);
                                acc1[c + 3] = __fmaf_rn(w.w, v1, acc1[c + 3]);
                            }
                        } else {
#pragma unroll
                            for (int c = 0; c < G; c += 2) {
                                const float2 w = *reinterpret_cast<const float2*>(wp + c);
                                acc0[c] = __fmaf_rn(w.x, v0, acc0[c]);
                                acc0[c + 1] = __fmaf_rn(w.y, v0, acc0[c + 1]);
                                acc1[c] = __fmaf_rn(w.x, v1, acc1[c]);
                                acc1[c + 1] = __fmaf_rn(w.y, v1, acc1[c + 1]);
                            }
                        }
                    }
#pragma unroll
            for (int c = 0; c < G; ++c) {
                out[((cg + c) * OH + oy0) * OW + ox0] = in0 ? (RELU ? (acc0[c] > 0.0f ? acc0[c] : 0.0f) : acc0[c]) : 0.0f;
                if (has1)
                    out[((cg + c) * OH + oy1) * OW + ox1] =
                        in1 ? (RELU ? (acc1[c] > 0.0f ? acc1[c] : 0.0f) : acc1[c]) : 0.0f;
            }
        }
    }
}

// Scratch of one tile of UxU predictions.
template <int U>
struct NetScratch {
    float x[2][U + 6][U + 6];
    float h1[kNetC][U + 4][U + 4];
    float h2[kNetC][U + 2][U + 2];
    float y[2][U][U];
};

// The predictions of the U x U tile at (r0, c0): prev(i, j) returns the
// reconstructed slice t-1 value (zero outside the field); out(li, lj, pred)
// receives each prediction inside the field.  One warp.
template <int U, class Prev, class Out>
__device__ __forceinline__ void net_tile(const NetDev& nd, NetScratch<U>& s, int r0, int c0, int H, int W, const Prev& prev,
                         const Out& out) {
    const int lane = (int)(threadIdx.x & 31u);
    constexpr int XS = U + 6;
    for (int p = lane; p < XS * XS; p += 32) {
        const int yy = p / XS, xx = p - (p / XS) * XS;
        const int2 v = prev(r0 - 3 + yy, c0 - 3 + xx);  // |v| < 2^24: the 2^-23 scaling is exact
        s.x[0][yy][xx] = __fmul_rn(__int2float_rn(v.x), 1.1920928955078125e-07f);
        s.x[1][yy][xx] = __fmul_rn(__int2float_rn(v.y), 1.1920928955078125e-07f);
    }
    __syncwarp();
    net_layer<2, kNetC, true>(&s.x[0][0][0], nd.w1t, nd.b1, &s.h1[0][0][0], U + 4, U + 4, r0 - 2, c0 - 2, H, W);
    __syncwarp();
    net_layer<kNetC, kNetC, true>(&s.h1[0][0][0], nd.w2t, nd.b2, &s.h2[0][0][0], U + 2, U + 2, r0 - 1, c0 - 1, H, W);
    __syncwarp();
    net_layer<kNetC, 2, false>(&s.h2[0][0][0], nd.w3t, nd.b3, &s.y[0][0][0], U, U, r0, c0, H, W);
    __syncwarp();
    for (int p = lane; p < U * U; p += 32) {
        const int li = p / U, lj = p % U;
        if (r0 + li >= H || c0 + lj >= W) continue;
        const int2 q = prev(r0 + li, c0 + lj);
        int2 pr;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float d = s.y[c][li][lj];
            if (!(d == d)) d = 0.0f;
            d = d < -2.0f ? -2.0f : (d > 2.0f ? 2.0f : d);
            const int dq = __float2int_rn(__fmul_rn(d, 8388608.0f));
            if (c == 0) pr.x = q.x + dq;
            else pr.y = q.y + dq;
        }
        out(li, lj, pr);
    }
    __syncwarp();
}

}  // namespace cpt
