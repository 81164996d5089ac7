// Field-wide kernels: value range (for the fixed-point scale, Alg. 3
// Convert_FixedPoint), conversion to fixed point, the crossed-face masks of
// the space-time mesh (Alg. 3 face loop with Alg. 1) and the verification of
// a reconstruction (Eq. 4 on every face plus the pointwise bound).
#include "cpt_dev.cuh"
#include "cpt_internal.h"

namespace cpt {

// ---------------------------------------------------------------------------
// Range: per-block partial (min, max, max|x|, non-finite flag).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) range_kernel(const float4* __restrict__ uv, size_t n4,
                                                    const float* __restrict__ tail, int ntail,
                                                    RangePartial* __restrict__ part) {
    float mn = INFINITY, mx = -INFINITY, am = 0.f;
    unsigned bad = 0;
    auto acc = [&](float x) {
        bad |= !isfinite(x);
        mn = fminf(mn, x);
        mx = fmaxf(mx, x);
        am = fmaxf(am, fabsf(x));
    };
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n4; k += (size_t)gridDim.x * blockDim.x) {
        float4 a = __ldcs(uv + k);
        acc(a.x); acc(a.y); acc(a.z); acc(a.w);
    }
    if (blockIdx.x == 0 && (int)threadIdx.x < ntail) acc(tail[threadIdx.x]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ float smn[8], smx[8], sam[8];
    __shared__ unsigned sbad[8];
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { smn[w] = mn; smx[w] = mx; sam[w] = am; sbad[w] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            mn = fminf(mn, smn[k]); mx = fmaxf(mx, smx[k]); am = fmaxf(am, sam[k]); bad |= sbad[k];
        }
        part[blockIdx.x] = RangePartial{mn, mx, am, bad};
    }
}

// q = rint(x * 2^k) (round half to even); x * 2^k is exact in FP64.
__global__ void __launch_bounds__(256) to_fixed_kernel(const float4* __restrict__ uv, size_t n4,
                                                       const float* __restrict__ tail, int ntail, double scale,
                                                       int4* __restrict__ q, int* __restrict__ qtail) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n4; k += (size_t)gridDim.x * blockDim.x) {
        float4 a = __ldcs(uv + k);
        int4 r;
        r.x = __double2int_rn((double)a.x * scale);
        r.y = __double2int_rn((double)a.y * scale);
        r.z = __double2int_rn((double)a.z * scale);
        r.w = __double2int_rn((double)a.w * scale);
        q[k] = r;
    }
    if (blockIdx.x == 0 && (int)threadIdx.x < ntail) qtail[threadIdx.x] = __double2int_rn((double)tail[threadIdx.x] * scale);
}

// ---------------------------------------------------------------------------
// Face masks.  One thread per owner vertex (t,i,j); its 8 corner values
// (A,R,D,G at t and t+1) give the 12 owned faces.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_corners(const int2* __restrict__ q, int H, int W, int T, int t, int i, int j,
                                             int2 c[8]) {
    bool r = j + 1 < W, d = i + 1 < H, n = t + 1 < T;
    size_t v = ((size_t)t * H + i) * W + j, sl = (size_t)H * W;
    c[0] = q[v];
    c[1] = r ? q[v + 1] : make_int2(0, 0);
    c[2] = d ? q[v + W] : make_int2(0, 0);
    c[3] = (r && d) ? q[v + W + 1] : make_int2(0, 0);
    if (n) {
        c[4] = q[v + sl];
        c[5] = r ? q[v + sl + 1] : make_int2(0, 0);
        c[6] = d ? q[v + sl + W] : make_int2(0, 0);
        c[7] = (r && d) ? q[v + sl + W + 1] : make_int2(0, 0);
    } else {
        c[4] = c[5] = c[6] = c[7] = make_int2(0, 0);
    }
}

__global__ void __launch_bounds__(256) face_mask_kernel(const int2* __restrict__ q, int H, int W, int T,
                                                        uint16_t* __restrict__ mask,
                                                        unsigned long long* __restrict__ ncrossed) {
    int j = blockIdx.x * 32 + (threadIdx.x & 31);
    int i = blockIdx.y * 8 + (threadIdx.x >> 5);
    int t = blockIdx.z;
    unsigned cnt = 0;
    if (i < H && j < W) {
        int2 c[8];
        load_corners(q, H, W, T, t, i, j, c);
        uint16_t m = owned_face_mask(c, owned_valid(H, W, T, t, i, j));
        mask[((size_t)t * H + i) * W + j] = m;
        cnt = __popc(m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(ncrossed, (unsigned long long)cnt);
}

// Verification: recompute the owned-face masks on the encoder's reconstruction
// words and compare with the original (slice faces = types 0,1; slab faces =
// 2..11); also the largest |x_hat - x| with x_hat = qhat * 2^-k in float32.
__global__ void __launch_bounds__(256) verify_kernel(const int2* __restrict__ qhat, const uint16_t* __restrict__ mask,
                                                     const float2* __restrict__ uv, int H, int W, int T,
                                                     double inv_scale, VerifyOut* __restrict__ out) {
    int j = blockIdx.x * 32 + (threadIdx.x & 31);
    int i = blockIdx.y * 8 + (threadIdx.x >> 5);
    int t = blockIdx.z;
    unsigned ms = 0, mb = 0;
    double err = 0.0, sq = 0.0;
    if (i < H && j < W) {
        int2 c[8];
        load_corners(qhat, H, W, T, t, i, j, c);
        {   // the reconstruction words carry the tag in y (absent corners read as zero)
            const bool r = j + 1 < W, d = i + 1 < H, n = t + 1 < T;
            const bool has[8] = {true, r, d, r && d, n, n && r, n && d, n && r && d};
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (has[k]) c[k].y ^= kQhatTag;
        }
        size_t v = ((size_t)t * H + i) * W + j;
        uint16_t m = owned_face_mask(c, owned_valid(H, W, T, t, i, j));
        unsigned x = (unsigned)(m ^ mask[v]);
        ms = __popc(x & 3u);
        mb = __popc(x & ~3u);
        float2 o = uv[v];
        float a = (float)((double)c[0].x * inv_scale), b = (float)((double)c[0].y * inv_scale);
        double e0 = fabs((double)a - (double)o.x), e1 = fabs((double)b - (double)o.y);
        err = fmax(e0, e1);
        sq = e0 * e0 + e1 * e1;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ms += __shfl_xor_sync(0xffffffffu, ms, o);
        mb += __shfl_xor_sync(0xffffffffu, mb, o);
        err = fmax(err, __shfl_xor_sync(0xffffffffu, err, o));
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ms) atomicAdd(&out->mismatch_slice, (unsigned long long)ms);
        if (mb) atomicAdd(&out->mismatch_slab, (unsigned long long)mb);
        // err >= 0: the IEEE bit pattern orders like an unsigned integer
        atomicMax(&out->linf_bits, (unsigned long long)__double_as_longlong(err));
        atomicAdd(&out->sq_err, sq);
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_range(const float* uv, size_t n, RangePartial* part, int nblocks, cudaStream_t s) {
    size_t n4 = n / 4;
    range_kernel<<<nblocks, 256, 0, s>>>(reinterpret_cast<const float4*>(uv), n4, uv + 4 * n4, (int)(n - 4 * n4),
                                         part);
}

void launch_to_fixed(const float* uv, size_t n, double scale, int32_t* q, int nblocks, cudaStream_t s) {
    size_t n4 = n / 4;
    to_fixed_kernel<<<nblocks, 256, 0, s>>>(reinterpret_cast<const float4*>(uv), n4, uv + 4 * n4,
                                            (int)(n - 4 * n4), scale, reinterpret_cast<int4*>(q), q + 4 * n4);
}

void launch_face_masks(const int32_t* q, int H, int W, int T, uint16_t* mask, unsigned long long* ncrossed,
                       cudaStream_t s) {
    dim3 grid((W + 31) / 32, (H + 7) / 8, T);
    face_mask_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const int2*>(q), H, W, T, mask, ncrossed);
}

void launch_verify(const int32_t* qhat, const uint16_t* mask, const float* uv, int H, int W, int T, double inv_scale,
                   VerifyOut* out, cudaStream_t s) {
    dim3 grid((W + 31) / 32, (H + 7) / 8, T);
    verify_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const int2*>(qhat), mask,
                                       reinterpret_cast<const float2*>(uv), H, W, T, inv_scale, out);
}

}  // namespace cpt
