// Field-wide kernels: value range (for the fixed-point scale, Alg. 3
// Convert_FixedPoint), conversion to fixed point, the crossed-face masks of
// the space-time mesh (Alg. 3 face loop with Alg. 1) and the verification of
// a reconstruction (Eq. 4 on every face plus the pointwise bound).
#include <cmath>

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

// q = rint(x * 2^k) (round half to even).  |x * 2^k| < 2^24, so the product
// is exact in FP32 as well; it is formed as (x * 2^a) * 2^b, a + b = k, with
// both factors representable (an intermediate is never larger than the
// result when k > 0, and results below 2^-126 round to 0 either way).
__global__ void __launch_bounds__(256) to_fixed_kernel(const float4* __restrict__ uv, size_t n4,
                                                       const float* __restrict__ tail, int ntail, float f1, float f2,
                                                       int4* __restrict__ q, int* __restrict__ qtail) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n4; k += (size_t)gridDim.x * blockDim.x) {
        float4 a = __ldcs(uv + k);
        int4 r;
        r.x = __float2int_rn(__fmul_rn(__fmul_rn(a.x, f1), f2));
        r.y = __float2int_rn(__fmul_rn(__fmul_rn(a.y, f1), f2));
        r.z = __float2int_rn(__fmul_rn(__fmul_rn(a.z, f1), f2));
        r.w = __float2int_rn(__fmul_rn(__fmul_rn(a.w, f1), f2));
        __stcs(q + k, r);
    }
    if (blockIdx.x == 0 && (int)threadIdx.x < ntail)
        qtail[threadIdx.x] = __float2int_rn(__fmul_rn(__fmul_rn(tail[threadIdx.x], f1), f2));
}

// ---------------------------------------------------------------------------
// Face masks and verification.  A warp walks kFaceRows rows of one slice over
// 32 columns: lane l reads column j0 + l and owns it for l < 31 (lane 31
// supplies the right-hand corners).  Per row each lane loads its vertex at
// (t, i+1) and (t+1, i+1); (t, i) and (t+1, i) are the previous row's.  The
// right-hand corners come from lane l+1 by shuffle.  A face whose three
// vertices share one strict sign of u or of v cannot contain the origin, also
// after perturbation; only the remaining candidates (rare) take the exact SoS
// test, with the corner values fetched by shuffle.
// ---------------------------------------------------------------------------
constexpr int kFaceRows = 16;

struct FaceRowOut {
    uint16_t m;     // owned-face mask of the lane's vertex
    bool owner;     // the lane owns a vertex in this row
};

// Loader: (t, i, j) inside the field -> value; q reads the array, Tagged the
// encoder's reconstruction words.
struct PlainLoad {
    const int2* q;
    __device__ __forceinline__ int2 operator()(size_t v) const { return __ldg(q + v); }
};
struct TaggedLoad {
    const int2* q;
    __device__ __forceinline__ int2 operator()(size_t v) const {
        int2 x = __ldg(q + v);
        x.y ^= kQhatTag;
        return x;
    }
};

template <class Load, class Pre, class Visit>
__device__ __forceinline__ void face_rows(const Load& ld, int H, int W, int T, int t, int ib, int j0, Pre pre,
                                          Visit visit) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, j = j0 + lane;
    const bool colok = j < W, nx = t + 1 < T;
    const size_t sl = (size_t)H * W, base = (size_t)t * sl;
    const int2 z = make_int2(0, 0);
    // rows i (A), i + 1 (D) and i + 2 (Dn, loaded one row ahead)
    auto load_row = [&](int r, int2& v, int2& vp) {
        v = z;
        vp = z;
        if (colok && r < H) {
            v = ld(base + (size_t)r * W + j);
            if (nx) vp = ld(base + sl + (size_t)r * W + j);
        }
    };
    int2 A, Ap, D, Dp;
    load_row(ib, A, Ap);
    load_row(ib + 1, D, Dp);
    unsigned cA = sign_class(A.x, A.y), cAp = sign_class(Ap.x, Ap.y);
    const int ie = min(H, ib + kFaceRows);
    for (int i = ib; i < ie; ++i) {
        int2 Dn, Dnp;
        load_row(i + 2 < ib + kFaceRows + 1 ? i + 2 : H, Dn, Dnp);
        const auto P = pre(i, j);
        const unsigned cD = sign_class(D.x, D.y), cDp = sign_class(Dp.x, Dp.y);
        const unsigned cR = __shfl_down_sync(FULL, cA, 1), cG = __shfl_down_sync(FULL, cD, 1);
        const unsigned cRp = __shfl_down_sync(FULL, cAp, 1), cGp = __shfl_down_sync(FULL, cDp, 1);
        const bool owner = lane < 31 && colok;
        // a strict sign shared by all existing corners rules out every owned
        // face at once (absent corners count as sharing every sign)
        const bool r = j + 1 < W, d = i + 1 < H;
        const unsigned all = cA & (r ? cR : 15u) & (d ? cD : 15u) & (r && d ? cG : 15u) &
                             (nx ? cAp & (r ? cRp : 15u) & (d ? cDp : 15u) & (r && d ? cGp : 15u) : 15u);
        unsigned m = 0;
        if (__any_sync(FULL, owner && all == 0u)) {
            // candidates: no strict sign shared by the three corners (corner 0 is A)
            const unsigned cc[8] = {cA, cR, cD, cG, cAp, cRp, cDp, cGp};
            unsigned cand = 0;
#define CPT_C(ty, a, b, c) cand |= ((cc[a] & cc[b] & cc[c]) == 0u ? 1u : 0u) << (ty);
            CPT_OWNED_FACES(CPT_C)
#undef CPT_C
            cand = (owner && all == 0u) ? cand & owned_valid(H, W, T, t, i, j) : 0u;
            int2 c[8];
            c[0] = A; c[2] = D; c[4] = Ap; c[6] = Dp;
            c[1].x = __shfl_down_sync(FULL, A.x, 1); c[1].y = __shfl_down_sync(FULL, A.y, 1);
            c[3].x = __shfl_down_sync(FULL, D.x, 1); c[3].y = __shfl_down_sync(FULL, D.y, 1);
            c[5].x = __shfl_down_sync(FULL, Ap.x, 1); c[5].y = __shfl_down_sync(FULL, Ap.y, 1);
            c[7].x = __shfl_down_sync(FULL, Dp.x, 1); c[7].y = __shfl_down_sync(FULL, Dp.y, 1);
            if (cand) {
#define CPT_X(ty, a, b, cidx) \
    if (((cand >> (ty)) & 1u) && face_crossed(c[a], c[b], c[cidx])) m |= 1u << (ty);
                CPT_OWNED_FACES(CPT_X)
#undef CPT_X
            }
        }
        visit(i, j, FaceRowOut{(uint16_t)m, owner}, A, P);
        A = D;
        Ap = Dp;
        D = Dn;
        Dp = Dnp;
        cA = cD;
        cAp = cDp;
    }
}

// Work item -> (t, first row, first column); items run in slice order so that
// slice t+1, read again as slice t, is still in L2.
__device__ __forceinline__ bool face_item(int H, int W, int T, long long item, int& t, int& ib, int& j0) {
    const int nj = (W + 30) / 31, ni = (H + kFaceRows - 1) / kFaceRows;
    const long long per_t = (long long)ni * nj;
    if (item >= per_t * T) return false;
    t = (int)(item / per_t);
    const long long r = item % per_t;
    ib = (int)(r / nj) * kFaceRows;
    j0 = (int)(r % nj) * 31;
    return true;
}

__global__ void __launch_bounds__(256) face_mask_kernel(const int2* __restrict__ q, int H, int W, int T,
                                                        uint16_t* __restrict__ mask,
                                                        unsigned long long* __restrict__ ncrossed) {
    const long long item = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    unsigned cnt = 0;
    int t, ib, j0;
    if (face_item(H, W, T, item, t, ib, j0)) {
        const size_t base = (size_t)t * H * W;
        face_rows(PlainLoad{q}, H, W, T, t, ib, j0, [](int, int) { return 0; }, [&](int i, int j, FaceRowOut o, int2, int) {
            if (o.owner) {
                mask[base + (size_t)i * W + j] = o.m;
                cnt += __popc(o.m);
            }
        });
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    __shared__ unsigned sc[8];
    if ((threadIdx.x & 31) == 0) sc[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int w = 0; w < 8; ++w) tot += sc[w];
        if (tot) atomicAdd(ncrossed, tot);
    }
}

// Exact |x_hat - x| for floats: s + e = x_hat - x exactly (TwoSum; no
// contraction in this build).  Pairs compare by (|s|, e with the sign of s)
// like the exact differences; the largest is rounded to double once, which
// equals the largest of the differences rounded to double one by one.
struct ErrMax {
    float s, e;  // |s|, e * sign(s)
};
__device__ __forceinline__ ErrMax err_pair(float xh, float x) {
    const float s = __fsub_rn(xh, x);
    const float bb = __fsub_rn(s, xh);
    const float e = __fadd_rn(__fsub_rn(xh, __fsub_rn(s, bb)), __fsub_rn(-x, bb));
    return ErrMax{fabsf(s), s < 0.f ? -e : e};
}
__device__ __forceinline__ ErrMax err_max(ErrMax a, ErrMax b) {
    return (b.s > a.s || (b.s == a.s && b.e > a.e)) ? b : a;
}

__global__ void __launch_bounds__(256) verify_kernel(const int2* __restrict__ qhat, const uint16_t* __restrict__ mask,
                                                     const float2* __restrict__ uv, int H, int W, int T,
                                                     float g1, float g2, VerifyOut* __restrict__ out) {
    const long long item = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    unsigned ms = 0, mb = 0;
    ErrMax em{0.f, 0.f};
    float sq = 0.f;
    int t, ib, j0;
    if (face_item(H, W, T, item, t, ib, j0)) {
        const size_t base = (size_t)t * H * W;
        // the original mask and values of the row, loaded before its faces are evaluated
        struct Orig {
            unsigned m;
            float2 x;
        };
        auto pre = [&](int i, int j) {
            Orig r{0u, make_float2(0.f, 0.f)};
            if (j < W && (threadIdx.x & 31) < 31) {
                const size_t v = base + (size_t)i * W + j;
                r.m = mask[v];
                r.x = __ldcs(uv + v);
            }
            return r;
        };
        face_rows(TaggedLoad{qhat}, H, W, T, t, ib, j0, pre, [&](int i, int j, FaceRowOut o, int2 A, Orig P) {
            if (!o.owner) return;
            const unsigned x = (unsigned)o.m ^ P.m;
            ms += __popc(x & 3u);
            mb += __popc(x & ~3u);
            const float2 ov = P.x;
            // x_hat = qhat * 2^-k, exact in FP32 (|qhat| < 2^24)
            const float a = __fmul_rn(__fmul_rn(__int2float_rn(A.x), g1), g2);
            const float b = __fmul_rn(__fmul_rn(__int2float_rn(A.y), g1), g2);
            const ErrMax e0 = err_pair(a, ov.x), e1 = err_pair(b, ov.y);
            em = err_max(em, err_max(e0, e1));
            sq = __fadd_rn(sq, __fadd_rn(__fmul_rn(e0.s, e0.s), __fmul_rn(e1.s, e1.s)));
        });
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ms += __shfl_xor_sync(0xffffffffu, ms, o);
        mb += __shfl_xor_sync(0xffffffffu, mb, o);
        sq = __fadd_rn(sq, __shfl_xor_sync(0xffffffffu, sq, o));
        ErrMax p{__shfl_xor_sync(0xffffffffu, em.s, o), __shfl_xor_sync(0xffffffffu, em.e, o)};
        em = err_max(em, p);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ms) atomicAdd(&out->mismatch_slice, (unsigned long long)ms);
        if (mb) atomicAdd(&out->mismatch_slab, (unsigned long long)mb);
        // the exact largest difference rounded once; >= 0, so its bit pattern
        // orders like an unsigned integer
        const double err = (double)em.s + (double)em.e;
        if (err > 0.0) atomicMax(&out->linf_bits, (unsigned long long)__double_as_longlong(err));
        if (sq > 0.f) atomicAdd(&out->sq_err, (double)sq);
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

void launch_to_fixed(const float* uv, size_t n, int k, int32_t* q, int nblocks, cudaStream_t s) {
    size_t n4 = n / 4;
    const int a = k / 2, b = k - a;
    to_fixed_kernel<<<nblocks, 256, 0, s>>>(reinterpret_cast<const float4*>(uv), n4, uv + 4 * n4,
                                            (int)(n - 4 * n4), std::ldexp(1.0f, a), std::ldexp(1.0f, b),
                                            reinterpret_cast<int4*>(q), q + 4 * n4);
}

static unsigned face_blocks(int H, int W, int T) {
    const long long items = (long long)T * ((H + kFaceRows - 1) / kFaceRows) * ((W + 30) / 31);
    return (unsigned)((items + 7) / 8);
}

void launch_face_masks(const int32_t* q, int H, int W, int T, uint16_t* mask, unsigned long long* ncrossed,
                       cudaStream_t s) {
    face_mask_kernel<<<face_blocks(H, W, T), 256, 0, s>>>(reinterpret_cast<const int2*>(q), H, W, T, mask, ncrossed);
}

void launch_verify(const int32_t* qhat, const uint16_t* mask, const float* uv, int H, int W, int T, int k,
                   VerifyOut* out, cudaStream_t s) {
    const int a = -k / 2, b = -k - a;
    verify_kernel<<<face_blocks(H, W, T), 256, 0, s>>>(reinterpret_cast<const int2*>(qhat), mask,
                                                       reinterpret_cast<const float2*>(uv), H, W, T,
                                                       std::ldexp(1.0f, a), std::ldexp(1.0f, b), out);
}

}  // namespace cpt
