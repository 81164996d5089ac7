// Field-wide kernels: value range (for the fixed-point scale, Alg. 3
// Convert_FixedPoint), conversion to fixed point, the crossed-face masks of
// the space-time mesh (Alg. 3 face loop with Alg. 1) and the verification of
// a reconstruction (Eq. 4 on every face plus the pointwise bound).
#include <algorithm>
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
// Face masks and verification (Eq. 2 under SoS on every face, Alg. 3's face
// loop; Eq. 4 for the verification).  A warp walks kFaceRows rows of one
// slice over 64 columns, two adjacent columns per lane (one 16-byte load per
// lane and slice when W is even); lanes 0..30 own their columns, lane 31's
// two columns are the next strip's first and only supply right-hand corners,
// so strips advance by 62 columns.  Per row it loads row i + 1 of slices t
// and t + 1 (prefetched one row ahead); rows i and i + 1 give the 2 x 2 x 2
// corner cube of each owned vertex.
//
// Filter: a face whose three vertices share one strict sign of u or of v
// cannot contain the origin, also after perturbation.  Each vertex value
// becomes a sign word whose byte sign bits are u < 0, v < 0, u > 0, v > 0;
// the AND of the eight corner words keeps the strict signs the whole cube
// shares, which rules out every owned face at once.  The cube's AND is built
// from column pairs (t and t + 1), row pairs and the right neighbour (one
// shuffle per lane).  Only vertices whose cube shares no sign take the exact
// test: the candidate faces (the AND of their three corner words has no sign
// bit) go through the SoS predicate.  Absent corners (outside the field) use
// a word with every sign bit set; faces through them are not valid.
// ---------------------------------------------------------------------------
constexpr int kFaceRows = 32;
constexpr int kStrip = 62;  // owned columns of a warp (lanes 0..30)
constexpr unsigned kSignBits = 0x80808080u;
constexpr unsigned kNoCorner = 0xffffffffu;

__device__ __forceinline__ unsigned sign_word(int u, int v) {
    unsigned a, b;
    // bytes (u.b3, v.b3, u.b3, v.b3) and the same of (-u, -v); |u|, |v| < 2^31
    asm("prmt.b32 %0, %1, %2, 0x7373;" : "=r"(a) : "r"(u), "r"(v));
    asm("prmt.b32 %0, %1, %2, 0x7373;" : "=r"(b) : "r"(-u), "r"(-v));
    return (a & 0x0000ffffu) | (b & 0xffff0000u);
}

// Owned-face mask of one vertex from its eight corners (index bit0 = +j,
// bit1 = +i, bit2 = +t), their sign words and the valid face types.
__device__ __forceinline__ unsigned exact_mask(const int2* c, const unsigned* w, unsigned valid) {
    unsigned cand = 0;
#define CPT_C(ty, a, b, cc) cand |= (((w[a] & w[b] & w[cc]) & kSignBits) == 0u ? 1u : 0u) << (ty);
    CPT_OWNED_FACES(CPT_C)
#undef CPT_C
    cand &= valid;
    unsigned m = 0;
    if (cand) {
#define CPT_X(ty, a, b, cc) \
    if (((cand >> (ty)) & 1u) && face_crossed(c[a], c[b], c[cc])) m |= 1u << (ty);
        CPT_OWNED_FACES(CPT_X)
#undef CPT_X
    }
    return m;
}

// One row of a lane's two columns c0, c0 + 1 at one slice.  kVec: W even,
// so (row * W + c0) is even and the pair is one aligned 16-byte load.
// kTag: the encoder's reconstruction words.
struct RowVals {
    int2 v0, v1;
};

template <bool kVec, bool kTag, bool kIn = false>
__device__ __forceinline__ RowVals load_row(const int2* __restrict__ q, size_t row_base, int c0, int W, bool ok) {
    RowVals r;
    r.v0 = r.v1 = make_int2(0, 0);
    if (ok) {
        if (kVec) {
            if (kIn || c0 < W) {
                const int4 x = __ldg(reinterpret_cast<const int4*>(q + row_base + c0));
                r.v0 = make_int2(x.x, x.y);
                r.v1 = make_int2(x.z, x.w);
            }
        } else {
            if (c0 < W) r.v0 = __ldg(q + row_base + c0);
            if (c0 + 1 < W) r.v1 = __ldg(q + row_base + c0 + 1);
        }
        if (kTag) {
            r.v0.y ^= kQhatTag;
            r.v1.y ^= kQhatTag;
        }
    }
    return r;
}

// The tag of reconstruction words removed (verification input), applied when
// a prefetched row is consumed rather than right after its load.
template <bool kTag>
__device__ __forceinline__ RowVals untag(RowVals r) {
    if (kTag) {
        r.v0.y ^= kQhatTag;
        r.v1.y ^= kQhatTag;
    }
    return r;
}

struct RowWords {
    unsigned w0, w1;
};
__device__ __forceinline__ RowWords row_words(const RowVals& r, bool ok, bool ok0, bool ok1) {
    RowWords w;
    w.w0 = ok && ok0 ? sign_word(r.v0.x, r.v0.y) : kNoCorner;
    w.w1 = ok && ok1 ? sign_word(r.v1.x, r.v1.y) : kNoCorner;
    return w;
}

struct ErrMax {
    float s, e;  // |s|, e * sign(s)
};

struct FaceAcc {
    unsigned long long crossed;
    unsigned ms, mb;
    ErrMax em;
    float sq;
};

// Exact |x_hat - x| for floats: s + e = x_hat - x exactly (TwoSum; no
// contraction in this build).  Pairs compare by (|s|, e with the sign of s)
// like the exact differences; the largest is rounded to double once, which
// equals the largest of the differences rounded to double one by one.
__device__ __forceinline__ ErrMax err_pair(float xh, float x) {
    const float s = __fsub_rn(xh, x);
    const float bb = __fsub_rn(s, xh);
    const float e = __fadd_rn(__fsub_rn(xh, __fsub_rn(s, bb)), __fsub_rn(-x, bb));
    return ErrMax{fabsf(s), s < 0.f ? -e : e};
}
__device__ __forceinline__ ErrMax err_max(ErrMax a, ErrMax b) {
    return (b.s > a.s || (b.s == a.s && b.e > a.e)) ? b : a;
}

// One reconstructed component against the original: the largest exact
// difference and the sum of squared differences (a statistic, fused).
// Rounding is monotonic, so a rounded difference below the largest one's
// comes from a smaller exact difference: the TwoSum runs only for the
// others.
__device__ __forceinline__ void err_acc(FaceAcc& acc, float xh, float x) {
    const float s = __fsub_rn(xh, x);
    if (fabsf(s) >= acc.em.s) acc.em = err_max(acc.em, err_pair(xh, x));
    acc.sq = __fmaf_rn(s, s, acc.sq);
}

// A corner value for the exact test (zero and an all-signs word outside the
// field; faces through such corners are not valid).
template <bool kTag>
__device__ __forceinline__ int2 corner(const int2* __restrict__ q, int H, int W, int T, int t, int i, int j,
                                       unsigned& w) {
    if (t >= T || i >= H || j >= W) {
        w = kNoCorner;
        return make_int2(0, 0);
    }
    int2 x = __ldg(q + ((size_t)t * H + i) * W + j);
    if (kTag) x.y ^= kQhatTag;
    w = sign_word(x.x, x.y);
    return x;
}

// Verification: the original masks (two per word) and values of a lane's
// owned vertices in one row.
template <bool kVec>
__device__ __forceinline__ void orig_row(const uint16_t* __restrict__ mask_in, const float2* __restrict__ uv,
                                         size_t vrow, int c0, bool own0, bool own1, unsigned& om, float4& ox) {
    om = 0;
    ox = make_float4(0.f, 0.f, 0.f, 0.f);
    if (kVec) {
        if (own0) {
            om = __ldg(reinterpret_cast<const unsigned*>(mask_in + vrow + c0));
            ox = __ldcs(reinterpret_cast<const float4*>(uv + vrow + c0));
        }
    } else {
        if (own0) {
            om = __ldg(mask_in + vrow + c0);
            const float2 a = __ldcs(uv + vrow + c0);
            ox.x = a.x;
            ox.y = a.y;
        }
        if (own1) {
            om |= (unsigned)__ldg(mask_in + vrow + c0 + 1) << 16;
            const float2 b = __ldcs(uv + vrow + c0 + 1);
            ox.z = b.x;
            ox.w = b.y;
        }
    }
}

// The warp's deferred vertices: the 2 x 2 x 2 cube shares no strict sign.
// Entries (row - ib) << 6 | (column - j0).  Interior items queue them in
// kQueueCap entries, worked off before a row (at most kStrip entries) could
// overflow it; the others in the warp's ring storage, which holds every
// owned vertex of an item.
constexpr int kQueueCap = 512;

// The exact test of the queued vertices, one per lane, their corners read
// again (from L2).  Returns (crossed faces, 0) for the masks and (slice,
// slab mismatches) for the verification.
template <bool kVerify>
__device__ __forceinline__ uint2 face_exact(const int2* __restrict__ q, int H, int W, int T, int t, int ib, int j0,
                                         uint16_t* __restrict__ mask_out, const uint16_t* __restrict__ mask_in,
                                         const uint16_t* __restrict__ queue, int nq) {
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)t * H * W;
    uint2 r = make_uint2(0u, 0u);
    __syncwarp();
    for (int k = lane; k < nq; k += 32) {
        const unsigned e = queue[k];
        const int i = ib + (int)(e >> 6), j = j0 + (int)(e & 63u);
        int2 c[8];
        unsigned w[8];
#pragma unroll
        for (int n = 0; n < 8; ++n) c[n] = corner<kVerify>(q, H, W, T, t + (n >> 2), i + ((n >> 1) & 1), j + (n & 1), w[n]);
        const unsigned m = exact_mask(c, w, owned_valid(H, W, T, t, i, j));
        const size_t v = base + (size_t)i * W + j;
        if (kVerify) {
            const unsigned x = m ^ (unsigned)mask_in[v];
            r.x += __popc(x & 3u);
            r.y += __popc(x & 0xffcu);
        } else {
            mask_out[v] = (uint16_t)m;
            r.x += __popc(m);
        }
    }
    __syncwarp();
    return r;
}

__device__ __forceinline__ void add_exact(FaceAcc& acc, uint2 r, bool verify) {
    if (verify) {
        acc.ms += r.x;
        acc.mb += r.y;
    } else {
        acc.crossed += r.x;
    }
}

// One work item: rows [ib, ib + kFaceRows) of slice t, columns [j0, j0 + 62).
// The rows are streamed with the sign filter only; vertices that pass it
// are queued for face_exact.  It returns the updated accumulators.  kInner:
// rows ib .. ib + kFaceRows, the lanes' columns and slice t + 1 all lie in
// the field, so every validity test folds away.
template <bool kVerify, bool kVec, bool kInner = false>
__device__ __forceinline__ FaceAcc face_item_rows(const int2* __restrict__ q, int H, int W, int T, int t, int ib,
                                               int j0, uint16_t* __restrict__ mask_out,
                                               const uint16_t* __restrict__ mask_in,
                                               const float2* __restrict__ uv, float g1, float g2, FaceAcc acc,
                                               uint16_t* __restrict__ queue) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int c0 = j0 + 2 * lane, c1 = c0 + 1;
    const bool in0 = kInner || c0 < W, in1 = kInner || c1 < W;  // columns inside the field
    const bool own0 = in0 && lane < 31, own1 = in1 && lane < 31;
    const bool nx = kInner || t + 1 < T;
    const size_t sl = (size_t)H * W, base = (size_t)t * sl;
    const int ie = kInner ? ib + kFaceRows : min(H, ib + kFaceRows);
    int nq = 0;
    // rows i (A: slice t, P: slice t + 1) and i + 1 (D, Dp); rows i + 2 (N,
    // Np) are loaded one row step ahead, without their tag removed yet
    const int re = kInner ? ib + kFaceRows + 1 : min(H, ib + kFaceRows + 1);  // rows the item reads: [ib, re)
    RowVals A = load_row<kVec, kVerify, kInner>(q, base + (size_t)ib * W, c0, W, true);
    RowVals P = load_row<kVec, kVerify, kInner>(q, base + sl + (size_t)ib * W, c0, W, nx);
    RowVals D = load_row<kVec, kVerify, kInner>(q, base + (size_t)(ib + 1) * W, c0, W, kInner || ib + 1 < H);
    RowVals Dp = load_row<kVec, kVerify, kInner>(q, base + sl + (size_t)(ib + 1) * W, c0, W, nx && (kInner || ib + 1 < H));
    RowVals N = load_row<kVec, false, kInner>(q, base + (size_t)(ib + 2) * W, c0, W, ib + 2 < re);
    RowVals Np = load_row<kVec, false, kInner>(q, base + sl + (size_t)(ib + 2) * W, c0, W, ib + 2 < re && nx);
    RowWords wa = row_words(A, true, in0, in1), wp = row_words(P, nx, in0, in1);
    unsigned col0 = wa.w0 & wp.w0, col1 = wa.w1 & wp.w1;
    unsigned omN = 0;
    float4 oxN = make_float4(0.f, 0.f, 0.f, 0.f);
    if (kVerify) orig_row<kVec>(mask_in, uv, base + (size_t)ib * W, c0, own0, own1, omN, oxN);
    for (int i = ib; i < ie; ++i) {
        const bool dn = kInner || i + 1 < H, n3 = i + 3 < re;
        // prefetch row i + 3
        const RowVals NN = load_row<kVec, false, kInner>(q, base + (size_t)(i + 3) * W, c0, W, n3);
        const RowVals NNp = load_row<kVec, false, kInner>(q, base + sl + (size_t)(i + 3) * W, c0, W, n3 && nx);
        const size_t vrow = base + (size_t)i * W;
        // verification: the original masks and values of row i (loaded one
        // row ahead), and those of row i + 1 for the next iteration
        const unsigned om = omN;
        const float4 ox = oxN;
        if (kVerify && dn && i + 1 < ie) orig_row<kVec>(mask_in, uv, vrow + W, c0, own0, own1, omN, oxN);
        const RowWords wd = row_words(D, dn, in0, in1), wdp = row_words(Dp, dn && nx, in0, in1);
        const unsigned dcol0 = wd.w0 & wdp.w0, dcol1 = wd.w1 & wdp.w1;
        const unsigned vp0 = col0 & dcol0, vp1 = col1 & dcol1;
        const unsigned right = __shfl_down_sync(FULL, vp0, 1);
        const bool need0 = own0 && ((vp0 & vp1 & kSignBits) == 0u);
        const bool need1 = own1 && ((vp1 & right & kSignBits) == 0u);
        const unsigned b0 = __ballot_sync(FULL, need0), b1 = __ballot_sync(FULL, need1);
        if (b0 | b1) {
            int pos = nq + __popc(b0 & lt) + __popc(b1 & lt);
            const uint16_t e = (uint16_t)(((i - ib) << 6) | (2 * lane));
            if (need0) queue[pos++] = e;
            if (need1) queue[pos] = (uint16_t)(e + 1);
            nq += __popc(b0) + __popc(b1);
        }
        if (kVerify) {
            // a queued vertex is counted after its exact test
            const unsigned x = om & ~((need0 ? 0x0000ffffu : 0u) | (need1 ? 0xffff0000u : 0u));
            acc.ms += __popc(x & 0x00030003u);
            acc.mb += __popc(x & 0x0ffc0ffcu);
            // x_hat = qhat * 2^-k, exact in FP32 (|qhat| < 2^24)
            if (own0) {
                const float a = __fmul_rn(__fmul_rn(__int2float_rn(A.v0.x), g1), g2);
                const float b = __fmul_rn(__fmul_rn(__int2float_rn(A.v0.y), g1), g2);
                err_acc(acc, a, ox.x);
                err_acc(acc, b, ox.y);
            }
            if (own1) {
                const float a = __fmul_rn(__fmul_rn(__int2float_rn(A.v1.x), g1), g2);
                const float b = __fmul_rn(__fmul_rn(__int2float_rn(A.v1.y), g1), g2);
                err_acc(acc, a, ox.z);
                err_acc(acc, b, ox.w);
            }
        } else {
            // every owned face of a vertex that passes no test is uncrossed
            if (kVec) {
                if (own0) *reinterpret_cast<unsigned*>(mask_out + vrow + c0) = 0u;
            } else {
                if (own0) mask_out[vrow + c0] = 0;
                if (own1) mask_out[vrow + c1] = 0;
            }
        }
        A = D;
        P = Dp;
        D = untag<kVerify>(N);
        Dp = untag<kVerify>(Np);
        N = NN;
        Np = NNp;
        wa = wd;
        wp = wdp;
        col0 = dcol0;
        col1 = dcol1;
    }
    if (nq) add_exact(acc, face_exact<kVerify>(q, H, W, T, t, ib, j0, mask_out, mask_in, queue, nq), kVerify);
    return acc;
}

// The same out of line, beside the interior path (its registers are then its
// own).
template <bool kVerify, bool kVec>
__device__ __noinline__ FaceAcc face_item_rows_call(const int2* __restrict__ q, int H, int W, int T, int t, int ib,
                                                    int j0, uint16_t* __restrict__ mask_out,
                                                    const uint16_t* __restrict__ mask_in,
                                                    const float2* __restrict__ uv, float g1, float g2, FaceAcc acc,
                                                    uint16_t* __restrict__ queue) {
    return face_item_rows<kVerify, kVec>(q, H, W, T, t, ib, j0, mask_out, mask_in, uv, g1, g2, acc, queue);
}

// The vertices of rows [i_from, ib + kFaceRows) of an interior item whose
// cube shares no strict sign, tested one by one (corners from L2): the
// interior path's fallback once its queue is full (rough fields).
template <bool kVerify>
__device__ __noinline__ uint2 face_rescan(const int2* __restrict__ q, int H, int W, int T, int t, int ib, int j0,
                                          int i_from, uint16_t* __restrict__ mask_out,
                                          const uint16_t* __restrict__ mask_in) {
    const int lane = threadIdx.x & 31;
    const size_t base = (size_t)t * H * W;
    uint2 r = make_uint2(0u, 0u);
    if (lane < 31) {
        for (int i = i_from; i < ib + kFaceRows; ++i) {
            for (int d = 0; d < 2; ++d) {
                const int j = j0 + 2 * lane + d;
                int2 c[8];
                unsigned w[8];
#pragma unroll
                for (int n = 0; n < 8; ++n)
                    c[n] = corner<kVerify>(q, H, W, T, t + (n >> 2), i + ((n >> 1) & 1), j + (n & 1), w[n]);
                const unsigned all = w[0] & w[1] & w[2] & w[3] & w[4] & w[5] & w[6] & w[7];
                if (all & kSignBits) continue;  // handled by the row loop
                const unsigned m = exact_mask(c, w, owned_valid(H, W, T, t, i, j));
                const size_t v = base + (size_t)i * W + j;
                if (kVerify) {
                    const unsigned x = m ^ (unsigned)mask_in[v];
                    r.x += __popc(x & 3u);
                    r.y += __popc(x & 0xffcu);
                } else {
                    mask_out[v] = (uint16_t)m;
                    r.x += __popc(m);
                }
            }
        }
    }
    return r;
}

// Interior items (W even; rows ib .. ib + kFaceRows, columns j0 .. j0 + 63
// and slice t + 1 inside the field): every corner exists, so the sign words
// need no validity selects.  The rows of slices t and t + 1 stream through
// a per-warp ring of kRing shared-memory stages filled by 16-byte async
// copies, kRing rows ahead of the one in use; a lane reads back only what
// its own copies wrote.
template <bool kOne>
__device__ __forceinline__ float x_hat(int q, float g1, float g2) {
    return kOne ? __fmul_rn(__int2float_rn(q), g1) : __fmul_rn(__fmul_rn(__int2float_rn(q), g1), g2);
}

constexpr int kRing = 4;
struct FaceRing {
    int4 r[kRing][2][32];  // [stage][slice t, t + 1][lane]
};

// kOne: 2^-k is a normal float (in g1, g2 = 1), so one multiply forms
// x_hat = qhat * 2^-k with the same single rounding as the two-step product.
template <bool kVerify, bool kOne = false>
__device__ __forceinline__ void face_item_inner(const int2* __restrict__ q, int H, int W, int T, int t, int ib,
                                                int j0, uint16_t* __restrict__ mask_out,
                                                const uint16_t* __restrict__ mask_in,
                                                const float2* __restrict__ uv, float g1, float g2, FaceAcc& acc,
                                                uint16_t* __restrict__ queue, FaceRing& ring) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const bool own = lane < 31;
    const int c0 = j0 + 2 * lane;
    const size_t sl = (size_t)H * W, base = (size_t)t * sl;
    const int2* src = q + base + (size_t)ib * W + c0;  // (t, ib, c0)
#pragma unroll
    for (int s = 0; s < kRing; ++s) {
        cp_async16(&ring.r[s][0][lane], src + (size_t)s * W, true);
        cp_async16(&ring.r[s][1][lane], src + sl + (size_t)s * W, true);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const int2* nxt = src + (size_t)kRing * W;  // the next row to fetch
    int stage = 0, nq = 0, i_over = ib + kFaceRows;  // i_over: first row not queued
    unsigned cw0 = 0, cw1 = 0;  // column words (slices t and t + 1) of the row above
    int4 above = make_int4(0, 0, 0, 0);  // its slice-t values (verification)
    unsigned omN = 0;
    float4 oxN = make_float4(0.f, 0.f, 0.f, 0.f);
    if (kVerify) orig_row<true>(mask_in, uv, base + (size_t)ib * W, c0, own, own, omN, oxN);
    for (int r = 0; r <= kFaceRows; ++r) {
        // row ib + r of both slices has landed once at most kRing - 1 newer
        // copy groups are pending
        asm volatile("cp.async.wait_group %0;" ::"n"(kRing - 1) : "memory");
        int4 a = ring.r[stage][0][lane], p = ring.r[stage][1][lane];
        if (kVerify) {
            a.y ^= kQhatTag;
            a.w ^= kQhatTag;
            p.y ^= kQhatTag;
            p.w ^= kQhatTag;
        }
        const unsigned w0 = sign_word(a.x, a.y) & sign_word(p.x, p.y);
        const unsigned w1 = sign_word(a.z, a.w) & sign_word(p.z, p.w);
        // the stage is refilled only after its values are in registers
        asm volatile("" ::"r"(w0), "r"(w1), "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w));
        if (r + kRing <= kFaceRows) {
            cp_async16(&ring.r[stage][0][lane], nxt, true);
            cp_async16(&ring.r[stage][1][lane], nxt + sl, true);
            nxt += W;
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        stage = stage + 1 == kRing ? 0 : stage + 1;
        if (r > 0) {
            // vertex row i = ib + r - 1: its cube is the row above and this one
            const int i = ib + r - 1;
            const size_t vrow = base + (size_t)i * W;
            const unsigned om = omN;
            const float4 ox = oxN;
            if (kVerify && r < kFaceRows) orig_row<true>(mask_in, uv, vrow + W, c0, own, own, omN, oxN);
            const unsigned vp0 = cw0 & w0, vp1 = cw1 & w1;
            const unsigned right = __shfl_down_sync(FULL, vp0, 1);
            const bool need0 = own && ((vp0 & vp1 & kSignBits) == 0u);
            const bool need1 = own && ((vp1 & right & kSignBits) == 0u);
            if (__any_sync(FULL, need0 || need1) && i_over > i) {
                const unsigned b0 = __ballot_sync(FULL, need0), b1 = __ballot_sync(FULL, need1);
                const int add = __popc(b0) + __popc(b1);
                if (nq + add > kQueueCap) {
                    i_over = i;  // this row and the rest: face_rescan
                } else {
                    int pos = nq + __popc(b0 & lt) + __popc(b1 & lt);
                    const uint16_t e = (uint16_t)(((i - ib) << 6) | (2 * lane));
                    if (need0) queue[pos++] = e;
                    if (need1) queue[pos] = (uint16_t)(e + 1);
                    nq += add;
                }
            }
            if (kVerify) {
                // a queued vertex is counted after its exact test
                const unsigned x = om & ~((need0 ? 0x0000ffffu : 0u) | (need1 ? 0xffff0000u : 0u));
                acc.ms += __popc(x & 0x00030003u);
                acc.mb += __popc(x & 0x0ffc0ffcu);
                if (own) {
                    // x_hat = qhat * 2^-k, exact in FP32 (|qhat| < 2^24)
                    const float ax = x_hat<kOne>(above.x, g1, g2), ay = x_hat<kOne>(above.y, g1, g2);
                    const float bx = x_hat<kOne>(above.z, g1, g2), by = x_hat<kOne>(above.w, g1, g2);
                    err_acc(acc, ax, ox.x);
                    err_acc(acc, ay, ox.y);
                    err_acc(acc, bx, ox.z);
                    err_acc(acc, by, ox.w);
                }
            } else if (own) {
                // a vertex that passes no test has every owned face uncrossed;
                // a queued one is written by its exact test
                if (!(need0 | need1))
                    *reinterpret_cast<unsigned*>(mask_out + vrow + c0) = 0u;
                else if (!need0)
                    mask_out[vrow + c0] = 0;
                else if (!need1)
                    mask_out[vrow + c0 + 1] = 0;
            }
        }
        cw0 = w0;
        cw1 = w1;
        above = a;
    }
    if (nq) add_exact(acc, face_exact<kVerify>(q, H, W, T, t, ib, j0, mask_out, mask_in, queue, nq), kVerify);
    if (i_over < ib + kFaceRows)
        add_exact(acc, face_rescan<kVerify>(q, H, W, T, t, ib, j0, i_over, mask_out, mask_in), kVerify);
}

struct FaceGrid {
    int nstrips, nchunks;
    long long items;
};
// work items over t_count slices
__host__ __device__ inline FaceGrid face_grid(int H, int W, int t_count) {
    FaceGrid g;
    g.nstrips = (W + kStrip - 1) / kStrip;
    g.nchunks = (H + kFaceRows - 1) / kFaceRows;
    g.items = (long long)t_count * g.nchunks * g.nstrips;
    return g;
}

// Work items run in slice order (then row chunk, then strip) over a grid of
// warps, so that slice t + 1, read again as slice t, is still in L2.
template <bool kVerify, bool kVec, bool kOne = false>
__global__ void __launch_bounds__(256, 4) face_kernel(const int2* __restrict__ q, int H, int W, int T,
                                                   uint16_t* __restrict__ mask_out,
                                                   const uint16_t* __restrict__ mask_in,
                                                   const float2* __restrict__ uv, float g1, float g2,
                                                   unsigned long long* __restrict__ ncrossed,
                                                   VerifyOut* __restrict__ vout, int t_first, int t_count) {
    const FaceGrid g = face_grid(H, W, t_count);
    const long long per_t = (long long)g.nchunks * g.nstrips;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    __shared__ uint16_t s_queue[8][kQueueCap];
    __shared__ FaceRing s_ring[8];
    static_assert(sizeof(FaceRing) >= kFaceRows * kStrip * sizeof(uint16_t), "queue of a general item");
    FaceAcc acc{0ull, 0u, 0u, ErrMax{0.f, 0.f}, 0.f};
    for (long long item = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < g.items;
         item += nwarps) {
        const int tr = (int)(item / per_t);
        const long long r = item - (long long)tr * per_t;
        const int t = t_first + tr;
        const int ib = (int)(r / g.nstrips) * kFaceRows;
        const int j0 = (int)(r % g.nstrips) * kStrip;
        uint16_t* const wq = reinterpret_cast<uint16_t*>(&s_ring[threadIdx.x >> 5]);
        const bool inner = ib + kFaceRows < H && j0 + 64 <= W && t + 1 < T;
        if (!kVerify && kVec && inner)
            acc = face_item_rows<kVerify, kVec, true>(q, H, W, T, t, ib, j0, mask_out, mask_in, uv, g1, g2, acc, wq);
        else if (!kVerify || !kVec)
            acc = face_item_rows<kVerify, kVec>(q, H, W, T, t, ib, j0, mask_out, mask_in, uv, g1, g2, acc, wq);
        else if (inner)
            face_item_inner<kVerify, kOne>(q, H, W, T, t, ib, j0, mask_out, mask_in, uv, g1, g2, acc,
                                     s_queue[threadIdx.x >> 5], s_ring[threadIdx.x >> 5]);
        else
            acc = face_item_rows_call<kVerify, kVec>(q, H, W, T, t, ib, j0, mask_out, mask_in, uv, g1, g2, acc, wq);
    }
    // warp, then block reduction; one set of atomics per block
    __shared__ unsigned long long s_c[8];
    __shared__ unsigned s_ms[8], s_mb[8];
    __shared__ float s_s[8], s_e[8], s_q[8];
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (kVerify) {
            acc.ms += __shfl_xor_sync(0xffffffffu, acc.ms, o);
            acc.mb += __shfl_xor_sync(0xffffffffu, acc.mb, o);
            acc.sq = __fadd_rn(acc.sq, __shfl_xor_sync(0xffffffffu, acc.sq, o));
            ErrMax p{__shfl_xor_sync(0xffffffffu, acc.em.s, o), __shfl_xor_sync(0xffffffffu, acc.em.e, o)};
            acc.em = err_max(acc.em, p);
        } else {
            acc.crossed += __shfl_xor_sync(0xffffffffu, acc.crossed, o);
        }
    }
    if ((threadIdx.x & 31) == 0) {
        s_c[w] = acc.crossed;
        s_ms[w] = acc.ms;
        s_mb[w] = acc.mb;
        s_s[w] = acc.em.s;
        s_e[w] = acc.em.e;
        s_q[w] = acc.sq;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        if (kVerify) {
            unsigned long long ms = 0, mb = 0;
            ErrMax em{0.f, 0.f};
            double sq = 0.0;
            for (int k = 0; k < nw; ++k) {
                ms += s_ms[k];
                mb += s_mb[k];
                em = err_max(em, ErrMax{s_s[k], s_e[k]});
                sq += (double)s_q[k];
            }
            if (ms) atomicAdd(&vout->mismatch_slice, ms);
            if (mb) atomicAdd(&vout->mismatch_slab, mb);
            // the exact largest difference rounded once; >= 0, so its bit
            // pattern orders like an unsigned integer
            const double err = (double)em.s + (double)em.e;
            if (err > 0.0) atomicMax(&vout->linf_bits, (unsigned long long)__double_as_longlong(err));
            if (sq > 0.0) atomicAdd(&vout->sq_err, sq);
        } else {
            unsigned long long c = 0;
            for (int k = 0; k < nw; ++k) c += s_c[k];
            if (c) atomicAdd(ncrossed, c);
        }
    }
}

// ---------------------------------------------------------------------------
// Repair of a failed verification (reading R14: the paper leaves the policy
// open).  flags[v] = 1 for every vertex of a face whose predicate differs
// between the original and the reconstruction, and for every vertex whose
// reconstruction breaks the pointwise bound; force_lossless_kernel then
// sets the classification of the flagged vertices to "lossless" (bound 0,
// no face left to evaluate) for the next encoding.
// ---------------------------------------------------------------------------
__device__ __constant__ const unsigned char kFaceCorner[12][3] = {
#define CPT_FC(ty, a, b, c) {a, b, c},
    CPT_OWNED_FACES(CPT_FC)
#undef CPT_FC
};

__global__ void __launch_bounds__(256) repair_flags_kernel(const int2* __restrict__ qhat, const float2* __restrict__ uv,
                                                           const uint16_t* __restrict__ m_orig,
                                                           const uint16_t* __restrict__ m_rec, int H, int W, int T,
                                                           int k, double bound, uint8_t* __restrict__ flags) {
    const size_t N = (size_t)H * W * T;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        const unsigned diff = (unsigned)(m_orig[v] ^ m_rec[v]);
        const int j = (int)(v % (size_t)W);
        const size_t r = v / (size_t)W;
        const int i = (int)(r % (size_t)H), t = (int)(r / (size_t)H);
        for (unsigned d = diff; d; d &= d - 1) {
            const int ty = __ffs(d) - 1;
            for (int c = 0; c < 3; ++c) {
                const int n = kFaceCorner[ty][c];
                const int tt = t + (n >> 2), ii = i + ((n >> 1) & 1), jj = j + (n & 1);
                if (tt < T && ii < H && jj < W) flags[((size_t)tt * H + ii) * W + jj] = 1;
            }
        }
        const int2 q = qhat[v];
        const float2 x = uv[v];
        const double eu = fabs(ldexp((double)q.x, -k) - (double)x.x), ev = fabs(ldexp((double)q.y, -k) - (double)x.y);
        if (!(eu <= bound) || !(ev <= bound)) flags[v] = 1;
    }
}

__global__ void __launch_bounds__(256) force_lossless_kernel(const uint8_t* __restrict__ flags, int H, int W, int T,
                                                             int2* __restrict__ cls) {
    const size_t N = (size_t)H * W * T;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        if (!flags[v]) continue;
        const int j = (int)(v % (size_t)W);
        const size_t r = v / (size_t)W;
        const int i = (int)(r % (size_t)H), t = (int)(r / (size_t)H);
        // strip-diagonal position of (t, i, j): strip i / 32, step j + i % 32, lane i % 32
        const size_t dv =
            (((size_t)t * ((H + 31) >> 5) + (i >> 5)) * (size_t)(W + 31) + (j + (i & 31))) * 32 + (i & 31);
        cls[dv] = make_int2(0, 0);
    }
}

void launch_repair_flags(const int32_t* qhat, const float* uv, const uint16_t* m_orig, const uint16_t* m_rec, int H,
                         int W, int T, int k, double bound, uint8_t* flags, cudaStream_t s) {
    repair_flags_kernel<<<1216, 256, 0, s>>>(reinterpret_cast<const int2*>(qhat), reinterpret_cast<const float2*>(uv),
                                             m_orig, m_rec, H, W, T, k, bound, flags);
}

void launch_force_lossless(const uint8_t* flags, int H, int W, int T, int2* cls, cudaStream_t s) {
    force_lossless_kernel<<<1216, 256, 0, s>>>(flags, H, W, T, cls);
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

// One wave of resident blocks (8 warps each) walks the work items; one set
// of atomics per block.
template <bool kVerify, bool kVec>
static unsigned face_blocks(int H, int W, int t_count) {
    static int resident = 0;
    if (!resident) {
        int dev = 0, nsm = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
            nsm = 152;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, face_kernel<kVerify, kVec>, 256, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        resident = nsm * per_sm;
    }
    const long long want = (face_grid(H, W, t_count).items + 7) / 8;
    return (unsigned)std::max(1ll, std::min(want, (long long)resident));
}

void launch_face_masks(const int32_t* q, int H, int W, int T, uint16_t* mask, unsigned long long* ncrossed,
                       cudaStream_t s, int t_first, int t_count) {
    if (t_count < 0) t_count = T - t_first;
    if (t_count <= 0) return;
    const int2* q2 = reinterpret_cast<const int2*>(q);
    if (W % 2 == 0)
        face_kernel<false, true><<<face_blocks<false, true>(H, W, t_count), 256, 0, s>>>(
            q2, H, W, T, mask, nullptr, nullptr, 0.f, 0.f, ncrossed, nullptr, t_first, t_count);
    else
        face_kernel<false, false><<<face_blocks<false, false>(H, W, t_count), 256, 0, s>>>(
            q2, H, W, T, mask, nullptr, nullptr, 0.f, 0.f, ncrossed, nullptr, t_first, t_count);
}

void launch_verify(const int32_t* qhat, const uint16_t* mask, const float* uv, int H, int W, int T, int k,
                   VerifyOut* out, cudaStream_t s, int t_first, int t_count) {
    if (t_count < 0) t_count = T - t_first;
    if (t_count <= 0) return;
    const int a = -k / 2, b = -k - a;
    const int2* q2 = reinterpret_cast<const int2*>(qhat);
    const float2* x2 = reinterpret_cast<const float2*>(uv);
    const float g1 = std::ldexp(1.0f, a), g2 = std::ldexp(1.0f, b);
    if (W % 2 == 0 && k >= -127 && k <= 126)  // 2^-k a normal float: one multiply
        face_kernel<true, true, true><<<face_blocks<true, true>(H, W, t_count), 256, 0, s>>>(
            q2, H, W, T, nullptr, mask, x2, std::ldexp(1.0f, -k), 1.0f, nullptr, out, t_first, t_count);
    else if (W % 2 == 0)
        face_kernel<true, true><<<face_blocks<true, true>(H, W, t_count), 256, 0, s>>>(
            q2, H, W, T, nullptr, mask, x2, g1, g2, nullptr, out, t_first, t_count);
    else
        face_kernel<true, false><<<face_blocks<true, false>(H, W, t_count), 256, 0, s>>>(
            q2, H, W, T, nullptr, mask, x2, g1, g2, nullptr, out, t_first, t_count);
}

}  // namespace cpt
