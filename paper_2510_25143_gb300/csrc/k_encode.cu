// Encoder kernels, launched once per slice t in raster order of slices
// (Alg. 3, loop over t):
//   sl_kernel    semi-Lagrangian predictions of slice t (Sec. VI-A)
//   mop_kernel   block-wise predictor choice of slice t (Sec. VI-B), which
//                also writes the SL predictions
//   pre_kernel   per vertex: membership of an incident face in C and the
//                Alg. 2 bound over the 22 incident faces that contain no
//                raster predecessor of the same slice (Alg. 4, first part)
//   wave_kernel  the dependency-carrying part: the 14 faces through raster
//                predecessors, xi quantisation, prediction and residual
//                quantisation with immediate write-back (Sec. V-A), run as a
//                warp-systolic anti-diagonal sweep that reproduces raster order.
#include "cpt_dev.cuh"
#include "cpt_internal.h"

namespace cpt {

constexpr int kStatusTimeout = -6;

__device__ __forceinline__ unsigned nb_valid(int H, int W, int T, int t, int i, int j) {
    unsigned tm = t > 0, tp = t + 1 < T, im = i > 0, ip = i + 1 < H, jm = j > 0, jp = j + 1 < W;
    return (tm & im & jm) | ((tm & im) << 1) | ((tm & jm) << 2) | (tm << 3) | ((im & jm) << 4) | (im << 5) |
           (jm << 6) | (jp << 7) | (ip << 8) | ((ip & jp) << 9) | (tp << 10) | ((tp & jp) << 11) |
           ((tp & ip) << 12) | ((tp & ip & jp) << 13);
}

// Loads the neighbours that do not belong to the current slice's raster
// predecessors: 0..3 from the reconstruction of slice t-1, 7..13 from the
// original field (slice t successors and slice t+1).  Invalid ones read 0.
__device__ __forceinline__ void load_far_neighbours(const int2* __restrict__ q, const int2* __restrict__ qhat,
                                                    int H, int W, int t, int i, int j, unsigned valid,
                                                    int2 nb[14]) {
    const size_t sl = (size_t)H * W;
    const size_t v = ((size_t)t * H + i) * W + j;
    const int2 z = make_int2(0, 0);
    nb[0] = (valid & (1u << 0)) ? __ldg(qhat + v - sl - W - 1) : z;
    nb[1] = (valid & (1u << 1)) ? __ldg(qhat + v - sl - W) : z;
    nb[2] = (valid & (1u << 2)) ? __ldg(qhat + v - sl - 1) : z;
    nb[3] = (valid & (1u << 3)) ? __ldg(qhat + v - sl) : z;
    nb[7] = (valid & (1u << 7)) ? __ldg(q + v + 1) : z;
    nb[8] = (valid & (1u << 8)) ? __ldg(q + v + W) : z;
    nb[9] = (valid & (1u << 9)) ? __ldg(q + v + W + 1) : z;
    nb[10] = (valid & (1u << 10)) ? __ldg(q + v + sl) : z;
    nb[11] = (valid & (1u << 11)) ? __ldg(q + v + sl + 1) : z;
    nb[12] = (valid & (1u << 12)) ? __ldg(q + v + sl + W) : z;
    nb[13] = (valid & (1u << 13)) ? __ldg(q + v + sl + W + 1) : z;
}

#define CPT_FACE(a, b)                                                                  \
    if (xi > 0 && ((valid >> (a)) & (valid >> (b)) & 1u))                               \
        xi = min_alg2(xi, nb[a].x, nb[a].y, nb[b].x, nb[b].y, qv.x, qv.y);

// ---------------------------------------------------------------------------
// pre_kernel: C membership of the 36 incident faces, the bound over the 22
// predecessor-free faces, and the set of the 14 predecessor faces that may
// still lower that bound once the predecessors are reconstructed.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr bool is_pred(int n) { return n >= 4 && n <= 6; }

#define CPT_PRED_MARK(a, b)                                                                       \
    if (((valid >> (a)) & (valid >> (b)) & 1u) &&                                                 \
        !pred_face_inert(nb[a], nb[b], qv, is_pred(a), is_pred(b), E, xi))                        \
        pm |= 1u << bit;                                                                          \
    ++bit;

__global__ void __launch_bounds__(256) pre_kernel(SliceArgs a) {
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int H = a.H, W = a.W, T = a.T, t = a.t;
    if (i >= H || j >= W) return;
    bool crossed = false;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        int ot = t + kOwners[o].dt, oi = i + kOwners[o].di, oj = j + kOwners[o].dj;
        if (ot >= 0 && oi >= 0 && oj >= 0)
            crossed |= (__ldg(a.mask + ((size_t)ot * H + oi) * W + oj) & kOwners[o].types) != 0;
    }
    int xi = 0;
    unsigned pm = 0;
    if (!crossed && a.eps_int > 0) {
        xi = a.eps_int;
        const unsigned valid = nb_valid(H, W, T, t, i, j);
        int2 nb[14];
        load_far_neighbours(a.q, a.qhat, H, W, t, i, j, valid, nb);
        const size_t v = ((size_t)t * H + i) * W + j;
        const int2 qv = __ldg(a.q + v);
        CPT_FREE_FACES(CPT_FACE)
        if (xi > 0) {
            const int2 z = make_int2(0, 0);
            nb[4] = (valid & (1u << 4)) ? __ldg(a.q + v - W - 1) : z;
            nb[5] = (valid & (1u << 5)) ? __ldg(a.q + v - W) : z;
            nb[6] = (valid & (1u << 6)) ? __ldg(a.q + v - 1) : z;
            const int E = 1 << (31 - __clz(a.eps_int));
            int bit = 0;
            CPT_PRED_FACES(CPT_PRED_MARK)
        }
    }
    a.xi_part[(size_t)i * W + j] = xi;
    a.pmask[(size_t)i * W + j] = (uint16_t)pm;
}
#undef CPT_PRED_MARK

// ---------------------------------------------------------------------------
// sl_kernel: semi-Lagrangian predictions of every vertex of slice t >= 1.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sl_kernel(SliceArgs a) {
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int H = a.H, W = a.W;
    unsigned sub = 0, steps = 0;
    if (i < H && j < W) {
        const int2* P = a.qhat + (size_t)(a.t - 1) * H * W;
        int pu, pv;
        int md = sl_predict(P, H, W, i, j, a.cfl_x, a.cfl_y, pu, pv);
        a.psl[(size_t)i * W + j] = make_int2(pu, pv);
        sub = md > 0;
        steps = md;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sub += __shfl_xor_sync(0xffffffffu, sub, o);
        steps += __shfl_xor_sync(0xffffffffu, steps, o);
    }
    if ((threadIdx.x & 31) == 0 && sub) {
        atomicAdd(a.counters + 0, (unsigned long long)sub);
        atomicAdd(a.counters + 1, (unsigned long long)steps);
    }
}

// ---------------------------------------------------------------------------
// mop_kernel: one CTA per B x B block of slice t >= 1 (Sec. VI-B).
// ---------------------------------------------------------------------------
// log2(x) in Q32 for x >= 1: integer part from the bit length, then one
// fraction bit per squaring of the Q31 mantissa (binary logarithm by
// repeated squaring).
__device__ __forceinline__ unsigned long long log2_q32(unsigned x) {
    int e = 31 - __clz(x);
    unsigned long long m = ((unsigned long long)x << 31) >> e;  // [2^31, 2^32)
    unsigned long long r = (unsigned long long)e << 32;
    for (int b = 31; b >= 0; --b) {
        m = (m * m) >> 31;
        if (m >= (1ull << 32)) {
            m >>= 1;
            r |= 1ull << b;
        }
    }
    return r;
}

// Score in Q32 bits per sample: H0 + 16 L/(n+L) + 1/(2 B^2), over the
// symbols of the sampled sites (0 marks an overflow).
__device__ long long block_score(const unsigned* smp, int nslots, int B, long long* red, int* cnt) {
    const int tid = threadIdx.x;
    if (tid == 0) { red[0] = 0; cnt[0] = 0; cnt[1] = 0; }
    __syncthreads();
    for (int k = tid; k < nslots; k += blockDim.x) {
        unsigned x = smp[k];
        if (x == 0) { atomicAdd(cnt + 1, 1); continue; }
        atomicAdd(cnt, 1);
        int c = 0;
        bool first = true;
        for (int m = 0; m < nslots; ++m) {
            if (smp[m] == x) {
                ++c;
                if (m < k) first = false;
            }
        }
        if (first) atomicAdd((unsigned long long*)red, (unsigned long long)((long long)c * (long long)log2_q32(c)));
    }
    __syncthreads();
    long long nv = cnt[0], nf = cnt[1];
    long long h0 = 0;
    if (nv > 0) h0 = ((long long)nv * (long long)log2_q32((unsigned)nv) - red[0]) / nv;
    long long pen = 0;
    if (nv + nf > 0) pen = (long long)(((unsigned long long)(16 * nf) << 32) / (unsigned long long)(nv + nf));
    long long meta = (long long)((1ull << 32) / (unsigned long long)(2 * B * B));
    __syncthreads();
    return h0 + pen + meta;
}

__global__ void __launch_bounds__(1024) mop_kernel(SliceArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const int B = a.B, n = a.n, H = a.H, W = a.W, t = a.t;
    int2* cand = reinterpret_cast<int2*>(smem_raw);                       // (B+1)^2
    unsigned* s3 = reinterpret_cast<unsigned*>(cand + (B + 1) * (B + 1));  // 2 B^2
    unsigned* ss = s3 + 2 * B * B;                                         // 2 B^2
    __shared__ long long red[1];
    __shared__ int cnt[3];
    const int tid = threadIdx.x, bi = tid / B, bj = tid % B;
    const int i0 = blockIdx.y * B, j0 = blockIdx.x * B;
    const int i = i0 + bi, j = j0 + bj;
    const bool inb = i < H && j < W;
    const size_t sl = (size_t)H * W;
    const int2* P = a.qhat + (size_t)(t - 1) * sl;
    const int2* Qt = a.q + (size_t)t * sl;
    const int xiq = 1 << (31 - __clz(a.eps_int));
    if (tid == 0) cnt[2] = 0;
    for (int k = tid; k < (B + 1) * (B + 1); k += blockDim.x) {
        int ii = i0 - 1 + k / (B + 1), jj = j0 - 1 + k % (B + 1);
        cand[k] = (ii >= 0 && jj >= 0 && ii < H && jj < W) ? Qt[(size_t)ii * W + jj] : make_int2(0, 0);
    }
    int2 qv = make_int2(0, 0), p0 = qv, p1 = qv, p2 = qv, p3 = qv;
    unsigned ssu = 0, ssv = 0, sub = 0, steps = 0;
    if (inb) {
        qv = Qt[(size_t)i * W + j];
        int pu, pv;
        int md = sl_predict(P, H, W, i, j, a.cfl_x, a.cfl_y, pu, pv);
        a.psl[(size_t)i * W + j] = make_int2(pu, pv);
        sub = md > 0;
        steps = md;
        int dummy;
        ssu = quantize(qv.x, pu, xiq, dummy);
        ssv = quantize(qv.y, pv, xiq, dummy);
        if (i > 0 && j > 0) p0 = P[(size_t)(i - 1) * W + j - 1];
        if (i > 0) p1 = P[(size_t)(i - 1) * W + j];
        if (j > 0) p2 = P[(size_t)i * W + j - 1];
        p3 = P[(size_t)i * W + j];
    }
    __syncthreads();
    unsigned s3u = 0, s3v = 0;
    for (int s = 0; s <= 2 * (B - 1); ++s) {
        if (inb && bi + bj == s) {
            const int2 up = cand[bi * (B + 1) + bj + 1], left = cand[(bi + 1) * (B + 1) + bj],
                       ul = cand[bi * (B + 1) + bj];
            int pu = up.x + left.x + p3.x - ul.x - p1.x - p2.x + p0.x;
            int pv = up.y + left.y + p3.y - ul.y - p1.y - p2.y + p0.y;
            int2 r;
            s3u = quantize(qv.x, pu, xiq, r.x);
            s3v = quantize(qv.y, pv, xiq, r.y);
            cand[(bi + 1) * (B + 1) + bj + 1] = r;
        }
        __syncthreads();
    }
    // sampled sites: (i, j) with i % n == 0 and j % n == 0
    const bool sampled = inb && (i % n == 0) && (j % n == 0);
    if (sampled) {
        int slot = atomicAdd(cnt + 2, 1);
        s3[2 * slot] = s3u;
        s3[2 * slot + 1] = s3v;
        ss[2 * slot] = ssu;
        ss[2 * slot + 1] = ssv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sub += __shfl_xor_sync(0xffffffffu, sub, o);
        steps += __shfl_xor_sync(0xffffffffu, steps, o);
    }
    if ((tid & 31) == 0 && sub) {
        atomicAdd(a.counters + 0, (unsigned long long)sub);
        atomicAdd(a.counters + 1, (unsigned long long)steps);
    }
    __syncthreads();
    const int nslots = 2 * cnt[2];
    long long r3 = block_score(s3, nslots, B, red, cnt);
    long long rs = block_score(ss, nslots, B, red, cnt);
    if (tid == 0) {
        unsigned char m = (1000 * rs < 997 * r3) ? 1 : 0;
        a.modes[((size_t)t * a.nby + blockIdx.y) * a.nbx + blockIdx.x] = m;
        if (m) atomicAdd(a.counters + 2, 1ull);
    }
}

// ---------------------------------------------------------------------------
// wave_kernel: one warp per strip of 32 rows of slice t; lane l handles row
// 32*strip + l and at step k column k - l, so each lane receives the
// reconstruction of (i-1, j) from lane l-1 one step after it was produced.
// Row 32*strip - 1 comes from the previous strip through global memory,
// published by its lane 31 with release stores and read after an acquire.
// Strips take tickets in launch order, so a strip only ever waits for a
// strip that started before it; every wait is bounded in time and sets the
// status word on expiry.
// ---------------------------------------------------------------------------
struct StepIn {
    int2 qv;
    int xi;
    unsigned pm;
    int2 psl;
    unsigned use_sl;
    int2 nb[14];
};

__device__ __forceinline__ void load_step(const SliceArgs& a, int i, int j, StepIn& in) {
    const int H = a.H, W = a.W, t = a.t;
    in.xi = 0;
    in.pm = 0;
    in.use_sl = 0;
    if (i >= H || j < 0 || j >= W) return;
    const size_t v = ((size_t)t * H + i) * W + j;
    in.qv = __ldg(a.q + v);
    in.xi = __ldg(a.xi_part + (size_t)i * W + j);
    if (in.xi > 0) {
        in.pm = __ldg(a.pmask + (size_t)i * W + j);
        const unsigned valid = nb_valid(H, W, a.T, t, i, j);
        if (t >= 1 && (a.pred == 1 || (a.pred == 2 && a.modes[((size_t)t * a.nby + i / a.B) * a.nbx + j / a.B]))) {
            in.use_sl = 1;
            in.psl = __ldg(a.psl + (size_t)i * W + j);
        }
        if (in.pm) {
            load_far_neighbours(a.q, a.qhat, H, W, t, i, j, valid, in.nb);
        } else if (!in.use_sl) {
            const size_t sl = (size_t)H * W;
            const int2 z = make_int2(0, 0);
            in.nb[0] = (valid & 1u) ? __ldg(a.qhat + v - sl - W - 1) : z;
            in.nb[1] = (valid & 2u) ? __ldg(a.qhat + v - sl - W) : z;
            in.nb[2] = (valid & 4u) ? __ldg(a.qhat + v - sl - 1) : z;
            in.nb[3] = (valid & 8u) ? __ldg(a.qhat + v - sl) : z;
        }
    }
}

#define CPT_PRED_EVAL(a, b)                                                                       \
    if ((pm >> bit) & 1u) r = min(r, min_alg2(xi, nb[a].x, nb[a].y, nb[b].x, nb[b].y, qv.x, qv.y)); \
    ++bit;

constexpr int kPublishEvery = 16;  // columns between progress publications

__global__ void __launch_bounds__(32) wave_kernel(SliceArgs a) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    const int H = a.H, W = a.W, T = a.T, t = a.t;
    const int nstrips = (H + 31) / 32;
    int s = 0;
    if (lane == 0) s = (int)atomicAdd(a.ticket + t, 1u);
    s = __shfl_sync(FULL, s, 0);
    const int i = s * 32 + lane;
    const bool rowok = i < H;
    const size_t base = (size_t)t * H * W;
    unsigned* prog_prev = a.progress + (size_t)t * nstrips + (s > 0 ? s - 1 : 0);
    unsigned* prog_me = a.progress + (size_t)t * nstrips + s;
    int2 left = make_int2(0, 0), up = left, res = left;
    unsigned known = 0;
    StepIn cur, nxt;
    load_step(a, i, -lane, cur);
    for (int k = 0; k < W + 31; ++k) {
        const int j = k - lane;
        load_step(a, i, j + 1, nxt);
        int2 fromprev;
        fromprev.x = __shfl_up_sync(FULL, res.x, 1);
        fromprev.y = __shfl_up_sync(FULL, res.y, 1);
        const int2 upleft = up;
        int abort = 0;
        if (lane == 0) {
            if (s == 0 || j >= W) {
                up = make_int2(0, 0);
            } else {
                if ((unsigned)j >= known) {
                    unsigned long long t0 = 0;
                    for (;;) {
                        unsigned p = ld_acquire(prog_prev);
                        if (p > (unsigned)j) { known = p; break; }
                        if (*(volatile int*)a.status != 0) { abort = 1; break; }
                        unsigned long long now = global_ns();
                        if (t0 == 0) t0 = now;
                        else if ((long long)(now - t0) > a.timeout_ns) {
                            atomicCAS(a.status, 0, kStatusTimeout);
                            abort = 1;
                            break;
                        }
                    }
                }
                if (!abort) up = __ldcg(a.qhat + base + (size_t)(i - 1) * W + j);
            }
        } else {
            up = fromprev;
        }
        abort = __shfl_sync(FULL, abort, 0);
        if (abort) return;
        const bool active = rowok && j >= 0 && j < W;
        if (active) {
            int xi = cur.xi;
            const int2 qv = cur.qv;
            if (xi > 0 && cur.pm) {
                cur.nb[4] = upleft;
                cur.nb[5] = up;
                cur.nb[6] = left;
                const int2* nb = cur.nb;
                const unsigned pm = cur.pm;
                int r = xi, bit = 0;
                CPT_PRED_FACES(CPT_PRED_EVAL)
                xi = r;
            }
            const int code = xi_code(xi);
            int2 rec = qv;
            unsigned sym = 0;
            if (code > 0) {
                int pu, pv;
                if (cur.use_sl) {
                    pu = cur.psl.x;
                    pv = cur.psl.y;
                } else {
                    pu = up.x + left.x + cur.nb[3].x - upleft.x - cur.nb[1].x - cur.nb[2].x + cur.nb[0].x;
                    pv = up.y + left.y + cur.nb[3].y - upleft.y - cur.nb[1].y - cur.nb[2].y + cur.nb[0].y;
                }
                unsigned su = quantize_code(qv.x, pu, code, rec.x);
                unsigned sv = quantize_code(qv.y, pv, code, rec.y);
                sym = su | (sv << 16);
            }
            const size_t v = base + (size_t)i * W + j;
            a.qhat[v] = rec;
            a.qxi[v] = (uint8_t)code;
            a.sym[v] = sym;
            if (a.xi_out) a.xi_out[v] = xi;
            res = rec;
            if (lane == 31 && ((j % kPublishEvery) == kPublishEvery - 1 || j == W - 1))
                st_release(prog_me, (unsigned)(j + 1));
        } else {
            res = make_int2(0, 0);
        }
        left = res;
        cur = nxt;
    }
}
#undef CPT_PRED_EVAL

#undef CPT_FACE

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
int wave_strips(int H) { return (H + 31) / 32; }

void launch_pre(const SliceArgs& a, cudaStream_t s) {
    dim3 grid((a.W + 31) / 32, (a.H + 7) / 8);
    pre_kernel<<<grid, 256, 0, s>>>(a);
}

void launch_sl(const SliceArgs& a, cudaStream_t s) {
    dim3 grid((a.W + 31) / 32, (a.H + 7) / 8);
    sl_kernel<<<grid, 256, 0, s>>>(a);
}

void launch_mop(const SliceArgs& a, cudaStream_t s) {
    dim3 grid(a.nbx, a.nby);
    size_t smem = sizeof(int2) * (a.B + 1) * (a.B + 1) + sizeof(unsigned) * 4 * a.B * a.B;
    mop_kernel<<<grid, a.B * a.B, smem, s>>>(a);
}

void launch_wave(const SliceArgs& a, cudaStream_t s) {
    wave_kernel<<<wave_strips(a.H), 32, 0, s>>>(a);
}

}  // namespace cpt
