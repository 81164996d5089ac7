// Encoder kernels for the raster loop of Alg. 3.
//
// classify_kernel (fully parallel over every vertex of every slice) settles
// all of Alg. 4 that does not depend on reconstructions: whether an incident
// face is in C (the vertex is then lossless), the Alg. 2 bound over the 12
// faces whose other vertices still hold original values when the vertex is
// processed, and which of the 24 other faces (through slice t-1 or through a
// raster predecessor, whose reconstructions lie within +-E of the originals)
// could still lower that bound.
//
// encode_pipeline_kernel (one persistent launch over all slices of one field
// or of a batch of fields) does the rest, pipelining consecutive slices.  Its
// warps have one of two roles.
// wave(t, s)     rows 32s..32s+31 of slice t: the flagged faces with the actual
//                reconstructions, xi quantisation, prediction and residual
//                quantisation with immediate write-back (Sec. V-A).  Lane l
//                handles row 32s+l and, at step k, column k-l; the
//                reconstruction of (i-1, j) arrives from lane l-1 by shuffle,
//                the row above the strip from wave(t, s-1) and slice t-1 from
//                the waves of t-1 as tagged reconstruction words polled in
//                global memory.  The read-only inputs come from strip-diagonal
//                copies staged two chunks ahead into a shared-memory ring.
//                Wave warps take (field, t, s) from a ticket counter whose
//                order puts every wave an item depends on at a smaller ticket.
// prep units     (SL, MoP and the learned predictors) U x U squares of slice
//                t >= 1: semi-Lagrangian or learned predictions (Sec. VI-A) and
//                MoP block modes (Sec. VI-B).  A unit needs slice t-1 final
//                around it; the wave of slice t-1 that makes it so appends it
//                to a ready queue, and prep warps take the queue in order.
//                wave(t, s) waits for the units of each unit column.
// In decoding mode the same waves rebuild the reconstruction from the
// stream's codes (no face work) and MoP units read their modes.
// Waves wait only for waves with smaller tickets and for queued units; queued
// units wait for nothing but words already written.  Every warp is resident,
// so the pipeline cannot deadlock; each wait is bounded in time and sets the
// status word when it expires.
#include <algorithm>
#include <climits>
#include <type_traits>

#include "cpt_dev.cuh"
#include "cpt_internal.h"
#include "cpt_net.cuh"

namespace cpt {

constexpr int kPublishEvery = 8;   // steps between checks for prep units made ready
constexpr int kPrepShareSL = 45;   // percent of the warps working prep units (SL)
constexpr int kPrepShareMoP = 45;  // (MoP)
constexpr int kPrepShareNet = 65;  // (the learned predictors: the net's inference is the heavier side)
constexpr int kNoSL = (int)0x80000000;  // psl marker: the block keeps 3DL (no prediction reaches it)

__device__ __forceinline__ unsigned nb_valid(int H, int W, int T, int t, int i, int j) {
    unsigned tm = t > 0, tp = t + 1 < T, im = i > 0, ip = i + 1 < H, jm = j > 0, jp = j + 1 < W;
    return (tm & im & jm) | ((tm & im) << 1) | ((tm & jm) << 2) | (tm << 3) | ((im & jm) << 4) | (im << 5) |
           (jm << 6) | (jp << 7) | (ip << 8) | ((ip & jp) << 9) | (tp << 10) | ((tp & jp) << 11) |
           ((tp & ip) << 12) | ((tp & ip & jp) << 13);
}

__host__ __device__ constexpr bool is_uncertain(int n) { return n <= 6; }
constexpr unsigned kAllNeighbours = 0x3FFFu;  // nb_valid of an interior vertex
constexpr unsigned kAllUncFaces = (1u << 24) - 1u;  // every uncertain face present

// The CPT_UNC_FACES pairs as bytes (first | second << 4), face f in byte f % 8
// of word f / 8, for loops over a face mask.
constexpr unsigned long long kUncPairs0 = 0x8331733271208210ull;
constexpr unsigned long long kUncPairs1 = 0x50C6647554869330ull;
constexpr unsigned long long kUncPairs2 = 0x40A451A562A660B5ull;
__device__ __forceinline__ unsigned unc_pair(int f) {
    const unsigned long long w = f < 8 ? kUncPairs0 : (f < 16 ? kUncPairs1 : kUncPairs2);
    return (unsigned)(w >> (8 * (f & 7))) & 0xFFu;
}

#define CPT_FACE(a, b)                                                                  \
    if (xi > 0 && ((valid >> (a)) & (valid >> (b)) & 1u))                               \
        xi = min_alg2(xi, nb[a].x, nb[a].y, nb[b].x, nb[b].y, qv.x, qv.y);

#define CPT_UNC_MARK(a, b)                                                                   \
    if ((valid >> (a)) & (valid >> (b)) & 1u) {                                              \
        const int cls_ = unc_face_class(nb[a], nb[b], qv, is_uncertain(a), is_uncertain(b), E, xi); \
        if (cls_ == 2) um_full |= 1u << bit;                                                 \
        else if (cls_ == 1) um_m |= 1u << bit;                                               \
    }                                                                                        \
    ++bit;



// ---------------------------------------------------------------------------
// classify_kernel: out[v] = (bound over the certain faces, 0 = lossless;
// uncertain faces that need the full Alg. 2), out_m[v] = uncertain faces of
// which only M = 0 must be checked, in the strip-diagonal layout.  A block
// covers 32 columns x 32 rows of one slice.  Most vertices take the exact
// fast path (below); the others are queued in shared memory and classified
// at the end of the block with the full Alg. 2, one per thread, so that a
// rare slow vertex does not hold up the 31 fast ones of its warp.
// ---------------------------------------------------------------------------
constexpr int kClsRows = 32;

// The 14 neighbour values; an absent neighbour reads as the vertex's own
// value z (faces through it are never evaluated, and it passes the fast
// path's sign tests whenever the vertex itself does).
__device__ __forceinline__ void load_nb(const int2* __restrict__ q, size_t v, size_t sl, int W, unsigned valid,
                                        int2 nb[14], int2 z) {
    nb[0] = (valid & (1u << 0)) ? __ldg(q + v - sl - W - 1) : z;
    nb[1] = (valid & (1u << 1)) ? __ldg(q + v - sl - W) : z;
    nb[2] = (valid & (1u << 2)) ? __ldg(q + v - sl - 1) : z;
    nb[3] = (valid & (1u << 3)) ? __ldg(q + v - sl) : z;
    nb[4] = (valid & (1u << 4)) ? __ldg(q + v - W - 1) : z;
    nb[5] = (valid & (1u << 5)) ? __ldg(q + v - W) : z;
    nb[6] = (valid & (1u << 6)) ? __ldg(q + v - 1) : z;
    nb[7] = (valid & (1u << 7)) ? __ldg(q + v + 1) : z;
    nb[8] = (valid & (1u << 8)) ? __ldg(q + v + W) : z;
    nb[9] = (valid & (1u << 9)) ? __ldg(q + v + W + 1) : z;
    nb[10] = (valid & (1u << 10)) ? __ldg(q + v + sl) : z;
    nb[11] = (valid & (1u << 11)) ? __ldg(q + v + sl + 1) : z;
    nb[12] = (valid & (1u << 12)) ? __ldg(q + v + sl + W) : z;
    nb[13] = (valid & (1u << 13)) ? __ldg(q + v + sl + W + 1) : z;
}

__device__ __forceinline__ void store_cls(int2* __restrict__ out, unsigned* __restrict__ out_m,
                                          int2* __restrict__ qd, const int2* __restrict__ q, int H, int W, int t,
                                          int i, int j, size_t v, int xi, unsigned um_full, unsigned um_m) {
    // strip-diagonal position of (t, i, j): strip i / 32, step j + i % 32, lane i % 32
    const size_t dv = (((size_t)t * ((H + 31) >> 5) + (i >> 5)) * (size_t)(W + 31) + (j + (i & 31))) * 32 + (i & 31);
    out[dv] = make_int2(xi, (int)um_full);
    out_m[dv] = um_m;
    qd[dv] = __ldg(q + v);
}

__global__ void __launch_bounds__(256, 4) classify_kernel(const int2* __restrict__ q, const uint16_t* __restrict__ mask,
                                                       int H, int W, int T, int eps_int, int2* __restrict__ out,
                                                       unsigned* __restrict__ out_m, int2* __restrict__ qd,
                                                       int t_first) {
    __shared__ unsigned short s_slow[32 * kClsRows];  // (row in the block) * 32 + lane
    __shared__ int s_nslow;
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * 32 + lane;
    const int ib = blockIdx.y * kClsRows;
    const int t = t_first + (int)blockIdx.z;
    const size_t sl = (size_t)H * W;
    if (threadIdx.x == 0) s_nslow = 0;
    __syncthreads();
    for (int rr = threadIdx.x >> 5; rr < kClsRows; rr += 8) {
        const int i = ib + rr;
        bool slow = false;
        if (i < H && j < W) {
            const size_t v = ((size_t)t * H + i) * W + j;
            int xi = 0;
            unsigned um_m = 0;
            // the vertex's work, with a copy for interior vertices (every
            // neighbour present: the presence tests fold away)
            auto classify_vertex = [&](const unsigned valid) {
                // a crossed incident face: one of the eight owners' masks (the
                // owners lie at offsets (0..-1, 0..-1, 0..-1) from the vertex)
                bool crossed = false;
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    // owner present: t > 0, i > 0, j > 0 are bits 3, 5, 6 of valid
                    const bool ok = (kOwners[o].dt == 0 || ((valid >> 3) & 1u)) &&
                                    (kOwners[o].di == 0 || ((valid >> 5) & 1u)) &&
                                    (kOwners[o].dj == 0 || ((valid >> 6) & 1u));
                    const long long off = (long long)kOwners[o].dt * (long long)sl + (long long)kOwners[o].di * W +
                                          kOwners[o].dj;
                    if (ok) crossed |= (__ldg(mask + (long long)v + off) & kOwners[o].types) != 0;
                }
                if (!crossed && eps_int > 0) {
                    xi = eps_int;
                    const int2 qv = __ldg(q + v);
                    int2 nb[14];
                    load_nb(q, v, sl, W, valid, nb, qv);
                    const int E = 1 << (31 - __clz(eps_int));
                    // Fast path (exact): every existing neighbour keeps the vertex's
                    // strict sign of u (or of v), with margin E where its value may
                    // still change, and |q| - 1 >= eps'.  Then Alg. 2 keeps eps' on
                    // every face unless M = 0 (M = det(n_a - q, n_b - q)), and no
                    // uncertain face needs the full Alg. 2.  The sign tests are
                    // minima and maxima over the uncertain neighbours (0..6) and
                    // the others.
                    bool fast = false;
#pragma unroll
                    for (int c = 0; c < 2 && !fast; ++c) {
                        const int x0 = c ? qv.y : qv.x;
                        if (x0 == 0 || abs(x0) - 1 < eps_int) continue;
                        int lo_u = INT_MAX, hi_u = INT_MIN, lo_c = INT_MAX, hi_c = INT_MIN;
#pragma unroll
                        for (int k = 0; k < 14; ++k) {
                            const int x = c ? nb[k].y : nb[k].x;
                            if (is_uncertain(k)) {
                                lo_u = min(lo_u, x);
                                hi_u = max(hi_u, x);
                            } else {
                                lo_c = min(lo_c, x);
                                hi_c = max(hi_c, x);
                            }
                        }
                        fast = x0 > 0 ? (lo_c > 0 && lo_u > E) : (hi_c < 0 && hi_u < -E);
                    }
                    if (fast) {
                        // |differences| < 2^26: 32-bit, products widened (one 32 x 32 -> 64 multiply each)
                        int dx[14], dy[14];
#pragma unroll
                        for (int k = 0; k < 14; ++k) {
                            dx[k] = nb[k].x - qv.x;
                            dy[k] = nb[k].y - qv.y;
                        }
                        // M = 0 on a certain face: filtered on the low 32 bits of
                        // the two products, confirmed with the exact 64-bit ones
                        unsigned cand = 0;
                        int cbit = 0;
#define CPT_CERT_LO(a, b)                                                                                  \
        cand |= (((valid >> (a)) & (valid >> (b)) & 1u) &&                                                    \
                 (unsigned)dx[a] * (unsigned)dy[b] == (unsigned)dy[a] * (unsigned)dx[b] ? 1u : 0u) << cbit;   \
        ++cbit;
                        CPT_CERT_FACES(CPT_CERT_LO)
#undef CPT_CERT_LO
                        bool mz = false;
                        if (cand) {
                            cbit = 0;
#define CPT_CERT_M(a, b) \
        mz |= ((cand >> cbit) & 1u) && (long long)dx[a] * dy[b] == (long long)dy[a] * dx[b]; \
        ++cbit;
                            CPT_CERT_FACES(CPT_CERT_M)
#undef CPT_CERT_M
                        }
                        if (mz) {
                            xi = 0;
                        } else {
                            // every existing uncertain face keeps the same-sign
                            // clause; only its M = 0 check remains, done by the
                            // wave with the actual reconstructions (a face whose M
                            // cannot reach 0 passes that check anyway)
                            int bit = 0;
#define CPT_UNC_VALID(a, b) um_m |= ((valid >> (a)) & (valid >> (b)) & 1u) << bit; ++bit;
                            CPT_UNC_FACES(CPT_UNC_VALID)
#undef CPT_UNC_VALID
                        }
                    } else {
                        slow = true;
                    }
                }
            };
            const unsigned valid_nb = nb_valid(H, W, T, t, i, j);
            if (valid_nb == kAllNeighbours) classify_vertex(kAllNeighbours);
            else classify_vertex(valid_nb);
            if (!slow) store_cls(out, out_m, qd, q, H, W, t, i, j, v, xi, 0u, um_m);
        }
        // queue the slow vertices of the warp (one shared atomic per warp)
        const unsigned bal = __ballot_sync(0xffffffffu, slow);
        if (bal) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&s_nslow, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (slow) s_slow[base + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)(rr * 32 + lane);
        }
    }
    __syncthreads();
    // the full Alg. 2 over the 12 certain faces and the classes of the 24
    // uncertain ones for the queued vertices, one per thread
    const int nslow = s_nslow;
    for (int k = threadIdx.x; k < nslow; k += blockDim.x) {
        const unsigned e = s_slow[k];
        const int i = ib + (int)(e >> 5), jj = blockIdx.x * 32 + (int)(e & 31u);
        const size_t v = ((size_t)t * H + i) * W + jj;
        const unsigned valid = nb_valid(H, W, T, t, i, jj);
        const int2 qv = __ldg(q + v);
        int2 nb[14];
        load_nb(q, v, sl, W, valid, nb, qv);
        const int E = 1 << (31 - __clz(eps_int));
        int xi = eps_int;
        unsigned um_full = 0, um_m = 0;
        (void)E;
        CPT_CERT_FACES(CPT_FACE)
        if (xi > 0) {
            int bit = 0;
            CPT_UNC_FACES(CPT_UNC_MARK)
        }
        store_cls(out, out_m, qd, q, H, W, t, i, jj, v, xi, um_full, um_m);
    }
}

__device__ __forceinline__ unsigned warp_wait_geq(const SliceArgs& a, const unsigned* flag, unsigned target) {
    return warp_wait_geq(a.status, a.timeout_ns, flag, target);
}

// ---------------------------------------------------------------------------
// Reconstruction words.  Every reconstruction is written once, as one 64-bit
// word (x, y ^ kQhatTag) with a strong store; bits 30 and 31 of its y half
// differ (|y| < 2^30), those of the zeroed array do not.  A reader polls the
// word itself: the value and its presence travel together, so no fence is
// needed between the wave that writes it and the waves and prep units that
// read it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_word(const int2* p) {
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(w) : "l"(p));
    return w;
}
__device__ __forceinline__ void st_word(int2* p, int2 v) {
    const unsigned long long w =
        (unsigned long long)(unsigned)v.x | ((unsigned long long)(unsigned)(v.y ^ kQhatTag) << 32);
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ bool word_ready(unsigned long long w) {
    const int y = (int)(w >> 32);
    return ((y >> 30) ^ (y >> 31)) & 1;
}
__device__ __forceinline__ int2 word_value(unsigned long long w) {
    return make_int2((int)(unsigned)w, (int)(w >> 32) ^ kQhatTag);
}

// Re-reads *p until its word is ready, on the lanes with need; false (and the
// status word set) when the time limit expires or another warp failed.
__device__ bool poll_word(const SliceArgs& a, const int2* p, bool need, unsigned long long& w) {
    if (__all_sync(0xffffffffu, !need || word_ready(w))) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (need && !word_ready(w)) w = ld_word(p);
        if (__all_sync(0xffffffffu, !need || word_ready(w))) return true;
        const bool late = (long long)(global_ns() - t0) > a.timeout_ns;
        const bool failed = *(volatile int*)a.status != 0;
        if (__any_sync(0xffffffffu, late || failed)) {
            if ((threadIdx.x & 31u) == 0 && !failed) atomicCAS(a.status, 0, kStatusTimeout);
            return false;
        }
        __nanosleep(32);
    }
}

// Slice t-1 read through L2 for a semi-Lagrangian reach beyond the staged
// window: each word is awaited (it is present once the unit is queued; the
// wait is a bounded safeguard that sets the status word).
struct TaggedSlice {
    const int2* P;
    int W;
    int* status;
    long long timeout_ns;
    __device__ int2 at(int i, int j) const {
        const int2* p = P + (size_t)i * W + j;
        unsigned long long w = ld_word(p);
        if (!word_ready(w)) {
            const unsigned long long t0 = global_ns();
            while (!word_ready(w)) {
                if ((long long)(global_ns() - t0) > timeout_ns || *(volatile int*)status != 0) {
                    atomicCAS(status, 0, kStatusTimeout);
                    return make_int2(0, 0);
                }
                __nanosleep(32);
                w = ld_word(p);
            }
        }
        return word_value(w);
    }
};

// ---------------------------------------------------------------------------
// shared memory of one worker warp, sized by the predictor: prediction units
// of side at most UMAX (SL and MoP with blocks up to 16: 16; MoP blocks of
// 32: 32; none for 3DL) and, with NET, the learned predictor's scratch.  The
// smaller the slice, the more worker warps an SM holds.
// ---------------------------------------------------------------------------
constexpr int kStageR = 8;  // largest SL reach served from the staged window
template <int UMAX, bool NET>
struct PrepSmem {
    static constexpr int kPitch = UMAX + 2 + 2 * kStageR;  // pitch of the staged slice t-1 window
    int2 pp[kPitch * kPitch];              // qhat(t-1): rows/cols -1-R..U+R around the unit
    union {
        struct {                           // SL and MoP
            int2 qc[UMAX + 2][UMAX + 2];   // q(t): rows/cols -1..U around the unit
            int2 psl[UMAX][UMAX];          // SL predictions of the unit
            uint16_t smp[2][64 * UMAX];    // sampled symbols per mode, 2 B^2 slots per block
            unsigned hist[256];
            unsigned short list[UMAX * UMAX];  // sites (row * 32 + column) left for SL
            unsigned char modes[64];       // decisions of the unit's blocks
        };
        typename std::conditional<NET, NetScratch<8>, char>::type net;  // learned predictor (8 x 8 tiles)
    };
};
// A wave's read-only inputs, staged from the strip-diagonal arrays in chunks
// of kChunk steps (each step's 32 lanes contiguous), two chunks ahead, into
// three slots (slot = chunk mod 3): during chunk g the steps read chunks g
// and g + 1 (neighbours at steps k + 1, k + 2), while g + 2 is in flight.
constexpr int kChunk = 4;
struct alignas(16) WaveRing {
    int2 cl[3][kChunk][32];      // classification
    unsigned cm[3][kChunk][32];  // faces needing only the M = 0 check
    int2 q[3][kChunk][32];       // q(t)
    int2 qn[3][kChunk][32];      // q(t+1)
    int2 qb[3][kChunk];          // q(t) of the next strip's first row at column (consumer step - 31)
    int2 nb[3][kChunk];          // q(t+1) of the same
};
// The shared memory of a warp depends on its role: a prep warp holds a
// prediction unit's windows (PrepSlot), a wave warp the staging ring and the
// neighbour values of its face loops (WaveSlot).  A CTA holds its prep warps'
// slots, then its wave warps' slots, then (learned predictor) the net's
// second-layer weights.
template <int UMAX, bool NET>
struct alignas(16) PrepSlot {
    static constexpr int kUmax = UMAX;
    static constexpr bool kNet = NET;
    PrepSmem<UMAX, NET> prep;
    SliceArgs args;  // the field of the current unit (copied from the launch's field table)
};
struct alignas(16) WaveSlot {
    WaveRing ring;
    int2 nbs[32][15];  // per-lane neighbour values for the face loops
    SliceArgs args;    // the field of the current item (copied from the launch's field table)
};
template <int UMAX, bool NET>
constexpr size_t prep_slot_bytes() {
    if constexpr (UMAX > 0) return sizeof(PrepSlot<UMAX, NET>);
    else return 0;
}

// Copies the arguments of field f into the warp's shared slot.
template <class Sm>
__device__ __forceinline__ const SliceArgs& load_field(const SliceArgs* __restrict__ fields, int f, Sm& sm) {
    static_assert(sizeof(SliceArgs) % 4 == 0, "field arguments copied as words");
    constexpr int kWords = (int)(sizeof(SliceArgs) / 4);
    const unsigned* src = reinterpret_cast<const unsigned*>(fields + f);
    unsigned* dst = reinterpret_cast<unsigned*>(&sm.args);
    __syncwarp();
    for (int k = (int)(threadIdx.x & 31u); k < kWords; k += 32) dst[k] = __ldg(src + k);
    __syncwarp();
    return sm.args;
}

// ---------------------------------------------------------------------------
// prep units: semi-Lagrangian predictions and MoP modes
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

// Score of one block and mode in Q32 bits per sample (Eq. 10 plus the
// overflow penalty and the metadata term): H0 + 16 L/(n+L) + 1/(2 B^2).
// smp holds the nslots symbols of the block's sampled sites (0 = overflow).
__device__ long long warp_block_score(const uint16_t* smp, int nslots, int B, unsigned* hist,
                                      const unsigned long long* __restrict__ lg) {
    const int lane = (int)(threadIdx.x & 31u);
    const unsigned lo = (unsigned)kRadius - 128u;
    for (int k = lane; k < 256; k += 32) hist[k] = 0;
    __syncwarp();
    unsigned nv = 0, nf = 0;
    unsigned long long acc = 0;
    for (int k = lane; k < nslots; k += 32) {
        const unsigned x = smp[k];
        if (x == 0) { ++nf; continue; }
        ++nv;
        if (x - lo < 256u) {
            atomicAdd(&hist[x - lo], 1u);
        } else {
            // symbol outside the window: count its multiplicity directly
            unsigned c = 0;
            bool first = true;
            for (int m = 0; m < nslots; ++m) {
                if ((unsigned)smp[m] == x) {
                    ++c;
                    if (m < k) first = false;
                }
            }
            if (first) acc += (unsigned long long)c * __ldg(lg + c);
        }
    }
    __syncwarp();
    for (int k = lane; k < 256; k += 32) {
        unsigned h = hist[k];
        if (h) acc += (unsigned long long)h * __ldg(lg + h);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nv += __shfl_xor_sync(0xffffffffu, nv, o);
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    }
    long long h0 = 0;
    if (nv > 0) h0 = ((long long)nv * (long long)__ldg(lg + nv) - (long long)acc) / (long long)nv;
    long long pen = 0;
    if (nv + nf > 0) pen = (long long)(((unsigned long long)(16u * nf) << 32) / (unsigned long long)(nv + nf));
    const int lgB = __ffs(B) - 1;  // B is a power of two: 2^32 / (2 B^2) exactly
    long long meta = (long long)((1ull << 32) >> (2 * lgB + 1));
    __syncwarp();
    return h0 + pen + meta;
}

// MoP decisions of the blocks inside a prep unit (B divides U), from the
// staged window.  Lanes are grouped by block: lane l handles row l % B of
// block l / B of the current group of 32 / B blocks; the 3DL micro-encoding
// runs as an anti-diagonal sweep inside each block with the original slice t
// outside the block (context-preserving candidate buffer).  The SL symbols of
// the sampled sites come from psl.
template <class PS>
__device__ void mop_unit(const SliceArgs& a, int t, int r0, int c0, PS& ps, int Rw) {
    constexpr int kPP = PS::kPitch;
    const int lane = (int)(threadIdx.x & 31u), B = a.B, H = a.H, W = a.W;
    const int lgB = __ffs(B) - 1, lgN = __ffs(a.U) - 1 - lgB;  // B and U are powers of two
    const int nbu = 1 << lgN, nbt = nbu * nbu;                 // blocks per unit side, per unit
    const int bpp = 32 >> lgB;                                 // blocks per pass
    const int code = xi_code(a.eps_int);
    const int r = lane & (B - 1), bl = lane >> lgB;
    const int nslots = 2 * B * B;  // room per block; a block's sampled sites fill the first ones
    const FastDiv n(a.n);
    const int2* pp = ps.pp + (Rw + 1) * kPP + (Rw + 1);  // (0,0) = vertex (r0, c0) of slice t-1
    // sampled sites of the block at (ib, jb): rows and columns from the
    // first multiple of n, every n-th
    auto sampled = [&](int ib, int jb, int& fr, int& fc, int& nrs, int& ncs) {
        const int ih = min(B, H - ib), iw = min(B, W - jb);
        fr = (int)n.mod(n.d - n.mod(ib));
        fc = (int)n.mod(n.d - n.mod(jb));
        nrs = ih > fr ? (int)n.div(ih - fr + n.d - 1) : 0;
        ncs = iw > fc ? (int)n.div(iw - fc + n.d - 1) : 0;
    };
    for (int b0 = 0; b0 < nbt; b0 += bpp) {
        const int bi = b0 + bl;
        const int ib = r0 + ((bi >> lgN) << lgB), jb = c0 + ((bi & (nbu - 1)) << lgB);
        const int i = ib + r, li = i - r0;
        const bool live = bi < nbt && i < H && jb < W;
        int fr = 0, fc = 0, nrs = 0, ncs = 0;
        if (live) sampled(ib, jb, fr, fc, nrs, ncs);
        // this lane's row is sampled when r = fr (mod n); its slots start at
        // row_slot, and column jj = fc + n m takes slot row_slot + 2 m
        const bool row_s = live && r >= fr && n.mod(r - fr) == 0;
        const int row_slot = bl * nslots + (row_s ? 2 * (int)n.div(r - fr) * ncs : 0);
        __syncwarp();
        if (row_s) {
            int m = 0;
            for (int jj = fc; jj < B && jb + jj < W; jj += n.d, ++m) {
                const int lj = jb + jj - c0;
                const int2 qv = ps.qc[li + 1][lj + 1];
                const int2 p = ps.psl[li][lj];
                int d;
                uint16_t* dst = &ps.smp[1][row_slot + 2 * m];
                dst[0] = (uint16_t)quantize_code(qv.x, p.x, code, d);
                dst[1] = (uint16_t)quantize_code(qv.y, p.y, code, d);
            }
        }
        // 3DL micro-encoding: anti-diagonal sweep, lane r at column k - r;
        // jn = the next sampled column of this row, m its slot
        int jn = fc, m = 0;
        int2 res = make_int2(0, 0), up = res, left = res;
        for (int k = 0; k < 2 * B - 1; ++k) {
            const int jj = k - r;
            const int j = jb + jj, lj = j - c0;
            int2 fromprev;
            fromprev.x = __shfl_up_sync(0xffffffffu, res.x, 1);
            fromprev.y = __shfl_up_sync(0xffffffffu, res.y, 1);
            const int2 upleft_in = up;
            if (live && jj >= 0 && jj < B && j < W) {
                const int2 u = r > 0 ? fromprev : ps.qc[li][lj + 1];
                const int2 lft = jj > 0 ? left : ps.qc[li + 1][lj];
                const int2 ul = (r > 0 && jj > 0) ? upleft_in : ps.qc[li][lj];
                const int2 p0 = pp[(li - 1) * kPP + lj - 1], p1 = pp[(li - 1) * kPP + lj];
                const int2 p2 = pp[li * kPP + lj - 1], p3 = pp[li * kPP + lj];
                const int pu = u.x + lft.x + p3.x - ul.x - p1.x - p2.x + p0.x;
                const int pv = u.y + lft.y + p3.y - ul.y - p1.y - p2.y + p0.y;
                const int2 qv = ps.qc[li + 1][lj + 1];
                int2 rec;
                const unsigned su = quantize_code(qv.x, pu, code, rec.x);
                const unsigned sv = quantize_code(qv.y, pv, code, rec.y);
                if (row_s && jj == jn) {
                    uint16_t* dst = &ps.smp[0][row_slot + 2 * m];
                    dst[0] = (uint16_t)su;
                    dst[1] = (uint16_t)sv;
                    jn += n.d;
                    ++m;
                }
                up = u;
                res = rec;
                left = rec;
            } else {
                res = make_int2(0, 0);
                up = make_int2(0, 0);
            }
        }
        __syncwarp();
        const int nbp = min(bpp, nbt - b0);
        for (int b = 0; b < nbp; ++b) {
            const int bb = b0 + b;
            const int ibb = r0 + ((bb >> lgN) << lgB), jbb = c0 + ((bb & (nbu - 1)) << lgB);
            if (ibb >= H || jbb >= W) continue;
            int frb, fcb, nrb, ncb;
            sampled(ibb, jbb, frb, fcb, nrb, ncb);
            const int used = 2 * nrb * ncb;
            const long long r3 = warp_block_score(&ps.smp[0][b * nslots], used, B, ps.hist, a.log2tab);
            const long long rs = warp_block_score(&ps.smp[1][b * nslots], used, B, ps.hist, a.log2tab);
            if (lane == 0) {
                const unsigned char md = (1000 * rs < 997 * r3) ? 1 : 0;
                a.modes[((size_t)t * a.nby + (ibb >> lgB)) * a.nbx + (jbb >> lgB)] = md;
                ps.modes[bb] = md;
                if (md) atomicAdd(a.counters + 2, 1ull);
            }
        }
        __syncwarp();
    }
}

// Decoding: the modes of the unit's blocks from the stream's mode bits.
__device__ void unit_modes_from_bits(const SliceArgs& a, int t, int r0, int c0, unsigned char* modes) {
    const int lgB = __ffs(a.B) - 1, lgN = __ffs(a.U) - 1 - lgB;  // B and U are powers of two
    const int nbu = 1 << lgN;
    for (int bb = (int)(threadIdx.x & 31u); bb < nbu * nbu; bb += 32) {
        const int ib = (r0 >> lgB) + (bb >> lgN), jb = (c0 >> lgB) + (bb & (nbu - 1));
        unsigned char m = 0;
        if (ib < a.nby && jb < a.nbx) {
            const size_t x = ((size_t)t * a.nby + ib) * a.nbx + jb;
            m = (unsigned char)((__ldg(a.mode_bits + (x >> 3)) >> (x & 7)) & 1u);
        }
        modes[bb] = m;
    }
    __syncwarp();
}

// One prep unit: the U x U vertices from (r0, c0) of slice t >= 1 (it enters
// the ready queue once slice t-1 is reconstructed around it).  Leaves in psl
// the SL prediction of every vertex that uses SL, and with MoP the marker
// kNoSL on the vertices of blocks that keep 3DL.
template <class Sm>
__device__ void prep_unit(const SliceArgs& a, int t, int r0, int c0, Sm& sm, const float* w2s) {
    const unsigned FULL = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31u), H = a.H, W = a.W, U = a.U;
    const int uh = min(U, H - r0), uw = min(U, W - c0);
    // unit and block sides are powers of two: the unit's sites as k = li U + lj
    const int lgU = __ffs(U) - 1;
    const int lgB = __ffs(a.B) - 1, lgN = lgU - lgB;  // (MoP) block of site (li, lj): (li >> lgB) << lgN | lj >> lgB
    auto block_of = [&](int li, int lj) { return ((li >> lgB) << lgN) + (lj >> lgB); };
    const FastDiv ns((unsigned)a.n);  // (MoP) sampling stride
    auto& ps = sm.prep;
    constexpr int kPP = std::remove_reference<decltype(ps)>::type::kPitch;
    const size_t sl = (size_t)H * W;
    const int2 z = make_int2(0, 0);
    const bool mop = a.pred == 2;
    const bool dec = a.decode != 0;  // decoding: the block modes come from the stream
    if (mop && !dec) {
        // q(t) with a one-cell halo (asynchronous copies)
        const int2* Qt = a.q + (size_t)t * sl;
        for (int rr = 0; rr < U + 2; ++rr) {
            const int i = r0 - 1 + rr;
            for (int cc = lane; cc < U + 2; cc += 32) {
                const int j = c0 - 1 + cc;
                const bool ok = i >= 0 && i < H && j >= 0 && j < W;
                cp_async8(&ps.qc[rr][cc], Qt + (ok ? (size_t)i * W + j : 0), ok);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // slice t-1 around the unit, widened by the reach when it fits the window
    // (reconstruction words, several rows in flight)
    const bool staged = U + 2 + 2 * a.R <= kPP;
    const int Rw = staged ? a.R : 0;
    const int span = U + 2 + 2 * Rw;
    const int2* P = a.qhat + (size_t)(t - 1) * sl;
    // asynchronous copies of the reconstruction words (an L1 line read before
    // a word was written holds zero, which reads as "not ready"), then every
    // word not ready yet is awaited through L2 and the tags are removed
    for (int rr = 0; rr < span; ++rr) {
        const int i = r0 - 1 - Rw + rr;
        for (int cc = lane; cc < span; cc += 32) {
            const int j = c0 - 1 - Rw + cc;
            const bool ok = i >= 0 && i < H && j >= 0 && j < W;
            cp_async8(&ps.pp[rr * kPP + cc], P + (ok ? (size_t)i * W + j : 0), ok);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    cp_async_wait_all();
    __syncwarp();
    // (row rr, column cc) of word k = lane + 32 m, advanced without a division
    int rr = 0, cc = lane;
    while (cc >= span) { cc -= span; ++rr; }
    for (int k = lane; k < span * span; k += 32, cc += 32) {
        while (cc >= span) { cc -= span; ++rr; }
        const int i = r0 - 1 - Rw + rr, j = c0 - 1 - Rw + cc;
        if (i < 0 || i >= H || j < 0 || j >= W) continue;  // zero-filled
        int2& e = ps.pp[rr * kPP + cc];
        unsigned long long wv = (unsigned long long)(unsigned)e.x | ((unsigned long long)(unsigned)e.y << 32);
        if (!word_ready(wv)) {
            const int2* p = P + (size_t)i * W + j;
            const unsigned long long t0 = global_ns();
            do {
                if ((long long)(global_ns() - t0) > a.timeout_ns || *(volatile int*)a.status != 0) {
                    atomicCAS(a.status, 0, kStatusTimeout);
                    break;
                }
                wv = ld_word(p);
            } while (!word_ready(wv));
        }
        e = word_value(wv);
    }
    if (__any_sync(FULL, *(volatile int*)a.status != 0)) return;
    const SmemSlice Ps{ps.pp, r0 - 1 - Rw, c0 - 1 - Rw, kPP};
    const TaggedSlice Pg{P, W, a.status, a.timeout_ns};
    int2* Psl = a.psl + (size_t)t * sl;
    if constexpr (Sm::kNet) {
        if (a.pred == 3 || a.pred == 4) {
            // learned predictor: the unit's 8 x 8 tiles from the staged window
            // (reach 3), the second layer's weights from the CTA's shared copy
            NetDev nd = a.net;
            nd.w2t = w2s;
            nd.b2 = w2s + kNetW2;
            auto prev = [&](int i, int j) -> int2 { return Ps.at(i, j); };
            for (int tr = 0; tr < uh; tr += 8)
                for (int tc = 0; tc < uw; tc += 8) {
                    // the learned predictor alone: the final (tagged) word; the
                    // mixture: a plain value, tagged once the block's mode is known
                    auto out = [&](int li, int lj, int2 p) {
                        int2* d = Psl + (size_t)(r0 + tr + li) * W + c0 + tc + lj;
                        if (a.pred == 3) st_word(d, p);
                        else *d = p;
                    };
                    net_tile<8>(nd, ps.net, r0 + tr, c0 + tc, H, W, prev, out);
                }
            if (a.pred == 4 && dec) {
                unit_modes_from_bits(a, t, r0, c0, ps.modes);
            } else if (a.pred == 4) {
                // the learned mixture: block modes as MoP's with the net in SL's
                // place; the scratch of the net gives way to q(t) and the samples
                __threadfence();  // the predictions are read back through L2 by other lanes
                __syncwarp();
                const int2* Qt = a.q + (size_t)t * sl;
                for (int rr = 0; rr < U + 2; ++rr) {
                    const int i = r0 - 1 + rr;
                    for (int cc = lane; cc < U + 2; cc += 32) {
                        const int j = c0 - 1 + cc;
                        const bool ok = i >= 0 && i < H && j >= 0 && j < W;
                        cp_async8(&ps.qc[rr][cc], Qt + (ok ? (size_t)i * W + j : 0), ok);
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                for (int k = lane; k < U * U; k += 32) {
                    const int li = k >> lgU, lj = k & (U - 1);
                    if (li < uh && lj < uw && ns.mod(r0 + li) == 0 && ns.mod(c0 + lj) == 0)
                        ps.psl[li][lj] = __ldcg(Psl + (size_t)(r0 + li) * W + c0 + lj);
                }
                cp_async_wait_all();
                __syncwarp();
                mop_unit(a, t, r0, c0, ps, Rw);
            }
            if (a.pred == 4) {
                // the mixture's final words: the net's prediction in the blocks
                // that chose it, the 3DL marker in the others
                __threadfence();  // the plain values are read back through L2 by other lanes
                __syncwarp();
                for (int k = lane; k < U * U; k += 32) {
                    const int li = k >> lgU, lj = k & (U - 1);
                    if (li >= uh || lj >= uw) continue;
                    int2* d = Psl + (size_t)(r0 + li) * W + c0 + lj;
                    st_word(d, ps.modes[block_of(li, lj)] ? __ldcg(d) : make_int2(kNoSL, 0));
                }
            }
            return;
        }
    }
    unsigned sub = 0, steps = 0;
    // semi-Lagrangian predictions, lanes over a compact list of sites: every
    // vertex (pure SL) or the sampled sites (MoP encoding, for the decisions)
    auto predict_site = [&](int li, int lj) {
        const int i = r0 + li, j = c0 + lj;
        int pu, pv;
        const int md = staged ? sl_predict(Ps, H, W, i, j, a.cfl_x, a.cfl_y, pu, pv)
                              : sl_predict(Pg, H, W, i, j, a.cfl_x, a.cfl_y, pu, pv);
        const int2 p = make_int2(pu, pv);
        // MoP keeps a sampled prediction until its block's mode is known
        if (mop) ps.psl[li][lj] = p;
        else st_word(Psl + (size_t)i * W + j, p);
        sub += md > 0;
        steps += md;
    };
    if (!mop) {
        for (int k = lane; k < U * U; k += 32) {
            const int li = k >> lgU, lj = k & (U - 1);
            if (li < uh && lj < uw) predict_site(li, lj);
        }
    } else if (!dec) {
        // sampled sites: rows fr, fr + n, ..., columns fc, fc + n, ...
        const unsigned n = ns.d;
        const int fr = (int)ns.mod(n - ns.mod(r0)), fc = (int)ns.mod(n - ns.mod(c0));
        const int nr = uh > fr ? (int)ns.div(uh - fr + n - 1) : 0;
        const int nc = uw > fc ? (int)ns.div(uw - fc + n - 1) : 0;
        const FastDiv ncd((unsigned)max(nc, 1));
        for (int k = lane; k < nr * nc; k += 32) {
            const int q = (int)ncd.div(k);
            predict_site(fr + q * (int)n, fc + (k - q * nc) * (int)n);
        }
    }
    __syncwarp();
    if (mop) {
        if (dec) unit_modes_from_bits(a, t, r0, c0, ps.modes);
        else mop_unit(a, t, r0, c0, ps, Rw);
        // the other vertices of the blocks that chose SL (decoding: all of
        // them), gathered into a list
        int cnt = 0;
        for (int base = 0; base < U * U; base += 32) {
            const int k = base + lane;
            const int li = k >> lgU, lj = k & (U - 1);
            const bool in = li < uh && lj < uw;
            const bool mode_sl = in && ps.modes[block_of(li, lj)] != 0;
            const bool sampled = !dec && ns.mod(r0 + li) == 0 && ns.mod(c0 + lj) == 0;
            const bool need = mode_sl && !sampled;
            const unsigned bal = __ballot_sync(FULL, need);
            if (need) ps.list[cnt + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)(li * 32 + lj);
            cnt += __popc(bal);
            // the sampled predictions of the blocks that chose SL, and the
            // marker instead of a prediction in the blocks that kept 3DL
            if (mode_sl && sampled) st_word(Psl + (size_t)(r0 + li) * W + c0 + lj, ps.psl[li][lj]);
            if (in && !mode_sl) st_word(Psl + (size_t)(r0 + li) * W + c0 + lj, make_int2(kNoSL, 0));
        }
        __syncwarp();
        for (int m = lane; m < cnt; m += 32) {
            const unsigned v = ps.list[m];
            const int i = r0 + (int)(v >> 5), j = c0 + (int)(v & 31u);
            int pu, pv;
            const int md = staged ? sl_predict(Ps, H, W, i, j, a.cfl_x, a.cfl_y, pu, pv)
                                  : sl_predict(Pg, H, W, i, j, a.cfl_x, a.cfl_y, pu, pv);
            st_word(Psl + (size_t)i * W + j, make_int2(pu, pv));
            sub += md > 0;
            steps += md;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sub += __shfl_xor_sync(FULL, sub, o);
        steps += __shfl_xor_sync(FULL, steps, o);
    }
    if (lane == 0 && sub) {
        atomicAdd(a.counters + 0, (unsigned long long)sub);
        atomicAdd(a.counters + 1, (unsigned long long)steps);
    }
}

// Units of slice t (t >= 1) that became ready while wave(t-1, s) went from
// step k0 to step k1 (after step k, lane l has finished columns <= k - l).
// Unit (ur, uc) needs slice t-1 up to row r = min(H-1, ur*U + U - 1 + R) and
// column c = min(W-1, uc*U + U - 1 + R); rows above r are further ahead.  It
// is queued by the wave of the strip holding row r, at the step c + (r mod 32)
// that finishes (r, c): every unit exactly once.  The queue orders the work
// only: a unit still awaits each reconstruction word it reads.
__device__ void enqueue_units(const SliceArgs& a, int t, int s, int k0, int k1) {
    const int U = a.U, R = a.R, W = a.W, H = a.H, lane = (int)(threadIdx.x & 31u);
    const int nstrips = (H + 31) / 32;
    const int lgU = __ffs(U) - 1;  // unit sides are powers of two
    auto ready_cols = [&](int x) -> int {  // unit columns whose column need is <= x
        if (x >= W - 1) return a.nuc;
        const int v = x - U + 1 - R;
        return v < 0 ? 0 : min(a.nuc, (v >> lgU) + 1);
    };
    auto first_row = [&](int sx) -> int {  // first unit row whose row need is in strip sx or below
        const int num = 32 * sx - U + 1 - R;
        return num <= 0 ? 0 : min(a.nur, (num + U - 1) >> lgU);
    };
    const int ur0 = first_row(s), ur1 = s + 1 < nstrips ? first_row(s + 1) : a.nur;
    auto need_lane = [&](int ur) { return min(H - 1, ur * U + U - 1 + R) - 32 * s; };
    unsigned cnt = 0;
    for (int ur = ur0; ur < ur1; ++ur) {
        const int l = need_lane(ur);
        cnt += (unsigned)max(0, ready_cols(k1 - l) - ready_cols(k0 - l));
    }
    if (cnt == 0) return;
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(a.qtail, cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int ur = ur0; ur < ur1; ++ur) {
        const int l = need_lane(ur);
        const int lo = ready_cols(k0 - l), n = max(0, ready_cols(k1 - l) - lo);
        for (int m = lane; m < n; m += 32) {
            const unsigned id =
                ((unsigned)(t - 1) * (unsigned)a.nur + (unsigned)ur) * (unsigned)a.nuc + (unsigned)(lo + m);
            if (base + m < a.queue_len) st_relaxed(a.qslot + base + m, a.unit_base + id + 1u);
            else atomicCAS(a.status, 0, kStatusCorrupt);  // cannot happen: every unit is queued once
        }
        base += (unsigned)n;
    }
}

// A prep warp: takes queue positions in order and works each unit once its
// slot is filled.  A slot holds the unit's global id + 1; its field is the
// last one whose first unit id does not exceed it.  kBatch: the field's
// arguments are copied into the warp's shared slot; otherwise the launch has
// one field, read from parameter space.
template <bool kBatch, class Sm>
__device__ void prep_loop(const PipeArgs& p, Sm& sm, const float* w2s) {
    for (;;) {
        unsigned pos = 0;
        int stop = 0;
        if ((threadIdx.x & 31u) == 0) {
            pos = atomicAdd(p.qhead, 1u);
            stop = *(volatile int*)p.status != 0;
        }
        pos = __shfl_sync(0xffffffffu, pos, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (pos >= p.queue_len || stop) return;
        const unsigned v = warp_wait_geq(p.status, p.timeout_ns, p.one.qslot + pos, 1u);
        if (!v) return;
        const unsigned gid = v - 1u;
        int lo = 0;
        if (kBatch) {
            int hi = p.nfields - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(&p.fields[mid].unit_base) <= gid) lo = mid;
                else hi = mid - 1;
            }
        }
        const SliceArgs& a = kBatch ? load_field(p.fields, lo, sm) : p.one;
        const unsigned id = gid - a.unit_base;
        const int uc = (int)(id % (unsigned)a.nuc);
        const unsigned rest = id / (unsigned)a.nuc;
        const int ur = (int)(rest % (unsigned)a.nur);
        const int t = (int)(rest / (unsigned)a.nur) + 1;
        prep_unit(a, t, ur * a.U, uc * a.U, sm, w2s);
    }
}

// ---------------------------------------------------------------------------
// wave(t, s)
// ---------------------------------------------------------------------------
// Stages chunk g of a wave's inputs (steps kChunk g ..) into slot g % 3:
// contiguous 16-byte copies of the strip-diagonal arrays, zero past the
// strip's last step.  Dn, Db and Dnb must be readable pointers even when their
// data does not exist (has_next, below_ok false): the copies then read nothing.
__device__ __forceinline__ void stage_chunk(WaveRing& r, int g, const int2* cls, const unsigned* cm, const int2* Dq,
                                            const int2* Dn, const int2* Db, const int2* Dnb, bool has_next,
                                            bool below_ok, bool with_cm, int W) {
    const int lane = (int)(threadIdx.x & 31u), slot = g % 3, k0 = g * kChunk, nsteps = W + 31;
    for (int p = lane; p < kChunk * 16; p += 32) {  // 8-byte elements: 16 pieces per step
        const int st = p >> 4, e = (p & 15) * 2, k = k0 + st;
        const bool ok = k < nsteps;
        const size_t off = ok ? (size_t)k * 32 + e : 0;
        cp_async16(&r.cl[slot][st][e], cls + off, ok);
        cp_async16(&r.q[slot][st][e], Dq + off, ok);
        cp_async16(&r.qn[slot][st][e], Dn + off, ok && has_next);
    }
    for (int p = lane; with_cm && p < kChunk * 8; p += 32) {  // 4-byte elements: 8 pieces per step
        const int st = p >> 3, e = (p & 7) * 4, k = k0 + st;
        const bool ok = k < nsteps;
        cp_async16(&r.cm[slot][st][e], cm + (ok ? (size_t)k * 32 + e : 0), ok);
    }
    if (lane < kChunk) {  // lane 31 of consumer step k reads column k - 31 of the next strip's first row
        const int jj = k0 + lane - 31;
        const bool ok = below_ok && jj >= 0 && jj < W;
        const size_t off = ok ? (size_t)jj * 32 : 0;
        cp_async8(&r.qb[slot][lane], Db + off, ok);
        cp_async8(&r.nb[slot][lane], Dnb + off, ok && has_next);
    }
}

// wave(t, s).  Lane l owns row i = 32s + l and at step k handles column
// j = k - l.  Its neighbours (indices of the 14-vertex neighbourhood):
//   0..3   slice t-1 at (i-1, j-1), (i-1, j), (i, j-1), (i, j): own words read
//          one step ahead, kept for two more steps, the row above from lane
//          l-1 by shuffle (lane 0 reads row i-1 itself)
//   4..6   (i-1, j-1), (i-1, j), (i, j-1) of slice t: registers and shuffles,
//          lane 0 reads row i-1 (written by wave(t, s-1)) one step ahead
//   7..12  original values of slices t and t+1 from the staged ring: (i, j+1)
//          is this lane's element of step k + 1, (i+1, j) and (i+1, j+1) lane
//          l+1's of steps k + 1 and k + 2 (lane 31: the next strip's first row).
// The classification of (i, j) comes from the ring as well.
// All 24 uncertain faces are evaluated here with the actual reconstructions.
template <class Sm>
__device__ bool wave_item(const SliceArgs& a, int t, int s, Sm& sm) {
    const unsigned FULL = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31u), H = a.H, W = a.W, T = a.T;
    const int i0 = 32 * s, i = i0 + lane;
    const bool rowok = i < H, below_ok = i0 + 32 < H;
    const size_t sl = (size_t)H * W, base = (size_t)t * sl;
    // strip-diagonal inputs of this wave and of the same strip of slice t+1
    const int nstrips = (H + 31) >> 5;
    const size_t dstride = (size_t)(W + 31) * 32;  // one strip
    const size_t db = ((size_t)t * nstrips + s) * dstride;
    const int2* cls = a.cls + db;
    const unsigned* cm = a.cls_m + db;
    const int2* Dq = a.qd + db;
    const int2* Dn = t + 1 < T ? a.qd + db + (size_t)nstrips * dstride : Dq;  // slice t+1
    const int2* Db = below_ok ? Dq + dstride : Dq;   // the next strip's first row (lane 0)
    const int2* Dnb = below_ok ? Dn + dstride : Dq;
    const int2* Pm = a.qhat + (t >= 1 ? base - sl : base);  // slice t-1
    int2* Pc = a.qhat + base;                                // slice t
    const int2* Psl = a.psl + base;
    const bool has_prev = t >= 1, has_above = s > 0;
    const bool need_sl = has_prev && a.n_units > 0;  // SL predictions present for this slice
    const bool mop = a.pred == 2 || a.pred == 4;  // psl carries the 3DL marker
    const bool feeds = a.n_units > 0 && t + 1 < a.t_end;  // queues the prep units of slice t+1
    const bool has_next = t + 1 < T;
    const bool dec = a.decode != 0;  // decoding: reconstruct from the stream's symbols
    const bool stage_next = has_next && !dec, stage_below = below_ok && !dec;
    const int2 z = make_int2(0, 0);
    int published = -1;  // last step whose ready units were queued
    // outputs (a refers to the warp's shared slot: keep the pointers in registers)
    int2* const out_qhat = a.qhat;
    uint8_t* const out_qxi = a.qxi;
    uint32_t* const out_sym = a.sym;
    int* const out_xi = a.xi_out;

    // loads for a step, issued two steps ahead (two alternating register sets)
    struct Pf {
        unsigned long long wp, wa, wu;  // slice t-1 at (i, j); lane 0: slice t-1 and t at (i-1, j)
        unsigned long long wn;          // SL prediction word at (i, j) (tagged like a reconstruction)
    };
    auto issue = [&](int kk, Pf& f) {
        const int jj = kk - lane;
        const bool col = jj >= 0 && jj < W;
        f.wp = 0;
        f.wa = 0;
        f.wu = 0;
        if (has_prev && rowok && col) f.wp = ld_word(Pm + (size_t)i * W + jj);
        if (lane == 0 && has_above && col) {
            if (has_prev) f.wa = ld_word(Pm + (size_t)(i0 - 1) * W + jj);
            f.wu = ld_word(Pc + (size_t)(i0 - 1) * W + jj);
        }
        f.wn = 0;
        if (need_sl && rowok && col) f.wn = ld_word(Psl + (size_t)i * W + jj);
    };
    WaveRing& ring = sm.ring;
    __syncwarp();
    stage_chunk(ring, 0, cls, cm, Dq, Dn, Db, Dnb, stage_next, stage_below, !dec, W);
    asm volatile("cp.async.commit_group;" ::: "memory");
    stage_chunk(ring, 1, cls, cm, Dq, Dn, Db, Dnb, stage_next, stage_below, !dec, W);
    asm volatile("cp.async.commit_group;" ::: "memory");
    Pf fa, fb;
    issue(0, fa);
    issue(1, fb);

    int2 h0 = z, h1 = z, h2 = z;  // slice t-1 at (i, j), (i, j-1), (i, j-2)
    int2 a0 = z, a1 = z;          // lane 0: slice t-1 at (i-1, j), (i-1, j-1)
    int2 left = z, up = z, res = z;
    auto step = [&](int k, Pf& f) -> bool {
        const int j = k - lane;
        const bool col = j >= 0 && j < W;
        // this step's words (issued two steps ago) and the SL prediction,
        // once its unit has written it: one vote when all are present
        const bool np = has_prev && rowok && col, na = lane == 0 && has_above && has_prev && col;
        const bool nu = lane == 0 && has_above && col, nn = need_sl && rowok && col;
        const bool present = (!np || word_ready(f.wp)) && (!na || word_ready(f.wa)) && (!nu || word_ready(f.wu)) &&
                             (!nn || word_ready(f.wn));
        if (!__all_sync(FULL, present)) {
            if (!poll_word(a, Pm + (size_t)(rowok ? i : 0) * W + (col ? j : 0), np, f.wp)) return false;
            if (!poll_word(a, Pm + (size_t)(i0 > 0 ? i0 - 1 : 0) * W + (col ? j : 0), na, f.wa)) return false;
            if (!poll_word(a, Pc + (size_t)(i0 > 0 ? i0 - 1 : 0) * W + (col ? j : 0), nu, f.wu)) return false;
            if (!poll_word(a, Psl + (size_t)(rowok ? i : 0) * W + (col ? j : 0), nn, f.wn)) return false;
        }
        const int2 pk = (has_prev && rowok && col) ? word_value(f.wp) : z;
        const int2 ak = (lane == 0 && has_above && has_prev && col) ? word_value(f.wa) : z;
        const int2 uk = (lane == 0 && has_above && col) ? word_value(f.wu) : z;
        const int2 pslk = (need_sl && rowok && col) ? word_value(f.wn) : z;
        // chunk g of the staged inputs starts: stage g + 2 over the slot of
        // g - 1 (no longer read), then wait for g and g + 1
        if (k % kChunk == 0) {
            __syncwarp();
            stage_chunk(ring, k / kChunk + 2, cls, cm, Dq, Dn, Db, Dnb, stage_next, stage_below, !dec, W);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncwarp();
        }
        issue(k + 2, f);
        // neighbours 0..3
        h2 = h1;
        h1 = h0;
        h0 = pk;
        a1 = a0;
        a0 = ak;
        int2 n0, n1;
        n1.x = __shfl_up_sync(FULL, h1.x, 1);
        n1.y = __shfl_up_sync(FULL, h1.y, 1);
        n0.x = __shfl_up_sync(FULL, h2.x, 1);
        n0.y = __shfl_up_sync(FULL, h2.y, 1);
        if (lane == 0) {
            n1 = a0;
            n0 = a1;
        }
        const int2 n2 = h1, n3 = h0;
        // neighbours 4..6
        int2 fromprev;
        fromprev.x = __shfl_up_sync(FULL, res.x, 1);
        fromprev.y = __shfl_up_sync(FULL, res.y, 1);
        const int2 upleft = up;
        up = lane == 0 ? uk : fromprev;
        if (rowok && col && dec) {
            // decoding: qhat = prediction + code * width per component with a
            // symbol, else the verbatim value
            const int s0 = (k / kChunk) % 3, r0 = k % kChunk;
            const int2 cs = ring.cl[s0][r0][lane];
            const int code = cs.x;
            const unsigned sy = (unsigned)cs.y;
            int2 rec = ring.q[s0][r0][lane];
            if (code > 0) {
                int pu, pv;
                if (need_sl && (!mop || pslk.x != kNoSL)) {
                    pu = pslk.x;
                    pv = pslk.y;
                } else {
                    pu = up.x + left.x + n3.x - upleft.x - n1.x - n2.x + n0.x;
                    pv = up.y + left.y + n3.y - upleft.y - n1.y - n2.y + n0.y;
                }
                const unsigned w = (2u << (code - 1)) + 1u;
                const unsigned su = sy & 0xFFFFu, sv = sy >> 16;
                if (su) rec.x = (int)((unsigned)pu + (su - (unsigned)kRadius) * w);
                if (sv) rec.y = (int)((unsigned)pv + (sv - (unsigned)kRadius) * w);
            }
            st_word(out_qhat + base + (size_t)i * W + j, rec);
            res = rec;
        } else if (rowok && col) {
            const int s0 = (k / kChunk) % 3, r0 = k % kChunk;
            const int s1 = ((k + 1) / kChunk) % 3, r1 = (k + 1) % kChunk;
            const int2 cl = ring.cl[s0][r0][lane];
            const unsigned mf = (unsigned)cl.y, mm = ring.cm[s0][r0][lane];
            int xi = cl.x;
            const int2 qv = ring.q[s0][r0][lane];
            if (xi > 0 && (mf | mm)) {
                const int s2 = ((k + 2) / kChunk) % 3, r2 = (k + 2) % kChunk;
                const int2 n7 = ring.q[s1][r1][lane];
                const int2 n8 = lane < 31 ? ring.q[s1][r1][lane + 1] : ring.qb[s0][r0];
                const int2 n9 = lane < 31 ? ring.q[s2][r2][lane + 1] : ring.qb[s1][r1];
                const int2 n10 = ring.qn[s0][r0][lane], n11 = ring.qn[s1][r1][lane];
                const int2 n12 = lane < 31 ? ring.qn[s1][r1][lane + 1] : ring.nb[s0][r0];
                const int2 n4 = upleft, n5 = up, n6 = left;  // (the uncertain faces do not use neighbour 13)
                // M = 0 checks of the 24 faces, branch free: with d = n - q(v),
                // M = d_a.x d_b.y - d_a.y d_b.x
#define CPT_D(k) const int dx##k = n##k.x - qv.x, dy##k = n##k.y - qv.y;
                CPT_D(0) CPT_D(1) CPT_D(2) CPT_D(3) CPT_D(4) CPT_D(5) CPT_D(6)
                CPT_D(7) CPT_D(8) CPT_D(9) CPT_D(10) CPT_D(11) CPT_D(12)
#undef CPT_D
                // The low 32 bits of the two products agree whenever M = 0:
                // that filter runs on 32-bit multiplies, and the rare faces
                // that pass it are confirmed with the exact 64-bit products.
                // When mm holds all 24 faces (interior vertices) the filter
                // is first folded into one predicate, and the face mask is
                // built only if some face passes it.
                bool any = true;
                if (mm == kAllUncFaces) {
                    bool z = false;
#define CPT_PZ(fa, fb) z = z | ((unsigned)dx##fa * (unsigned)dy##fb == (unsigned)dy##fa * (unsigned)dx##fb);
                    CPT_UNC_FACES(CPT_PZ)
#undef CPT_PZ
                    any = z;
                }
                unsigned hits = 0;
                int bit = 0;
                if (any) {
#define CPT_PM(fa, fb)                                                                            \
    hits |= ((unsigned)dx##fa * (unsigned)dy##fb == (unsigned)dy##fa * (unsigned)dx##fb ? 1u : 0u) << bit; \
    ++bit;
                    CPT_UNC_FACES(CPT_PM)
#undef CPT_PM
                    hits &= mm;
                }
                if (hits) {
                    unsigned exact = 0;
                    bit = 0;
#define CPT_PM64(fa, fb)                                                                  \
    exact |= ((long long)dx##fa * dy##fb == (long long)dy##fa * dx##fb ? 1u : 0u) << bit; \
    ++bit;
                    CPT_UNC_FACES(CPT_PM64)
#undef CPT_PM64
                    if (exact & hits) xi = 0;
                }
                if (xi > 0 && mf) {
                    int2* nb = sm.nbs[lane];
                    nb[0] = n0; nb[1] = n1; nb[2] = n2; nb[3] = n3;
                    nb[4] = n4; nb[5] = n5; nb[6] = n6;
                    nb[7] = n7; nb[8] = n8; nb[9] = n9;
                    nb[10] = n10; nb[11] = n11; nb[12] = n12;
                    for (unsigned m = mf; m && xi > 0; m &= m - 1) {
                        const unsigned pr = unc_pair(__ffs(m) - 1);
                        const int2 p0 = nb[pr & 15u], p1 = nb[pr >> 4];
                        xi = min_alg2(xi, p0.x, p0.y, p1.x, p1.y, qv.x, qv.y);
                    }
                }
            }
            const int code = xi_code(xi);
            int2 rec = qv;
            unsigned sym = 0;
            if (code > 0) {
                int pu, pv;
                if (need_sl && (!mop || pslk.x != kNoSL)) {
                    pu = pslk.x;
                    pv = pslk.y;
                } else {
                    pu = up.x + left.x + n3.x - upleft.x - n1.x - n2.x + n0.x;
                    pv = up.y + left.y + n3.y - upleft.y - n1.y - n2.y + n0.y;
                }
                const unsigned su = quantize_code(qv.x, pu, code, rec.x);
                const unsigned sv = quantize_code(qv.y, pv, code, rec.y);
                sym = su | (sv << 16);
            }
            const size_t v = base + (size_t)i * W + j;
            st_word(out_qhat + v, rec);
            out_qxi[v] = (uint8_t)code;
            out_sym[v] = sym;
            if (out_xi) out_xi[v] = xi;
            res = rec;
        } else {
            res = z;
        }
        left = res;
        // the last lane finished column k - 31: queue the units of slice t+1
        // that this makes ready
        if (feeds && ((k + 1) % kPublishEvery == 0 || k == W + 30)) {
            enqueue_units(a, t + 1, s, published, k);
            published = k;
        }
        return true;
    };
    for (int k = 0; k < W + 31; k += 2) {
        if (!step(k, fa) || (k + 1 < W + 31 && !step(k + 1, fb))) {
            cp_async_wait_all();
            return false;
        }
    }
    cp_async_wait_all();  // no copy into the ring outlives the item
    return true;
}

// Every warp is an independent worker with its own shared-memory slot; one
// CTA per SM holds as many of them as the slots and the registers allow.
// Two layouts: (0) every slot has the size of the larger role's and the first
// prep_warps warps of the grid work the prep queue, so whole SMs run the
// waves undisturbed; (1) the first prep_per_cta warps of every CTA work the
// prep queue with prep-sized slots, the others the waves with wave-sized
// slots (more warps fit, but the waves share every SM).
constexpr int kMaxWarpsPerCta = 12;  // 168 registers x 32 lanes x 12 <= 64 K registers
template <bool kBatch, int UMAX, bool NET>
__global__ void __maxnreg__(168) encode_pipeline_kernel(const __grid_constant__ PipeArgs p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int wid = (int)(threadIdx.x >> 5), wpc = (int)(blockDim.x >> 5);
    const bool mixed = p.mixed != 0;
    const int np = UMAX > 0 && mixed ? p.prep_per_cta : 0;
    constexpr size_t kPrepBytes = prep_slot_bytes<UMAX, NET>();
    // the learned net's second-layer weights and biases, one copy per CTA
    // after the warps' slots (every field of a launch shares the model)
    float* w2s = reinterpret_cast<float*>(
        smem_raw + (mixed ? kPrepBytes * np + sizeof(WaveSlot) * (wpc - np) : (size_t)p.slot_bytes * wpc));
    if constexpr (NET) {
        if (p.one.pred == 3 || p.one.pred == 4) {
            for (int k = (int)threadIdx.x; k < kNetW2 + kNetC; k += (int)blockDim.x)
                w2s[k] = k < kNetW2 ? __ldg(p.one.net.w2t + k) : __ldg(p.one.net.b2 + (k - kNetW2));
        }
        __syncthreads();
    }
    unsigned char* const slot =
        mixed ? (wid < np ? smem_raw + kPrepBytes * wid : smem_raw + kPrepBytes * np + sizeof(WaveSlot) * (wid - np))
              : smem_raw + (size_t)p.slot_bytes * wid;
    if constexpr (UMAX > 0) {
        if (mixed ? wid < np : (int)blockIdx.x * wpc + wid < p.prep_warps) {
            prep_loop<kBatch>(p, *reinterpret_cast<PrepSlot<UMAX, NET>*>(slot), w2s);
            return;
        }
    }
    if (!mixed && p.wave_cap > 0) {  // layout 0: only the first wave_cap wave warps of a CTA work
        const int first_wave = min(wpc, max(0, p.prep_warps - (int)blockIdx.x * wpc));
        if (wid - first_wave >= p.wave_cap) return;
    }
    WaveSlot& sm = *reinterpret_cast<WaveSlot*>(slot);
    int cur = -1;  // field whose arguments sit in the warp's slot
    for (;;) {
        unsigned item = 0;
        int stop = 0;
        if ((threadIdx.x & 31u) == 0) {
            item = atomicAdd(p.ticket, 1u);
            stop = *(volatile int*)p.status != 0;
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (item >= p.total_items || stop) return;
        if (item == p.skip_item) continue;  // failure injection: this wave never runs
        const int4 fts = __ldg(p.order + item);
        if (kBatch) {
            if (fts.x != cur) {
                load_field(p.fields, fts.x, sm);
                cur = fts.x;
            }
            if (!wave_item(sm.args, fts.y, fts.z, sm)) return;
        } else {
            if (!wave_item(p.one, fts.y, fts.z, sm)) return;
        }
    }
}

#undef CPT_FACE
#undef CPT_UNC_MARK

__global__ void __launch_bounds__(256) log2_table_kernel(unsigned long long* __restrict__ tab, int n) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        tab[x] = x >= 1 ? log2_q32((unsigned)x) : 0ull;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_log2_table(unsigned long long* tab, int n, cudaStream_t s) {
    log2_table_kernel<<<(n + 255) / 256, 256, 0, s>>>(tab, n);
}

// The padding of classify_kernel's strip-diagonal outputs: entries (strip,
// step s, lane l) with no vertex, i.e. s < l or s - l >= W (the first and last
// 31 steps of a strip), and every step of the lanes past H in a last, partial
// strip.  classify_kernel writes every other entry of slices [0, T), so this
// replaces zeroing the whole arrays.  One thread per entry of those steps.
__global__ void __launch_bounds__(256) diag_pad_kernel(int2* __restrict__ cls, unsigned* __restrict__ cls_m,
                                                       int2* __restrict__ qd, int H, int W, int T) {
    const int nstrips = (H + 31) >> 5;
    const int S = W + 31;  // steps per strip
    const int rows_last = H - ((nstrips - 1) << 5);
    const long long n_edge = (long long)T * nstrips * 62 * 32;
    const long long n_mid = rows_last < 32 && W > 31 ? (long long)T * (W - 31) * 32 : 0;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < n_edge + n_mid;
         x += (long long)gridDim.x * blockDim.x) {
        const int lane = (int)(x & 31);
        int t, strip, st;
        if (x < n_edge) {
            const long long line = x >> 5;  // (t, strip, edge step)
            const int e = (int)(line % 62);
            const long long ts = line / 62;
            strip = (int)(ts % nstrips);
            t = (int)(ts / nstrips);
            st = e < 31 ? e : W + (e - 31);
        } else {  // the middle steps of the partial strip
            const long long line = (x - n_edge) >> 5;
            st = 31 + (int)(line % (W - 31));
            t = (int)(line / (W - 31));
            strip = nstrips - 1;
        }
        const int i = (strip << 5) + lane, j = st - lane;
        if (i < H && j >= 0 && j < W) continue;  // a vertex's entry
        const size_t dv = (((size_t)t * nstrips + strip) * (size_t)S + st) * 32 + lane;
        cls[dv] = make_int2(0, 0);
        cls_m[dv] = 0u;
        qd[dv] = make_int2(0, 0);
    }
}

void launch_diag_pad(int2* cls, unsigned* cls_m, int2* qd, int H, int W, int T, cudaStream_t s) {
    const long long n = (long long)T * ((H + 31) / 32) * 62 * 32 + (long long)T * (W > 31 ? W - 31 : 0) * 32;
    const long long blocks = std::min<long long>((n + 255) / 256, 152 * 16);
    diag_pad_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, s>>>(cls, cls_m, qd, H, W, T);
}

void launch_classify(const int32_t* q, const uint16_t* mask, int H, int W, int T, int eps_int, int2* out,
                     unsigned* out_m, int2* qd, cudaStream_t s, int t_first, int t_count) {
    if (t_count < 0) t_count = T - t_first;
    if (t_count <= 0) return;
    dim3 grid((W + 31) / 32, (H + kClsRows - 1) / kClsRows, t_count);
    classify_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const int2*>(q), mask, H, W, T, eps_int, out, out_m, qd,
                                         t_first);
}

template <int UMAX, bool NET>
static cudaError_t launch_pipeline_t(const PipeArgs& p, int pred, int nsm, const PipeTuning& tune, cudaStream_t s) {
    const size_t pslot = prep_slot_bytes<UMAX, NET>(), wslot = sizeof(WaveSlot);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const size_t wshared = NET ? sizeof(float) * (kNetW2 + kNetC) : 0;  // the net's shared weights
    // with SL, MoP or the learned predictor a share of the warps works the
    // prep queue; the most warps whose slots fit the shared memory
    const bool prep = UMAX > 0 && p.queue_len > 0;
    const bool mixed = prep && tune.mixed == 1;
    const int share = tune.prep_share > 0 ? tune.prep_share
                                          : (NET ? kPrepShareNet : (pred == 1 ? kPrepShareSL : kPrepShareMoP));
    const size_t uslot = std::max(pslot, wslot);  // layout 0: one slot size
    int wmax = kMaxWarpsPerCta;
    if (tune.warps_per_sm > 0) wmax = std::min(wmax, tune.warps_per_sm);
    int wpc = 0, np = 0;
    for (int w = wmax; w >= (mixed ? 2 : 1) && !wpc; --w) {
        const int n = mixed ? std::max(1, std::min(w - 1, (int)((w * share + 50) / 100))) : 0;
        const size_t need = mixed ? pslot * n + wslot * (w - n) : uslot * w;
        if (need + wshared <= (size_t)optin) {
            wpc = w;
            np = n;
        }
    }
    if (wpc < 1) return cudaErrorInvalidConfiguration;
    const bool batch = p.nfields > 1;
    auto kern = batch ? encode_pipeline_kernel<true, UMAX, NET> : encode_pipeline_kernel<false, UMAX, NET>;
    const size_t smem = (mixed ? pslot * np + wslot * (wpc - np) : uslot * wpc) + wshared;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpc, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;  // every worker must be resident
    if (tune.warps_per_sm > 0) per_sm = 1;                 // exactly that many warps per SM
    PipeArgs b = p;
    b.mixed = mixed ? 1 : 0;
    b.prep_per_cta = np;
    b.slot_bytes = (unsigned)uslot;
    b.wave_cap = !mixed && tune.mixed >= 2 ? tune.mixed : 0;
    b.prep_warps = 0;
    if (prep && !mixed) {
        const int warps = nsm * per_sm * wpc;
        b.prep_warps = std::max(1, std::min(warps - 1, (int)((long long)warps * share / 100)));
    }
    kern<<<nsm * per_sm, 32 * wpc, smem, s>>>(b);
    return cudaGetLastError();
}

// The shared-memory layout of the predictor: 3DL none; SL and MoP with blocks
// up to 16: units of 16; the learned predictors: units of 16 and the net's
// scratch; MoP blocks of 32: units of 32 (with room for the net).
cudaError_t launch_encode_pipeline(const PipeArgs& p, int pred, int nsm, const PipeTuning& tune, cudaStream_t s) {
    const int B = p.one.B;
    if (pred == 0) return launch_pipeline_t<0, false>(p, pred, nsm, tune, s);
    if (pred == 1 || (pred == 2 && B <= 16)) return launch_pipeline_t<16, false>(p, pred, nsm, tune, s);
    if ((pred == 3 || pred == 4) && B <= 16) return launch_pipeline_t<16, true>(p, pred, nsm, tune, s);
    return launch_pipeline_t<32, true>(p, pred, nsm, tune, s);
}

}  // namespace cpt
