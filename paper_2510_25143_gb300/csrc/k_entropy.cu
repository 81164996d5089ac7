// Entropy stage (Alg. 3 lossless_comp): compaction of the residual symbols
// Q_d and the verbatim values L_d in raster order, symbol histograms for the
// canonical Huffman codebooks, and tiled bit packing of the code words
// (most significant bit first into 32-bit words).
#include "cpt_dev.cuh"
#include "cpt_internal.h"

namespace cpt {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

// ---------------------------------------------------------------------------
// exclusive scan of u64 (three passes: block totals, scan of totals, apply)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long block_exclusive_scan(unsigned long long x,
                                                                   unsigned long long* warp_tot,
                                                                   unsigned long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long v = lane < nw ? warp_tot[lane] : 0ull, vi = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) vi += y;
        }
        if (lane < nw) warp_tot[lane] = vi - v;
        if (lane == nw - 1) *total = vi;
    }
    __syncthreads();
    unsigned long long r = warp_tot[w] + inc - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const unsigned long long* __restrict__ d, size_t n,
                                                                   unsigned long long* __restrict__ sums) {
    __shared__ unsigned long long wt[32], tot;
    size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * kScanItems;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += d[base + k];
    block_exclusive_scan(s, wt, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(unsigned long long* __restrict__ sums, size_t nb) {
    __shared__ unsigned long long wt[32], tot;
    unsigned long long carry = 0;
    for (size_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        size_t k = b0 + threadIdx.x;
        unsigned long long x = k < nb ? sums[k] : 0ull;
        unsigned long long e = block_exclusive_scan(x, wt, &tot);
        if (k < nb) sums[k] = carry + e;
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(unsigned long long* __restrict__ d, size_t n,
                                                                  const unsigned long long* __restrict__ sums) {
    __shared__ unsigned long long wt[32], tot;
    size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * kScanItems;
    unsigned long long v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? d[base + k] : 0ull;
        s += v[k];
    }
    unsigned long long e = block_exclusive_scan(s, wt, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) d[base + k] = e;
        e += v[k];
    }
}

size_t scan_temp_elems(size_t n) { return (n + kScanBlock - 1) / kScanBlock + 1; }

void launch_exclusive_scan_u64(unsigned long long* data, size_t n, unsigned long long* tmp, cudaStream_t s) {
    if (n == 0) return;
    size_t nb = (n + kScanBlock - 1) / kScanBlock;
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, tmp);
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(tmp, nb);
    scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(data, n, tmp);
}

// ---------------------------------------------------------------------------
// compaction of Q_d (2 symbols per vertex with a nonzero bound code) and L_d
// (both values of a lossless vertex, or the value of an unpredictable
// component), counts packed as (n_qd << 32) | n_ld.  Tiles of kCmpTile
// vertices: one pass counts per tile, a scan of the tile counts gives each
// tile's offsets, and the scatter pass recounts its tile with a block scan.
// q is read only for the values that go to L_d.
// ---------------------------------------------------------------------------
constexpr int kCmpThreads = 256;
constexpr int kCmpPer = 16;
constexpr int kCmpTile = kCmpThreads * kCmpPer;  // 4096 vertices

__device__ __forceinline__ unsigned long long vertex_count(unsigned code, uint32_t s) {
    return code ? (2ull << 32) | (unsigned long long)(((s & 0xFFFFu) == 0) + ((s >> 16) == 0)) : 2ull;
}

// the 16 consecutive vertices of a thread: codes and symbols (zero past N)
__device__ __forceinline__ void load16(const uint8_t* __restrict__ qxi, const uint32_t* __restrict__ sym, size_t N,
                                       size_t base, unsigned char c[kCmpPer], uint32_t s[kCmpPer]) {
    if (base + kCmpPer <= N) {
        const uint4 cv = __ldcs(reinterpret_cast<const uint4*>(qxi + base));
        const unsigned cw[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
        for (int k = 0; k < kCmpPer; ++k) c[k] = (unsigned char)(cw[k >> 2] >> (8 * (k & 3)));
#pragma unroll
        for (int k = 0; k < kCmpPer; k += 4) {
            const uint4 sv = __ldcs(reinterpret_cast<const uint4*>(sym + base + k));
            s[k] = sv.x;
            s[k + 1] = sv.y;
            s[k + 2] = sv.z;
            s[k + 3] = sv.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kCmpPer; ++k) {
            const bool ok = base + k < N;
            c[k] = ok ? qxi[base + k] : (unsigned char)0;
            s[k] = ok ? sym[base + k] : 0u;
        }
    }
}

__global__ void __launch_bounds__(kCmpThreads) tile_count_kernel(const uint8_t* __restrict__ qxi,
                                                                 const uint32_t* __restrict__ sym, size_t N,
                                                                 unsigned long long* __restrict__ tile_cnt) {
    __shared__ unsigned long long wt[32], tot;
    const size_t base = (size_t)blockIdx.x * kCmpTile + (size_t)threadIdx.x * kCmpPer;
    unsigned char c[kCmpPer];
    uint32_t sy[kCmpPer];
    load16(qxi, sym, N, base, c, sy);
    unsigned long long n = 0;
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k)
        if (base + k < N) n += vertex_count(c[k], sy[k]);
    block_exclusive_scan(n, wt, &tot);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = tot;
}

// The tile's outputs are contiguous in both arrays: they are gathered in
// shared memory at their offsets within the tile, then copied out by the whole
// block with consecutive addresses (a thread's own 16 vertices would scatter
// narrow stores across the warp).
constexpr size_t kScatterSmem = (size_t)kCmpTile * 2 * sizeof(uint16_t) + (size_t)kCmpTile * 2 * sizeof(int32_t);

__global__ void __launch_bounds__(kCmpThreads) tile_scatter_kernel(const uint8_t* __restrict__ qxi,
                                                                   const uint32_t* __restrict__ sym,
                                                                   const int2* __restrict__ q,
                                                                   const unsigned long long* __restrict__ tile_off,
                                                                   size_t N, uint16_t* __restrict__ qd,
                                                                   int32_t* __restrict__ ld) {
    extern __shared__ __align__(16) unsigned char sm_scatter[];
    uint16_t* sq = reinterpret_cast<uint16_t*>(sm_scatter);                              // 2 per vertex at most
    int32_t* sld = reinterpret_cast<int32_t*>(sm_scatter + (size_t)kCmpTile * 2 * sizeof(uint16_t));
    __shared__ unsigned long long wt[32], tot;
    const size_t base = (size_t)blockIdx.x * kCmpTile + (size_t)threadIdx.x * kCmpPer;
    unsigned char c[kCmpPer];
    uint32_t sy[kCmpPer];
    load16(qxi, sym, N, base, c, sy);
    unsigned long long n = 0;
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k)
        if (base + k < N) n += vertex_count(c[k], sy[k]);
    const unsigned long long o = block_exclusive_scan(n, wt, &tot);  // offsets within the tile
    unsigned pq = (unsigned)(o >> 32), pl = (unsigned)(o & 0xFFFFFFFFull);
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k) {
        const size_t v = base + k;
        if (v >= N) break;
        if (c[k]) {
            const uint16_t su = (uint16_t)(sy[k] & 0xFFFFu), sv = (uint16_t)(sy[k] >> 16);
            sq[pq] = su;
            sq[pq + 1] = sv;
            pq += 2;
            if (su == 0) sld[pl++] = __ldg(q + v).x;
            if (sv == 0) sld[pl++] = __ldg(q + v).y;
        } else {
            const int2 x = __ldg(q + v);
            sld[pl] = x.x;
            sld[pl + 1] = x.y;
            pl += 2;
        }
    }
    __syncthreads();
    const unsigned long long g = tile_off[blockIdx.x];
    const size_t gq = (size_t)(g >> 32), gl = (size_t)(g & 0xFFFFFFFFull);
    const unsigned nq = (unsigned)(tot >> 32), nl = (unsigned)(tot & 0xFFFFFFFFull);
    for (unsigned k = threadIdx.x; k < nq; k += kCmpThreads) qd[gq + k] = sq[k];
    for (unsigned k = threadIdx.x; k < nl; k += kCmpThreads) ld[gl + k] = sld[k];
}

// ---------------------------------------------------------------------------
// histograms: each thread reads 16 bytes at a time and adds runs of equal
// symbols with one shared-memory atomic per run
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) hist_u8_kernel(const uint8_t* __restrict__ x, size_t n,
                                                      unsigned* __restrict__ hist) {
    __shared__ unsigned h[4][64];  // one copy per pair of warps
    for (int k = threadIdx.x; k < 4 * 64; k += blockDim.x) h[k >> 6][k & 63] = 0;
    __syncthreads();
    unsigned* hh = h[(threadIdx.x >> 6) & 3];
    unsigned cur = 0, cnt = 0;
    auto add = [&](unsigned b) {
        if (b == cur) {
            ++cnt;
        } else {
            if (cnt) atomicAdd(&hh[cur & 63], cnt);
            cur = b;
            cnt = 1;
        }
    };
    const size_t n16 = n / 16;
    const uint4* x4 = reinterpret_cast<const uint4*>(x);
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n16; k += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = __ldcs(x4 + k);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 16; ++e) add((w[e >> 2] >> (8 * (e & 3))) & 0xFFu);
    }
    if (blockIdx.x == 0)
        for (size_t k = 16 * n16 + threadIdx.x; k < n; k += blockDim.x) add(x[k]);
    if (cnt) atomicAdd(&hh[cur & 63], cnt);
    __syncthreads();
    if (threadIdx.x < 33) {
        const unsigned t = h[0][threadIdx.x] + h[1][threadIdx.x] + h[2][threadIdx.x] + h[3][threadIdx.x];
        if (t) atomicAdd(&hist[threadIdx.x], t);
    }
}

constexpr int kHistWin = 8192;  // privatised bins around the zero residual symbol

__global__ void __launch_bounds__(512) hist_u16_kernel(const uint16_t* __restrict__ x, size_t n,
                                                       unsigned* __restrict__ hist) {
    __shared__ unsigned h[kHistWin];
    for (int k = threadIdx.x; k < kHistWin; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const int lo = kRadius - kHistWin / 2;
    unsigned cur = 0, cnt = 0;
    auto flush = [&]() {
        if (!cnt) return;
        const unsigned r = cur - (unsigned)lo;
        if (r < (unsigned)kHistWin) atomicAdd(&h[r], cnt);
        else atomicAdd(&hist[cur], cnt);
    };
    auto add = [&](unsigned sy) {
        if (sy == cur) {
            ++cnt;
        } else {
            flush();
            cur = sy;
            cnt = 1;
        }
    };
    const size_t n8 = n / 8;
    const uint4* x4 = reinterpret_cast<const uint4*>(x);
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n8; k += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = __ldcs(x4 + k);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 8; ++e) add((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu);
    }
    if (blockIdx.x == 0)
        for (size_t k = 8 * n8 + threadIdx.x; k < n; k += blockDim.x) add(x[k]);
    flush();
    __syncthreads();
    for (int k = threadIdx.x; k < kHistWin; k += blockDim.x)
        if (h[k]) atomicAdd(&hist[lo + k], h[k]);
}


// ---------------------------------------------------------------------------
// Decoder: expansion of Q_xi, Q_d and L_d to the vertices, the inverse of the
// tiled compaction above.  Tiles of kCmpTile vertices in raster order: a
// count per tile (residual symbols from the bound codes), a scan of the tile
// counts, a pass that gathers each vertex's two residual symbols (block scan
// of the counts inside the tile) and counts the verbatim values they call
// for, a scan of those tile counts, and a pass that gathers the verbatim
// values.  The results are laid out in raster order and then moved to the
// pipeline's strip-diagonal layout by a transposing copy.  A stream whose
// counts do not match is reported through the status word; nothing reads or
// writes out of bounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load16_codes(const uint8_t* __restrict__ qxi, size_t N, size_t base,
                                             unsigned char c[kCmpPer]) {
    if (base + kCmpPer <= N) {
        const uint4 cv = __ldg(reinterpret_cast<const uint4*>(qxi + base));
        const unsigned cw[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
        for (int k = 0; k < kCmpPer; ++k) c[k] = (unsigned char)(cw[k >> 2] >> (8 * (k & 3)));
    } else {
#pragma unroll
        for (int k = 0; k < kCmpPer; ++k) c[k] = base + k < N ? qxi[base + k] : (unsigned char)0;
    }
}

// residual symbols per tile (2 per vertex with a nonzero bound code)
__global__ void __launch_bounds__(kCmpThreads) dec_tile_qd_kernel(const uint8_t* __restrict__ qxi, size_t N,
                                                                  unsigned long long* __restrict__ tile_cnt,
                                                                  int* __restrict__ status) {
    __shared__ unsigned long long wt[32], tot;
    const size_t base = (size_t)blockIdx.x * kCmpTile + (size_t)threadIdx.x * kCmpPer;
    unsigned char c[kCmpPer];
    load16_codes(qxi, N, base, c);
    unsigned long long n = 0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k) {
        n += c[k] ? 2u : 0u;
        bad |= c[k] > 24;
    }
    if (bad) atomicCAS(status, 0, kStatusCorrupt);
    block_exclusive_scan(n, wt, &tot);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = tot;
}

// sym[v] = both residual symbols of v (0 without a bound); tile_ld[b] = the
// verbatim values the tile's symbols call for
__global__ void __launch_bounds__(kCmpThreads) dec_tile_sym_kernel(const uint8_t* __restrict__ qxi, size_t N,
                                                                   const uint16_t* __restrict__ qd, size_t n_qd,
                                                                   const unsigned long long* __restrict__ qd_off,
                                                                   uint32_t* __restrict__ sym,
                                                                   unsigned long long* __restrict__ tile_ld,
                                                                   int* __restrict__ status) {
    __shared__ unsigned long long wt[32], tot;
    const size_t base = (size_t)blockIdx.x * kCmpTile + (size_t)threadIdx.x * kCmpPer;
    unsigned char c[kCmpPer];
    load16_codes(qxi, N, base, c);
    unsigned long long n = 0;
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k) n += c[k] ? 2u : 0u;
    size_t o = (size_t)(block_exclusive_scan(n, wt, &tot) + qd_off[blockIdx.x]);
    __syncthreads();  // wt is scanned again below
    unsigned long long nl = 0;
    uint32_t sy[kCmpPer];
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k) {
        uint32_t x = 0;
        if (c[k]) {
            if (o + 2 > n_qd) {
                atomicCAS(status, 0, kStatusCorrupt);
            } else {
                x = (uint32_t)qd[o] | ((uint32_t)qd[o + 1] << 16);
            }
            o += 2;
        }
        sy[k] = x;
        nl += vertex_count(c[k], x) & 0xFFFFFFFFull;
    }
    if (base + kCmpPer <= N) {
#pragma unroll
        for (int k = 0; k < kCmpPer; k += 4)
            *reinterpret_cast<uint4*>(sym + base + k) = make_uint4(sy[k], sy[k + 1], sy[k + 2], sy[k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < kCmpPer; ++k)
            if (base + k < N) sym[base + k] = sy[k];
    }
    // tiles past N count nothing (their codes read as 0, so nl counts 2 per
    // missing vertex: exclude them)
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k)
        if (base + k >= N) nl -= 2;
    block_exclusive_scan(nl, wt, &tot);
    if (threadIdx.x == 0) tile_ld[blockIdx.x] = tot;
}

// the vertices' (bound code, symbols) and verbatim values in raster order,
// gathered in shared memory and written out with consecutive addresses (a
// thread's own 16 vertices would scatter the stores across the warp)
constexpr size_t kRawSmem = (size_t)kCmpTile * 2 * sizeof(int2);
__global__ void __launch_bounds__(kCmpThreads) dec_tile_raw_kernel(const uint8_t* __restrict__ qxi,
                                                                   const uint32_t* __restrict__ sym, size_t N,
                                                                   const int32_t* __restrict__ ld, size_t n_ld,
                                                                   const unsigned long long* __restrict__ ld_off,
                                                                   int2* __restrict__ dcs, int2* __restrict__ raw,
                                                                   int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    int2* sdcs = reinterpret_cast<int2*>(sm_raw);  // [kCmpTile]
    int2* sraw = sdcs + kCmpTile;
    __shared__ unsigned long long wt[32], tot;
    const size_t tile0 = (size_t)blockIdx.x * kCmpTile;
    const size_t base = tile0 + (size_t)threadIdx.x * kCmpPer;
    unsigned char c[kCmpPer];
    uint32_t sy[kCmpPer];
    load16(qxi, sym, N, base, c, sy);
    unsigned long long n = 0;
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k)
        if (base + k < N) n += vertex_count(c[k], sy[k]) & 0xFFFFFFFFull;
    size_t o = (size_t)(block_exclusive_scan(n, wt, &tot) + ld_off[blockIdx.x]);
#pragma unroll
    for (int k = 0; k < kCmpPer; ++k) {
        const size_t v = base + k;
        if (v >= N) break;
        int2 rr = make_int2(0, 0);
        const bool need_u = c[k] == 0 || (sy[k] & 0xFFFFu) == 0, need_v = c[k] == 0 || (sy[k] >> 16) == 0;
        if (o + need_u + need_v > n_ld) {
            atomicCAS(status, 0, kStatusCorrupt);
        } else {
            if (need_u) rr.x = ld[o++];
            if (need_v) rr.y = ld[o++];
        }
        sraw[v - tile0] = rr;
        sdcs[v - tile0] = make_int2((int)c[k], (int)sy[k]);
    }
    __syncthreads();
    const size_t nt = min((size_t)kCmpTile, N - tile0);
    for (size_t x = threadIdx.x; x < nt; x += kCmpThreads) {
        dcs[tile0 + x] = sdcs[x];
        raw[tile0 + x] = sraw[x];
    }
}

// Raster [T][H][W] -> strip-diagonal [T][strip][W + 31][32] (step k of a
// strip, lane l = row 32s + l at column k - l), zero where no vertex sits.
// A block moves 32 steps of one strip: it reads the 32 row segments those
// steps touch (row l: columns k0 - l .. k0 + 31 - l) and writes 32 whole
// 256-byte step lines of each array.
constexpr int kDiagSteps = 32;
__global__ void __launch_bounds__(256) diag_transpose_kernel(const int2* __restrict__ a_in,
                                                             const int2* __restrict__ b_in, int H, int W, int T,
                                                             int2* __restrict__ a_out, int2* __restrict__ b_out) {
    __shared__ int2 sa[32][kDiagSteps + 1], sb[32][kDiagSteps + 1];  // [lane][step in the block]
    const int nstrips = (H + 31) >> 5, nsteps = W + 31;
    const int nkb = (nsteps + kDiagSteps - 1) / kDiagSteps;
    const long long nb = (long long)T * nstrips * nkb;
    const int lane = (int)(threadIdx.x & 31u), w = (int)(threadIdx.x >> 5);
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        const int kb = (int)(b % nkb);
        const long long ts = b / nkb;
        const int s = (int)(ts % nstrips), t = (int)(ts / nstrips);
        const int k0 = kb * kDiagSteps;
        // row l of the strip, columns k0 - l + m (m = lane): coalesced reads
        for (int l = w; l < 32; l += 8) {
            const int i = 32 * s + l, j = k0 - l + lane;
            const bool ok = i < H && j >= 0 && j < W;
            const size_t v = ((size_t)t * H + (ok ? i : 0)) * W + (ok ? j : 0);
            sa[l][lane] = ok ? __ldg(a_in + v) : make_int2(0, 0);
            sb[l][lane] = ok ? __ldg(b_in + v) : make_int2(0, 0);
        }
        __syncthreads();
        // step k0 + m: lane l's element is (row l, column k0 + m - l) = s?[l][m]
        for (int m = w; m < kDiagSteps; m += 8) {
            const int k = k0 + m;
            if (k >= nsteps) break;
            const size_t d = (((size_t)t * nstrips + s) * (size_t)nsteps + k) * 32 + lane;
            a_out[d] = sa[lane][m];
            b_out[d] = sb[lane][m];
        }
        __syncthreads();
    }
}

// Block modes (one byte each, nonzero = SL) as bits, least significant bit
// first: byte b of the output holds modes 8b .. 8b + 7.
__global__ void __launch_bounds__(256) pack_bits_kernel(const uint8_t* __restrict__ in, size_t n,
                                                        uint8_t* __restrict__ out) {
    const size_t nb = (n + 7) / 8;
    for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < nb; b += (size_t)gridDim.x * blockDim.x) {
        unsigned v = 0;
        for (int k = 0; k < 8; ++k) {
            const size_t x = 8 * b + k;
            if (x < n && in[x]) v |= 1u << k;
        }
        out[b] = (uint8_t)v;
    }
}

size_t compact_tiles(size_t N) { return (N + kCmpTile - 1) / kCmpTile; }

void launch_tile_count(const uint8_t* qxi, const uint32_t* sym, size_t N, unsigned long long* tile_cnt,
                       cudaStream_t s) {
    if (N) tile_count_kernel<<<(unsigned)compact_tiles(N), kCmpThreads, 0, s>>>(qxi, sym, N, tile_cnt);
}

void launch_tile_scatter(const uint8_t* qxi, const uint32_t* sym, const int32_t* q,
                         const unsigned long long* tile_off, size_t N, uint16_t* qd_out, int32_t* ld_out,
                         cudaStream_t s) {
    if (!N) return;
    // the gather buffer is above the default 48 KB of shared memory (set once;
    // if that failed, so does the launch, and the caller reads the error)
    static const cudaError_t attr = cudaFuncSetAttribute(
        tile_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterSmem);
    (void)attr;
    tile_scatter_kernel<<<(unsigned)compact_tiles(N), kCmpThreads, kScatterSmem, s>>>(
        qxi, sym, reinterpret_cast<const int2*>(q), tile_off, N, qd_out, ld_out);
}

void launch_dec_tile_qd(const uint8_t* qxi, size_t N, unsigned long long* tile_cnt, int* status, cudaStream_t s) {
    if (N) dec_tile_qd_kernel<<<(unsigned)compact_tiles(N), kCmpThreads, 0, s>>>(qxi, N, tile_cnt, status);
}
void launch_dec_tile_sym(const uint8_t* qxi, size_t N, const uint16_t* qd, size_t n_qd,
                         const unsigned long long* qd_off, uint32_t* sym, unsigned long long* tile_ld, int* status,
                         cudaStream_t s) {
    if (N)
        dec_tile_sym_kernel<<<(unsigned)compact_tiles(N), kCmpThreads, 0, s>>>(qxi, N, qd, n_qd, qd_off, sym, tile_ld,
                                                                              status);
}
void launch_dec_tile_raw(const uint8_t* qxi, const uint32_t* sym, size_t N, const int32_t* ld, size_t n_ld,
                         const unsigned long long* ld_off, int2* dcs, int2* raw, int* status, cudaStream_t s) {
    if (!N) return;
    // the gather buffers are above the default 48 KB of shared memory (set
    // once; if that failed, so does the launch, and the caller reads the error)
    static const cudaError_t attr =
        cudaFuncSetAttribute(dec_tile_raw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRawSmem);
    (void)attr;
    dec_tile_raw_kernel<<<(unsigned)compact_tiles(N), kCmpThreads, kRawSmem, s>>>(qxi, sym, N, ld, n_ld, ld_off, dcs,
                                                                                raw, status);
}
void launch_diag_transpose(const int2* a_in, const int2* b_in, int H, int W, int T, int2* a_out, int2* b_out,
                           cudaStream_t s) {
    const long long nb = (long long)T * ((H + 31) / 32) * ((W + 31 + kDiagSteps - 1) / kDiagSteps);
    if (nb) diag_transpose_kernel<<<(unsigned)std::min<long long>(nb, 152 * 16), 256, 0, s>>>(a_in, b_in, H, W, T,
                                                                                              a_out, b_out);
}

void launch_pack_bits(const uint8_t* in, size_t n, uint8_t* out, cudaStream_t s) {
    const size_t nb = (n + 7) / 8;
    if (nb) pack_bits_kernel<<<(unsigned)std::min<size_t>((nb + 255) / 256, 4096), 256, 0, s>>>(in, n, out);
}

void launch_hist_u8(const uint8_t* x, size_t n, unsigned* hist, cudaStream_t s) {
    if (n) hist_u8_kernel<<<608, 256, 0, s>>>(x, n, hist);
}

void launch_hist_u16(const uint16_t* x, size_t n, unsigned* hist, cudaStream_t s) {
    if (n) hist_u16_kernel<<<304, 512, 0, s>>>(x, n, hist);
}

// ---------------------------------------------------------------------------
// Bit packing.  table[sym] = (code << 5) | len.  A tile of kTileSyms symbols
// is packed by one CTA: 256 threads x 16 consecutive symbols, bit offsets by
// a block scan, bits OR-ed into a shared-memory copy of the tile's word span,
// interior words stored plainly and the two boundary words (shared with the
// neighbouring tiles) OR-ed into the zero-initialised output.
// ---------------------------------------------------------------------------
constexpr int kEncThreads = 256;
constexpr int kEncPer = kTileSyms / kEncThreads;  // 16
constexpr int kEncWords = kTileSyms * 24 / 32 + 2;

template <typename Sym>
__global__ void __launch_bounds__(kEncThreads) tile_bits_kernel(const Sym* __restrict__ x, size_t n,
                                                                const uint32_t* __restrict__ table,
                                                                unsigned long long* __restrict__ tile_bits) {
    __shared__ unsigned long long wt[32], tot;
    size_t base = (size_t)blockIdx.x * kTileSyms + (size_t)threadIdx.x * kEncPer;
    unsigned long long b = 0;
#pragma unroll
    for (int k = 0; k < kEncPer; ++k)
        if (base + k < n) b += __ldg(table + x[base + k]) & 31u;
    block_exclusive_scan(b, wt, &tot);
    if (threadIdx.x == 0) tile_bits[blockIdx.x] = tot;
}

template <typename Sym>
__global__ void __launch_bounds__(kEncThreads) encode_kernel(const Sym* __restrict__ x, size_t n,
                                                             const uint32_t* __restrict__ table,
                                                             const unsigned long long* __restrict__ tile_off,
                                                             uint32_t* __restrict__ words) {
    __shared__ unsigned long long wt[32], tot;
    __shared__ uint32_t buf[kEncWords];
    for (int k = threadIdx.x; k < kEncWords; k += kEncThreads) buf[k] = 0;
    size_t base = (size_t)blockIdx.x * kTileSyms + (size_t)threadIdx.x * kEncPer;
    uint32_t e[kEncPer];
    unsigned long long b = 0;
#pragma unroll
    for (int k = 0; k < kEncPer; ++k) {
        e[k] = base + k < n ? __ldg(table + x[base + k]) : 0u;
        b += e[k] & 31u;
    }
    unsigned long long off = block_exclusive_scan(b, wt, &tot);  // includes a __syncthreads
    const unsigned long long t0 = tile_off[blockIdx.x];
    unsigned pos = (unsigned)(t0 & 31ull) + (unsigned)off;      // bit position within buf
#pragma unroll
    for (int k = 0; k < kEncPer; ++k) {
        unsigned len = e[k] & 31u, code = e[k] >> 5;
        if (len == 0) continue;
        unsigned w = pos >> 5, r = pos & 31u;
        if (r + len <= 32) {
            atomicOr(&buf[w], code << (32 - r - len));
        } else {
            unsigned spill = r + len - 32;
            atomicOr(&buf[w], code >> spill);
            atomicOr(&buf[w + 1], code << (32 - spill));
        }
        pos += len;
    }
    __syncthreads();
    const unsigned total = (unsigned)(t0 & 31ull) + (unsigned)tot;
    const unsigned nw = (total + 31) >> 5;
    const size_t w0 = (size_t)(t0 >> 5);
    for (unsigned k = threadIdx.x; k < nw; k += kEncThreads) {
        if (k == 0 || k == nw - 1) atomicOr(&words[w0 + k], buf[k]);
        else words[w0 + k] = buf[k];
    }
}

static unsigned ntiles(size_t n) { return (unsigned)((n + kTileSyms - 1) / kTileSyms); }

void launch_tile_bits_u8(const uint8_t* x, size_t n, const uint32_t* table, unsigned long long* tile_bits,
                         cudaStream_t s) {
    if (n) tile_bits_kernel<uint8_t><<<ntiles(n), kEncThreads, 0, s>>>(x, n, table, tile_bits);
}
void launch_tile_bits_u16(const uint16_t* x, size_t n, const uint32_t* table, unsigned long long* tile_bits,
                          cudaStream_t s) {
    if (n) tile_bits_kernel<uint16_t><<<ntiles(n), kEncThreads, 0, s>>>(x, n, table, tile_bits);
}
void launch_encode_u8(const uint8_t* x, size_t n, const uint32_t* table, const unsigned long long* tile_off,
                      uint32_t* words, cudaStream_t s) {
    if (n) encode_kernel<uint8_t><<<ntiles(n), kEncThreads, 0, s>>>(x, n, table, tile_off, words);
}
void launch_encode_u16(const uint16_t* x, size_t n, const uint32_t* table, const unsigned long long* tile_off,
                       uint32_t* words, cudaStream_t s) {
    if (n) encode_kernel<uint16_t><<<ntiles(n), kEncThreads, 0, s>>>(x, n, table, tile_off, words);
}

}  // namespace cpt
