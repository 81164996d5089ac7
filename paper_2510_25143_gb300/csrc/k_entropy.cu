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
// component), counts packed as (n_qd << 32) | n_ld
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) count_pack_kernel(const uint8_t* __restrict__ qxi,
                                                         const uint32_t* __restrict__ sym, size_t N,
                                                         unsigned long long* __restrict__ cnt) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        unsigned long long c;
        if (qxi[v]) {
            uint32_t s = sym[v];
            c = (2ull << 32) | (unsigned long long)(((s & 0xFFFFu) == 0) + ((s >> 16) == 0));
        } else {
            c = 2ull;
        }
        cnt[v] = c;
    }
}

__global__ void __launch_bounds__(256) scatter_kernel(const uint8_t* __restrict__ qxi, const uint32_t* __restrict__ sym,
                                                      const int2* __restrict__ q,
                                                      const unsigned long long* __restrict__ off, size_t N,
                                                      uint16_t* __restrict__ qd, int32_t* __restrict__ ld) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        unsigned long long o = off[v];
        size_t pq = (size_t)(o >> 32), pl = (size_t)(o & 0xFFFFFFFFull);
        int2 x = q[v];
        if (qxi[v]) {
            uint32_t s = sym[v];
            uint16_t su = (uint16_t)(s & 0xFFFFu), sv = (uint16_t)(s >> 16);
            qd[pq] = su;
            qd[pq + 1] = sv;
            if (su == 0) ld[pl++] = x.x;
            if (sv == 0) ld[pl] = x.y;
        } else {
            ld[pl] = x.x;
            ld[pl + 1] = x.y;
        }
    }
}

// ---------------------------------------------------------------------------
// histograms
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) hist_u8_kernel(const uint8_t* __restrict__ x, size_t n,
                                                      unsigned* __restrict__ hist) {
    __shared__ unsigned h[64];
    if (threadIdx.x < 64) h[threadIdx.x] = 0;
    __syncthreads();
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        atomicAdd(&h[x[k] & 63], 1u);
    __syncthreads();
    if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

constexpr int kHistWin = 8192;  // privatised bins around the zero residual symbol

__global__ void __launch_bounds__(512) hist_u16_kernel(const uint16_t* __restrict__ x, size_t n,
                                                       unsigned* __restrict__ hist) {
    __shared__ unsigned h[kHistWin];
    for (int k = threadIdx.x; k < kHistWin; k += blockDim.x) h[k] = 0;
    __syncthreads();
    const int lo = kRadius - kHistWin / 2;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int s = x[k];
        unsigned r = (unsigned)(s - lo);
        if (r < (unsigned)kHistWin) atomicAdd(&h[r], 1u);
        else atomicAdd(&hist[s], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kHistWin; k += blockDim.x)
        if (h[k]) atomicAdd(&hist[lo + k], h[k]);
}

void launch_count_pack(const uint8_t* qxi, const uint32_t* sym, size_t N, unsigned long long* cnt, cudaStream_t s) {
    count_pack_kernel<<<1216, 256, 0, s>>>(qxi, sym, N, cnt);
}

void launch_scatter(const uint8_t* qxi, const uint32_t* sym, const int32_t* q, const unsigned long long* off,
                    size_t N, uint16_t* qd_out, int32_t* ld_out, cudaStream_t s) {
    scatter_kernel<<<1216, 256, 0, s>>>(qxi, sym, reinterpret_cast<const int2*>(q), off, N, qd_out, ld_out);
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
