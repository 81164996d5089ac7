// Decoder kernels: canonical Huffman decoding from the stream's sync points,
// the untagging of the reconstruction words and the conversion back to
// float.  (The expansion of the bound codes, residual symbols and verbatim
// values to the vertices, in the strip-diagonal layout of the encoder's
// pipeline, sits beside the encoder's compaction; the pipeline then runs in
// decoding mode: the inverse of the raster loop of Alg. 3, with bounds from
// the stream and no face work.)  A malformed stream sets the status word to a corruption code;
// nothing reads or writes out of bounds.
#include <cmath>

#include "cpt_dev.cuh"
#include "cpt_internal.h"

namespace cpt {

// ---------------------------------------------------------------------------
// Huffman decoding: one thread per chunk of kChunkSyms symbols (the stream's
// sync points), codes read most significant bit first.  The bits pass
// through a 64-bit register buffer refilled a word at a time; one lookup of
// the window's first 12 bits yields up to three complete short codes
// (lut3), codes longer than 12 bits take the canonical tables.  Symbols
// leave in 32-bit words.  The tables sit in shared memory.
// ---------------------------------------------------------------------------
template <typename Out>
__global__ void __launch_bounds__(64) huff_decode_kernel(HuffDecode h, Out* __restrict__ out, int* __restrict__ status) {
    __shared__ unsigned long long lut3[4096];
    __shared__ uint32_t first[25], count[25], base[25];
    for (int k = threadIdx.x; k < 4096; k += blockDim.x) lut3[k] = __ldg(h.lut3 + k);
    if (threadIdx.x < 25) {
        first[threadIdx.x] = __ldg(h.first + threadIdx.x);
        count[threadIdx.x] = __ldg(h.count + threadIdx.x);
        base[threadIdx.x] = __ldg(h.base + threadIdx.x);
    }
    __syncthreads();
    const unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nchunks = (h.nsym + kChunkSyms - 1) / kChunkSyms;
    if (c >= nchunks) return;
    const unsigned long long nbits = h.nwords * 32ull;
    const unsigned long long nw = h.nwords + 2;  // words has two zero words of padding
    unsigned long long p = h.chunk_off[c];
    if (p > nbits) { atomicCAS(status, 0, kStatusCorrupt); return; }
    // buf holds the stream's bits from p on, left aligned; nb of them are valid
    unsigned long long wi = p >> 5;
    unsigned long long buf = (((unsigned long long)__ldg(h.words + wi) << 32) | __ldg(h.words + wi + 1)) << (p & 31);
    int nb = 64 - (int)(p & 31);
    wi += 2;
    const unsigned long long x0 = c * kChunkSyms;
    const unsigned n = (unsigned)(min(h.nsym, x0 + kChunkSyms) - x0);  // symbols of this chunk
    Out* o = out + x0;  // 4-byte aligned: kChunkSyms * sizeof(Out) is
    constexpr unsigned kPerWord = 4 / sizeof(Out);
    uint32_t word = 0;  // symbols of the current output word
    unsigned x = 0, inw = 0;
    unsigned long long used = 0;  // bits consumed
    const unsigned long long avail = nbits - p;
    auto emit = [&](uint32_t sym) {
        word |= sym << (8 * sizeof(Out) * inw);
        if (++inw == kPerWord) {
            *reinterpret_cast<uint32_t*>(o + x + 1 - kPerWord) = word;
            word = 0;
            inw = 0;
        }
        ++x;
    };
    while (x < n) {
        if (nb <= 32) {  // keeps >= 24 valid bits (the longest code) before every lookup
            const unsigned long long w = wi < nw ? __ldg(h.words + wi) : 0u;
            buf |= w << (32 - nb);
            nb += 32;
            ++wi;
        }
        const unsigned long long e = lut3[(unsigned)(buf >> 52)];
        const unsigned cnt = (unsigned)(e & 3u);
        if (cnt > 0 && x + cnt <= n) {
            const unsigned len = (unsigned)(e >> 2) & 31u;
            emit((uint32_t)(e >> 7) & 0xFFFFu);
            if (cnt > 1) emit((uint32_t)(e >> 23) & 0xFFFFu);
            if (cnt > 2) emit((uint32_t)(e >> 39) & 0xFFFFu);
            buf <<= len;
            nb -= (int)len;
            used += len;
        } else {  // one code: longer than 12 bits, or the chunk's last symbols
            const unsigned w24 = (unsigned)(buf >> 40);
            unsigned sym = 0, l = 0;
            for (unsigned ll = 1; ll <= 24; ++ll) {
                const unsigned code = w24 >> (24 - ll);
                const unsigned k = code - first[ll];
                if (code >= first[ll] && k < count[ll]) {
                    sym = __ldg(h.sorted + base[ll] + k);
                    l = ll;
                    break;
                }
            }
            if (l == 0) { atomicCAS(status, 0, kStatusCorrupt); return; }
            emit(sym);
            buf <<= l;
            nb -= (int)l;
            used += l;
        }
        if (used > avail) { atomicCAS(status, 0, kStatusCorrupt); return; }
    }
    for (unsigned q = 0; q < inw; ++q)  // the last, partial word
        o[x - inw + q] = (Out)(word >> (8 * sizeof(Out) * q));
    p += used;
    if (c + 1 < nchunks && p != h.chunk_off[c + 1]) atomicCAS(status, 0, kStatusCorrupt);
}

// The pipeline's reconstruction words (x, y ^ kQhatTag) back to values.
__global__ void __launch_bounds__(256) untag_kernel(int2* __restrict__ q, size_t N) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x)
        q[v].y ^= kQhatTag;
}

// q_hat * 2^-k in float32: q_hat is exact in float (|q_hat| <= 2^24) and the
// power of two is applied as two factors 2^a 2^b (a + b = -k) that never
// leave the normal range on the way, so every product is exact.  tag: the
// y halves still carry the reconstruction words' tag (removed here).
__global__ void __launch_bounds__(256) to_float_kernel(const int4* __restrict__ qhat, size_t N2, float g1, float g2,
                                                       int tag, float4* __restrict__ out) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N2; v += (size_t)gridDim.x * blockDim.x) {
        int4 q = __ldcs(qhat + v);
        q.y ^= tag;
        q.w ^= tag;
        out[v] = make_float4(__fmul_rn(__fmul_rn(__int2float_rn(q.x), g1), g2),
                             __fmul_rn(__fmul_rn(__int2float_rn(q.y), g1), g2),
                             __fmul_rn(__fmul_rn(__int2float_rn(q.z), g1), g2),
                             __fmul_rn(__fmul_rn(__int2float_rn(q.w), g1), g2));
    }
}
__global__ void __launch_bounds__(256) to_float_v_kernel(const int2* __restrict__ qhat, size_t N, float g1, float g2,
                                                          int tag, float2* __restrict__ out) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        int2 q = qhat[v];
        q.y ^= tag;
        out[v] = make_float2(__fmul_rn(__fmul_rn(__int2float_rn(q.x), g1), g2),
                             __fmul_rn(__fmul_rn(__int2float_rn(q.y), g1), g2));
    }
}
__global__ void to_float_tail_kernel(const int2* __restrict__ qhat, float g1, float g2, int tag,
                                     float2* __restrict__ out) {
    int2 q = qhat[0];
    q.y ^= tag;
    out[0] = make_float2(__fmul_rn(__fmul_rn(__int2float_rn(q.x), g1), g2),
                         __fmul_rn(__fmul_rn(__int2float_rn(q.y), g1), g2));
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_huff_decode_u8(const HuffDecode& h, uint8_t* out, int* status, cudaStream_t s) {
    const unsigned long long nchunks = (h.nsym + kChunkSyms - 1) / kChunkSyms;
    if (nchunks) huff_decode_kernel<uint8_t><<<(unsigned)((nchunks + 63) / 64), 64, 0, s>>>(h, out, status);
}
void launch_huff_decode_u16(const HuffDecode& h, uint16_t* out, int* status, cudaStream_t s) {
    const unsigned long long nchunks = (h.nsym + kChunkSyms - 1) / kChunkSyms;
    if (nchunks) huff_decode_kernel<uint16_t><<<(unsigned)((nchunks + 63) / 64), 64, 0, s>>>(h, out, status);
}
void launch_untag(int2* qhat, size_t N, cudaStream_t s) { untag_kernel<<<1216, 256, 0, s>>>(qhat, N); }
void launch_to_float(const int2* qhat, size_t N, int k, float* out, cudaStream_t s, bool tagged) {
    const int tag = tagged ? kQhatTag : 0;
    const int a = -k / 2, b = -k - a;
    const float g1 = std::ldexp(1.0f, a), g2 = std::ldexp(1.0f, b);
    // two vertices per thread (16-byte accesses when out is 16-byte aligned)
    if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
        if (N / 2)
            to_float_kernel<<<1216, 256, 0, s>>>(reinterpret_cast<const int4*>(qhat), N / 2, g1, g2, tag,
                                                 reinterpret_cast<float4*>(out));
        if (N & 1)
            to_float_tail_kernel<<<1, 1, 0, s>>>(qhat + N - 1, g1, g2, tag, reinterpret_cast<float2*>(out) + N - 1);
    } else {  // output only 8-byte aligned: one vertex per thread
        to_float_v_kernel<<<1216, 256, 0, s>>>(qhat, N, g1, g2, tag, reinterpret_cast<float2*>(out));
    }
}

}  // namespace cpt
