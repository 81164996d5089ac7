// Decoder kernels: canonical Huffman decoding from the stream's sync points,
// expansion of the bound codes, residual symbols and verbatim values to the
// vertices (in the strip-diagonal layout of the encoder's pipeline, which
// then runs in decoding mode: the inverse of the raster loop of Alg. 3, with
// bounds from the stream and no face work), and the conversion back to
// float.  A malformed stream sets the status word to a corruption code;
// nothing reads or writes out of bounds.
#include "cpt_dev.cuh"
#include "cpt_internal.h"

namespace cpt {

// ---------------------------------------------------------------------------
// Huffman decoding: one thread per chunk of kChunkSyms symbols, starting at
// the chunk's recorded bit offset; codes are read most significant bit first.
// ---------------------------------------------------------------------------
template <typename Out>
__global__ void __launch_bounds__(128) huff_decode_kernel(HuffDecode h, Out* __restrict__ out, int* __restrict__ status) {
    const unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long nchunks = (h.nsym + kChunkSyms - 1) / kChunkSyms;
    if (c >= nchunks) return;
    const unsigned long long nbits = h.nwords * 32ull;
    unsigned long long p = h.chunk_off[c];
    const unsigned long long x0 = c * kChunkSyms;
    const unsigned long long x1 = min(h.nsym, x0 + kChunkSyms);
    for (unsigned long long x = x0; x < x1; ++x) {
        if (p >= nbits) { atomicCAS(status, 0, kStatusCorrupt); return; }
        const unsigned long long wi = p >> 5;  // words has two zero words of padding
        const unsigned long long w64 = (((unsigned long long)h.words[wi] << 32) | h.words[wi + 1]) << (p & 31);
        const unsigned w24 = (unsigned)(w64 >> 40);
        unsigned e = h.lut[w24 >> 12];
        if (e == 0) {
            for (int l = 13; l <= 24; ++l) {
                const unsigned code = w24 >> (24 - l);
                const unsigned k = code - h.first[l];
                if (code >= h.first[l] && k < h.count[l]) {
                    e = (h.sorted[h.base[l] + k] << 5) | (unsigned)l;
                    break;
                }
            }
            if (e == 0) { atomicCAS(status, 0, kStatusCorrupt); return; }
        }
        p += e & 31u;
        out[x] = (Out)(e >> 5);
    }
    if (p > nbits || (c + 1 < nchunks && p != h.chunk_off[c + 1])) atomicCAS(status, 0, kStatusCorrupt);
}

// ---------------------------------------------------------------------------
// expansion to the vertices
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) qd_count_kernel(const uint8_t* __restrict__ qxi, size_t N,
                                                       unsigned long long* __restrict__ cnt, int* __restrict__ status) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        const uint8_t c = qxi[v];
        if (c > 24) atomicCAS(status, 0, kStatusCorrupt);
        cnt[v] = c ? 2ull : 0ull;
    }
}

__global__ void __launch_bounds__(256) gather_sym_kernel(const uint8_t* __restrict__ qxi,
                                                         const unsigned long long* __restrict__ off,
                                                         const uint16_t* __restrict__ qd, size_t n_qd, size_t N,
                                                         uint32_t* __restrict__ sym, int* __restrict__ status) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        uint32_t s = 0;
        if (qxi[v]) {
            const size_t o = (size_t)off[v];
            if (o + 2 > n_qd) {
                atomicCAS(status, 0, kStatusCorrupt);
            } else {
                s = (uint32_t)qd[o] | ((uint32_t)qd[o + 1] << 16);
            }
        }
        sym[v] = s;
    }
}

// Verbatim values of each vertex from L_d, written with (bound code, residual
// symbols) in the strip-diagonal layout the reconstruction pipeline stages.
__global__ void __launch_bounds__(256) gather_raw_kernel(const uint8_t* __restrict__ qxi, const uint32_t* __restrict__ sym,
                                                         const unsigned long long* __restrict__ off,
                                                         const int32_t* __restrict__ ld, size_t n_ld, int H, int W,
                                                         int T, int2* __restrict__ dcs, int2* __restrict__ raw,
                                                         int* __restrict__ status) {
    const size_t N = (size_t)H * W * T, sl = (size_t)H * W;
    const size_t nstrips = (size_t)(H + 31) >> 5;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        const size_t t = v / sl, rem = v - t * sl;
        const int i = (int)(rem / W), j = (int)(rem - (size_t)i * W);
        const size_t dv = ((t * nstrips + (i >> 5)) * (size_t)(W + 31) + (j + (i & 31))) * 32 + (i & 31);
        size_t o = (size_t)(off[v] & 0xFFFFFFFFull);
        int2 r = make_int2(0, 0);
        if (qxi[v] == 0) {
            if (o + 2 > n_ld) { atomicCAS(status, 0, kStatusCorrupt); }
            else { r.x = ld[o]; r.y = ld[o + 1]; }
        } else {
            const uint32_t s = sym[v];
            const size_t need = ((s & 0xFFFFu) == 0) + ((s >> 16) == 0);
            if (o + need > n_ld) {
                atomicCAS(status, 0, kStatusCorrupt);
            } else {
                if ((s & 0xFFFFu) == 0) r.x = ld[o++];
                if ((s >> 16) == 0) r.y = ld[o];
            }
        }
        raw[dv] = r;
        dcs[dv] = make_int2((int)qxi[v], (int)sym[v]);
    }
}

// The pipeline's reconstruction words (x, y ^ kQhatTag) back to values.
__global__ void __launch_bounds__(256) untag_kernel(int2* __restrict__ q, size_t N) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x)
        q[v].y ^= kQhatTag;
}

// q_hat * 2^-k in float32 (exact: |q_hat| <= 2^24)
__global__ void __launch_bounds__(256) to_float_kernel(const int2* __restrict__ qhat, size_t N, double inv_scale,
                                                       float2* __restrict__ out) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        const int2 q = qhat[v];
        out[v] = make_float2((float)((double)q.x * inv_scale), (float)((double)q.y * inv_scale));
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_huff_decode_u8(const HuffDecode& h, uint8_t* out, int* status, cudaStream_t s) {
    const unsigned long long nchunks = (h.nsym + kChunkSyms - 1) / kChunkSyms;
    if (nchunks) huff_decode_kernel<uint8_t><<<(unsigned)((nchunks + 127) / 128), 128, 0, s>>>(h, out, status);
}
void launch_huff_decode_u16(const HuffDecode& h, uint16_t* out, int* status, cudaStream_t s) {
    const unsigned long long nchunks = (h.nsym + kChunkSyms - 1) / kChunkSyms;
    if (nchunks) huff_decode_kernel<uint16_t><<<(unsigned)((nchunks + 127) / 128), 128, 0, s>>>(h, out, status);
}
void launch_qd_count(const uint8_t* qxi, size_t N, unsigned long long* cnt, int* status, cudaStream_t s) {
    qd_count_kernel<<<1216, 256, 0, s>>>(qxi, N, cnt, status);
}
void launch_gather_sym(const uint8_t* qxi, const unsigned long long* off, const uint16_t* qd, size_t n_qd, size_t N,
                       uint32_t* sym, int* status, cudaStream_t s) {
    gather_sym_kernel<<<1216, 256, 0, s>>>(qxi, off, qd, n_qd, N, sym, status);
}
void launch_gather_raw(const uint8_t* qxi, const uint32_t* sym, const unsigned long long* off, const int32_t* ld,
                       size_t n_ld, int H, int W, int T, int2* dcs, int2* draw, int* status, cudaStream_t s) {
    gather_raw_kernel<<<1216, 256, 0, s>>>(qxi, sym, off, ld, n_ld, H, W, T, dcs, draw, status);
}
void launch_untag(int2* qhat, size_t N, cudaStream_t s) { untag_kernel<<<1216, 256, 0, s>>>(qhat, N); }
void launch_to_float(const int2* qhat, size_t N, double inv_scale, float* out, cudaStream_t s) {
    to_float_kernel<<<1216, 256, 0, s>>>(qhat, N, inv_scale, reinterpret_cast<float2*>(out));
}

}  // namespace cpt
