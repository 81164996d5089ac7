// Decoder kernels: canonical Huffman decoding from the stream's sync points,
// expansion of the bound codes, residual symbols and verbatim values to the
// vertices, and the reconstruction (the inverse of the raster loop of Alg. 3:
// bounds come from the stream, so there is no face work), pipelined over
// slices like the encoder: SL prep tiles and per-strip warp-systolic
// wavefronts.  A malformed stream sets the status word to a corruption code;
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

__global__ void __launch_bounds__(256) gather_raw_kernel(const uint8_t* __restrict__ qxi, const uint32_t* __restrict__ sym,
                                                         const unsigned long long* __restrict__ off,
                                                         const int32_t* __restrict__ ld, size_t n_ld, size_t N,
                                                         int2* __restrict__ raw, int* __restrict__ status) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
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
        raw[v] = r;
    }
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
// reconstruction pipeline
// ---------------------------------------------------------------------------
constexpr int kHaloD = 34;
struct DChunk {
    uint32_t sym[32][32];
    int2 raw[32][32];
    int2 psl[32][32];
    int2 qp[33][kHaloD];    // reconstruction of slice t-1, rows/cols -1..31 of the chunk
    uint8_t code[32][32];   // bound code, bit 7 = the vertex uses its SL prediction
};
struct DSmem {
    union {
        DChunk buf[2];        // waves
        NetScratch<8> net;    // prep tiles of the learned predictor
    };
    int2 border[64];
};

__device__ __forceinline__ bool uses_sl(const DecodeArgs& a, int t, int i, int j) {
    if (t < 1) return false;
    if (a.pred == 1 || a.pred == 3) return true;
    if (a.pred != 2 && a.pred != 4) return false;
    const size_t bidx = ((size_t)t * a.nby + i / a.B) * a.nbx + j / a.B;
    return (a.mode_bits[bidx >> 3] >> (bidx & 7)) & 1u;
}

// SL (or learned) predictions of tile (t, s, c) for the vertices that use them.
__device__ bool dprep_tile(const DecodeArgs& a, int t, int s, int c, DSmem& sm) {
    const int lane = threadIdx.x, H = a.H, W = a.W;
    const int nstrips = (H + 31) / 32;
    const int i0 = 32 * s, j0 = 32 * c;
    const int s_req = min(nstrips - 1, (i0 + 31 + a.R) >> 5);
    const unsigned col_req = (unsigned)min(W, j0 + 32 + a.R);
    if (!warp_wait_geq(a.status, a.timeout_ns, a.progress + (size_t)(t - 1) * nstrips + s_req, col_req)) return false;
    const GlobalSlice P{a.qhat + (size_t)(t - 1) * H * W, W};
    if (a.pred == 3 || a.pred == 4) {
        // learned predictor: the tile's 8 x 8 sub-tiles
        auto prev = [&](int i, int j) -> int2 {
            return (i >= 0 && i < H && j >= 0 && j < W) ? P.at(i, j) : make_int2(0, 0);
        };
        for (int r0 = i0; r0 < min(H, i0 + 32); r0 += 8)
            for (int c0 = j0; c0 < min(W, j0 + 32); c0 += 8) {
                auto out = [&](int li, int lj, int2 p) { a.psl[((size_t)t * H + r0 + li) * W + c0 + lj] = p; };
                net_tile<8>(a.net, sm.net, r0, c0, H, W, prev, out);
            }
        warp_publish(a.prep_done + ((size_t)t * nstrips + s) * a.nchunks + c, 1u);
        return true;
    }
    const int j = j0 + lane;
    if (j < W) {
        for (int rr = 0; rr < 32; ++rr) {
            const int i = i0 + rr;
            if (i >= H) break;
            const size_t v = ((size_t)t * H + i) * W + j;
            if (a.qxi[v] == 0 || !uses_sl(a, t, i, j)) continue;
            int pu, pv;
            sl_predict(P, H, W, i, j, a.cfl_x, a.cfl_y, pu, pv);
            a.psl[v] = make_int2(pu, pv);
        }
    }
    warp_publish(a.prep_done + ((size_t)t * nstrips + s) * a.nchunks + c, 1u);
    return true;
}

__device__ void dstage_chunk(const DecodeArgs& a, int t, int i0, int c, DChunk& b, bool need_sl) {
    const int lane = threadIdx.x, H = a.H, W = a.W;
    const int j = 32 * c + lane;
    const size_t sl = (size_t)H * W;
    const int2 z = make_int2(0, 0);
    for (int rr = 0; rr < 32; ++rr) {
        const int i = i0 + rr;
        const bool ok = i < H && j < W;
        const size_t v = ok ? ((size_t)t * H + i) * W + j : 0;
        cp_async4(&b.sym[rr][lane], a.sym + v, ok);
        cp_async8(&b.raw[rr][lane], a.raw + v, ok);
        b.code[rr][lane] = ok ? a.qxi[v] : 0;
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (t >= 1) {
        const int2* P = a.qhat + (size_t)(t - 1) * sl;
        const int jj = 32 * c - 1 + lane;
        const int j31 = 32 * c + 31;
        for (int r0 = 0; r0 < 33; r0 += 11) {
            int2 tmp[11], t31[11];
#pragma unroll
            for (int u = 0; u < 11; ++u) {
                const int i = i0 - 1 + r0 + u;
                const bool rok = i >= 0 && i < H;
                tmp[u] = (rok && jj >= 0 && jj < W) ? __ldcg(P + (size_t)i * W + jj) : z;
                t31[u] = (lane == 0 && rok && j31 < W) ? __ldcg(P + (size_t)i * W + j31) : z;
            }
#pragma unroll
            for (int u = 0; u < 11; ++u) {
                b.qp[r0 + u][lane] = tmp[u];
                if (lane == 0) b.qp[r0 + u][32] = t31[u];
            }
        }
    } else {
        for (int rr = 0; rr < 33; ++rr) {
            b.qp[rr][lane] = z;
            if (lane == 0) b.qp[rr][32] = z;
        }
    }
    if (need_sl) {
        for (int r0 = 0; r0 < 32; r0 += 8) {
            int2 tmp[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + r0 + u;
                tmp[u] = (i < H && j < W) ? __ldcg(a.psl + (size_t)t * sl + (size_t)i * W + j) : z;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) b.psl[r0 + u][lane] = tmp[u];
        }
    }
    for (int rr = 0; rr < 32; ++rr) {
        const int i = i0 + rr;
        if (i < H && j < W && b.code[rr][lane] && uses_sl(a, t, i, j)) b.code[rr][lane] |= 0x80;
    }
    cp_async_wait_all();
}

__device__ bool dwave_item(const DecodeArgs& a, int t, int s, DSmem& sm) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x, H = a.H, W = a.W;
    const int nstrips = (H + 31) / 32;
    const int i0 = 32 * s, i = i0 + lane;
    const bool rowok = i < H;
    const size_t base = (size_t)t * H * W;
    const unsigned* prog_prev = a.progress + (size_t)t * nstrips + (s > 0 ? s - 1 : 0);
    const unsigned* prog_below = a.progress + (size_t)(t > 0 ? t - 1 : 0) * nstrips + s;
    unsigned* prog_me = a.progress + (size_t)t * nstrips + s;
    const bool need_sl = t >= 1 && a.pred != 0 && a.prep_groups > 0;
    int2 left = make_int2(0, 0), up = left, res = left;
    int fetched = 0;
    for (int k = 0; k < W + 31; ++k) {
        const int j = k - lane;
        if ((k & 31) == 0 && k < W) {
            const int c = k >> 5;
            if (need_sl) {
                if (!warp_wait_geq(a.status, a.timeout_ns, a.prep_done + ((size_t)t * nstrips + s) * a.nchunks + c, 1u))
                    return false;
            } else if (t >= 1) {
                if (!warp_wait_geq(a.status, a.timeout_ns, prog_below, (unsigned)min(W, 32 * c + 32))) return false;
            }
            dstage_chunk(a, t, i0, c, sm.buf[c & 1], need_sl);
            __syncwarp();
        }
        if (s > 0 && k < W && k >= fetched) {
            const unsigned seen = warp_wait_geq(a.status, a.timeout_ns, prog_prev, (unsigned)(k + 1));
            if (!seen) return false;
            const int avail = min(min(W, k + 32), (int)seen);
            const int col = fetched + lane;
            if (col < avail) sm.border[col & 63] = __ldcg(a.qhat + base + (size_t)(i0 - 1) * W + col);
            fetched = avail;
            __syncwarp();
        }
        int2 fromprev;
        fromprev.x = __shfl_up_sync(FULL, res.x, 1);
        fromprev.y = __shfl_up_sync(FULL, res.y, 1);
        const int2 upleft = up;
        if (lane == 0) up = (s > 0 && k < W) ? sm.border[k & 63] : make_int2(0, 0);
        else up = fromprev;
        if (rowok && j >= 0 && j < W) {
            const DChunk& b = sm.buf[(j >> 5) & 1];
            const int cj = j & 31;
            const unsigned cf = b.code[lane][cj];
            const int code = (int)(cf & 0x7Fu);
            const int2 raw = b.raw[lane][cj];
            int2 rec = raw;
            if (code > 0) {
                int pu, pv;
                if (cf & 0x80u) {
                    const int2 p = b.psl[lane][cj];
                    pu = p.x;
                    pv = p.y;
                } else {
                    const int2 n0 = b.qp[lane][cj], n1 = b.qp[lane][cj + 1];
                    const int2 n2 = b.qp[lane + 1][cj], n3 = b.qp[lane + 1][cj + 1];
                    pu = up.x + left.x + n3.x - upleft.x - n1.x - n2.x + n0.x;
                    pv = up.y + left.y + n3.y - upleft.y - n1.y - n2.y + n0.y;
                }
                const unsigned w = (2u << (code - 1)) + 1u;
                const uint32_t sy = b.sym[lane][cj];
                const unsigned su = sy & 0xFFFFu, sv = sy >> 16;
                if (su) rec.x = (int)((unsigned)pu + (su - (unsigned)kRadius) * w);
                if (sv) rec.y = (int)((unsigned)pv + (sv - (unsigned)kRadius) * w);
            }
            a.qhat[base + (size_t)i * W + j] = rec;
            res = rec;
        } else {
            res = make_int2(0, 0);
        }
        left = res;
        const int jl = k - 31;
        if (jl >= 0 && jl < W && ((jl % 16) == 15 || jl == W - 1)) warp_publish(prog_me, (unsigned)(jl + 1));
    }
    return true;
}

__global__ void __maxnreg__(192) decode_pipeline_kernel(DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DSmem& sm = *reinterpret_cast<DSmem*>(smem_raw);
    const int nstrips = (a.H + 31) / 32;
    const unsigned per_strip = (unsigned)a.prep_groups + 1u;
    const unsigned per_slice = (unsigned)nstrips * per_strip;
    const unsigned total = per_slice * (unsigned)a.T;
    for (;;) {
        unsigned item = 0;
        int stop = 0;
        if (threadIdx.x == 0) {
            item = atomicAdd(a.ticket, 1u);
            stop = *(volatile int*)a.status != 0;
        }
        item = __shfl_sync(0xffffffffu, item, 0);
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (item >= total || stop) return;
        const int t = (int)(item / per_slice);
        const unsigned r = item % per_slice;
        const int s = (int)(r / per_strip);
        const int g = (int)(r % per_strip);
        bool ok = true;
        if (g < a.prep_groups) {
            if (t >= 1)
                for (int c = g; c < a.nchunks && ok; c += a.prep_groups) ok = dprep_tile(a, t, s, c, sm);
        } else {
            ok = dwave_item(a, t, s, sm);
        }
        if (!ok) return;
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
                       size_t n_ld, size_t N, int2* raw, int* status, cudaStream_t s) {
    gather_raw_kernel<<<1216, 256, 0, s>>>(qxi, sym, off, ld, n_ld, N, raw, status);
}
void launch_to_float(const int2* qhat, size_t N, double inv_scale, float* out, cudaStream_t s) {
    to_float_kernel<<<1216, 256, 0, s>>>(qhat, N, inv_scale, reinterpret_cast<float2*>(out));
}

cudaError_t launch_decode_pipeline(const DecodeArgs& a, int nsm, cudaStream_t s) {
    const size_t smem = sizeof(DSmem);
    cudaError_t e = cudaFuncSetAttribute(decode_pipeline_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_pipeline_kernel, 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    DecodeArgs b = a;
    const int warps = nsm * per_sm;
    const int nstrips = (a.H + 31) / 32;
    if (a.pred == 0 || a.T < 2) {
        b.prep_groups = 0;
    } else {
        int pg = warps / (8 * nstrips) - 1;
        b.prep_groups = pg < 1 ? 1 : (pg > a.nchunks ? a.nchunks : pg);
    }
    decode_pipeline_kernel<<<warps, 32, smem, s>>>(b);
    return cudaGetLastError();
}

}  // namespace cpt
