// Rate diagnostics (the distribution of quantisation codes behind the
// compression ratios of Sec. VII-E): the lengths of the maximal runs of the
// zero code in the Q_d stream, binned by length.
//
// A warp scans a chunk of kRunChunk symbols one 32-symbol word at a time and
// bins every run that starts and ends inside the chunk; the zeros before the
// chunk's first non-zero symbol (head) and after its last (tail) are left to
// a serial pass over the chunks, which joins runs across chunk boundaries.
#include <algorithm>

#include "cpt_dev.cuh"
#include "cpt_internal.h"

namespace cpt {

constexpr int kRunChunk = 65536;  // symbols per warp chunk
constexpr int kRunWarps = 4;      // warps per block

struct RunEdge {
    unsigned long long head;  // zeros before the first non-zero symbol (the whole chunk when all)
    unsigned long long tail;  // zeros after the last non-zero symbol
    unsigned all;             // 1: the chunk holds only zeros
    unsigned pad;
};

template <class Add>
__device__ __forceinline__ void bin_run(unsigned long long* bins, unsigned long long len, Add add) {
    if (len <= (unsigned long long)kRunMax) {
        add(&bins[len], 1ull);
    } else {
        add(&bins[kRunMax + 1], 1ull);
        add(&bins[0], len);
    }
}

__global__ void __launch_bounds__(32 * kRunWarps) zero_runs_kernel(const uint16_t* __restrict__ qd, size_t n,
                                                                  unsigned zs, size_t nchunks,
                                                                  unsigned long long* __restrict__ bins,
                                                                  RunEdge* __restrict__ edges) {
    __shared__ unsigned long long sb[kRunBins];
    for (int k = threadIdx.x; k < kRunBins; k += blockDim.x) sb[k] = 0;
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = (int)(threadIdx.x & 31u);
    auto sadd = [](unsigned long long* p, unsigned long long v) { atomicAdd(p, v); };
    for (size_t c = (size_t)blockIdx.x * kRunWarps + (threadIdx.x >> 5); c < nchunks;
         c += (size_t)gridDim.x * kRunWarps) {
        const size_t base = c * kRunChunk;
        const size_t len = min((size_t)kRunChunk, n - base);
        unsigned long long run = 0, head = 0;  // lane-uniform
        bool head_open = true;                 // no non-zero symbol seen yet in the chunk
        for (size_t off = 0; off < len; off += 32) {
            const int nv = (int)min((size_t)32, len - off);  // valid lanes of this word
            const bool valid = lane < nv;
            const bool z = valid && __ldg(qd + base + off + lane) == (uint16_t)zs;
            const unsigned m = __ballot_sync(FULL, z);
            const unsigned vm = nv == 32 ? FULL : ((1u << nv) - 1u);
            const unsigned nz = ~m & vm;  // non-zero symbols of the word
            if (nz == 0) {
                run += (unsigned)nv;
                continue;
            }
            const int first = __ffs(nz) - 1, last = 31 - __clz(nz);
            // the open run plus the zeros before the word's first non-zero symbol
            const unsigned long long tot = run + (unsigned)first;
            if (head_open) {
                head = tot;
                head_open = false;
            } else if (tot > 0 && lane == 0) {
                bin_run(sb, tot, sadd);
            }
            // runs between two non-zero symbols of the word: each ends at a
            // zero lane whose next lane is non-zero
            if (z && lane > first && lane + 1 < nv && ((nz >> (lane + 1)) & 1u)) {
                const unsigned k = __clz(~(m << (31 - lane)));  // consecutive zeros ending at this lane
                bin_run(sb, k, sadd);
            }
            run = (unsigned)(nv - 1 - last);
        }
        if (lane == 0) {
            RunEdge e;
            e.all = head_open ? 1u : 0u;
            e.head = head_open ? run : head;
            e.tail = head_open ? 0ull : run;
            e.pad = 0;
            edges[c] = e;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kRunBins; k += blockDim.x)
        if (sb[k]) atomicAdd(&bins[k], sb[k]);
}

// Joins the chunks' edges in order: a run crossing chunk boundaries is the
// tail of one chunk, whole zero chunks and the head of the next.
__global__ void zero_runs_merge_kernel(const RunEdge* __restrict__ edges, size_t nchunks,
                                       unsigned long long* __restrict__ bins) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    auto gadd = [](unsigned long long* p, unsigned long long v) { *p += v; };
    unsigned long long run = 0;
    for (size_t c = 0; c < nchunks; ++c) {
        const RunEdge e = edges[c];
        if (e.all) {
            run += e.head;
            continue;
        }
        const unsigned long long tot = run + e.head;
        if (tot > 0) bin_run(bins, tot, gadd);
        run = e.tail;
    }
    if (run > 0) bin_run(bins, run, gadd);
}

size_t zero_runs_ws_bytes(size_t n) { return sizeof(RunEdge) * ((n + kRunChunk - 1) / kRunChunk + 1); }

cudaError_t launch_zero_runs(const uint16_t* qd, size_t n, unsigned zero_sym, unsigned long long* bins, void* ws,
                             int nsm, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(unsigned long long) * kRunBins, s);
    if (e != cudaSuccess || n == 0) return e;
    const size_t nchunks = (n + kRunChunk - 1) / kRunChunk;
    RunEdge* edges = static_cast<RunEdge*>(ws);
    const size_t want = (nchunks + kRunWarps - 1) / kRunWarps;
    const int blocks = (int)std::min(want, (size_t)nsm * 8);
    zero_runs_kernel<<<blocks, 32 * kRunWarps, 0, s>>>(qd, n, zero_sym, nchunks, bins, edges);
    zero_runs_merge_kernel<<<1, 32, 0, s>>>(edges, nchunks, bins);
    return cudaGetLastError();
}

}  // namespace cpt
