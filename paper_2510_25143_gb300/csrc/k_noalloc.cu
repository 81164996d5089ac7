// Allocation-free fixed-point conversion.
//
// Some callers cannot allocate device memory at the point where they need
// this step: code running inside a memory budget that was fully reserved up
// front (a serving process that pre-allocates its pool at start-up), code
// called from a context where cudaMalloc would synchronise the device and
// stall other work, or embedders whose allocator forbids foreign
// allocations.  cpt_fixed_point_noalloc gives them the range reduction and
// the float -> fixed-point conversion that cpt_compress starts with, writing
// only into buffers the caller passes in.  The range reduction's per-block
// partial results live in a file-scope device array instead of scratch
// obtained from cudaMallocAsync.
//
// Limits and rules of use:
//   * the scratch array holds kNoAllocMaxBlocks partials; each block reduces
//     kNoAllocPerBlock values, so at most kNoAllocMaxBlocks * kNoAllocPerBlock
//     float values (2*H*W*T) are accepted; larger inputs get CPT_ERR_ARG;
//   * every GPU that loads the library keeps this array (256 KiB) until the
//     process exits;
//   * all calls share the one array, which keeps the last call's contents:
//     two calls whose kernels overlap on the GPU (different streams, or
//     different host threads) race on it and must be serialised by the
//     caller;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before capturing any stream into a CUDA graph.  The address is kept
//     together with the CUDA context it belongs to: after cudaDeviceReset or
//     any other teardown of the context, the module (and the array) may be
//     loaded at another address, so a call in a new context looks it up
//     again (once more, with the same advice about graph capture);
//   * an error already pending on the calling thread (cudaPeekAtLastError)
//     is not cleared: the call returns CPT_ERR_CUDA without launching, and
//     the caller's own error check still sees it.
#include <cuda.h>

#include <mutex>

#include "cpt.h"
#include "cpt_internal.h"

namespace cpt {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocVec = 16;                                     // float4 per thread
constexpr size_t kNoAllocPerBlock = (size_t)kNoAllocThreads * kNoAllocVec * 4;  // 16384 floats
constexpr int kNoAllocMaxBlocks = 16384;

// Per-block (min, max, max|x|, non-finite flag): 16 B x 16384 = 256 KiB.
static __device__ __align__(256) RangePartial g_noalloc_partials[kNoAllocMaxBlocks];

// One block per kNoAllocPerBlock values (no grid-stride loop), so the number
// of partials grows with the input and is checked against the array size.
__global__ void __launch_bounds__(kNoAllocThreads) noalloc_range_kernel(const float4* __restrict__ uv, size_t n4,
                                                                        const float* __restrict__ tail, int ntail,
                                                                        RangePartial* __restrict__ part) {
    float mn = INFINITY, mx = -INFINITY, am = 0.f;
    unsigned bad = 0;
    if (blockIdx.x == 0 && (int)threadIdx.x < ntail) {
        const float x = tail[threadIdx.x];
        bad |= !isfinite(x);
        mn = x;
        mx = x;
        am = fabsf(x);
    }
    const size_t base = (size_t)blockIdx.x * (kNoAllocPerBlock / 4);
#pragma unroll 4
    for (int k = 0; k < kNoAllocVec; ++k) {
        size_t idx = base + (size_t)k * kNoAllocThreads + threadIdx.x;
        if (idx < n4) {
            float4 a = __ldcs(uv + idx);
            float x[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                bad |= !isfinite(x[e]);
                mn = fminf(mn, x[e]);
                mx = fmaxf(mx, x[e]);
                am = fmaxf(am, fabsf(x[e]));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ RangePartial sp[kNoAllocThreads / 32];
    if ((threadIdx.x & 31) == 0) sp[threadIdx.x >> 5] = RangePartial{mn, mx, am, bad};
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kNoAllocThreads / 32; ++w) {
            mn = fminf(mn, sp[w].mn); mx = fmaxf(mx, sp[w].mx); am = fmaxf(am, sp[w].amax); bad |= sp[w].bad;
        }
        part[blockIdx.x] = RangePartial{mn, mx, am, bad};
    }
}

// Reduces the partials and writes k = 23 - e with max|x| < 2^e (0 for an
// all-zero field), or INT32_MIN when a value is not finite.
__global__ void __launch_bounds__(256) noalloc_scale_kernel(const RangePartial* __restrict__ part, int nparts,
                                                            int32_t* __restrict__ k_out) {
    float am = 0.f;
    unsigned bad = 0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        am = fmaxf(am, part[b].amax);
        bad |= part[b].bad;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ float sam[8];
    __shared__ unsigned sbad[8];
    if ((threadIdx.x & 31) == 0) { sam[threadIdx.x >> 5] = am; sbad[threadIdx.x >> 5] = bad; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { am = fmaxf(am, sam[w]); bad |= sbad[w]; }
        int k = 0;
        if (bad) {
            k = INT32_MIN;
        } else if (am > 0.f) {
            int e;
            frexp((double)am, &e);
            k = 23 - e;
        }
        *k_out = k;
    }
}

// q = rint(x * 2^k), k read from device memory (skipped when k is INT32_MIN).
__global__ void __launch_bounds__(256) noalloc_fixed_kernel(const float4* __restrict__ uv, size_t n4,
                                                            const float* __restrict__ tail, int ntail,
                                                            const int32_t* __restrict__ k_in, int4* __restrict__ q,
                                                            int32_t* __restrict__ qtail) {
    const int k = *k_in;
    if (k == INT32_MIN) return;
    const double scale = ldexp(1.0, k);
    if (blockIdx.x == 0 && (int)threadIdx.x < ntail) qtail[threadIdx.x] = __double2int_rn((double)tail[threadIdx.x] * scale);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
        float4 a = __ldcs(uv + i);
        q[i] = make_int4(__double2int_rn((double)a.x * scale), __double2int_rn((double)a.y * scale),
                         __double2int_rn((double)a.z * scale), __double2int_rn((double)a.w * scale));
    }
}

// The current CUDA context, through the driver's cuCtxGetCurrent (found via
// the runtime, so the library needs no link against libcuda).
static bool current_context(CUcontext* ctx) {
    using GetCurrent = CUresult (*)(CUcontext*);
    static GetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<GetCurrent>(f);
    }();
    *ctx = nullptr;
    return fn && fn(ctx) == CUDA_SUCCESS && *ctx;
}

// Device address of g_noalloc_partials, looked up once per device and
// context (a context created after a reset may load the module elsewhere).
static RangePartial* noalloc_scratch(int dev, cudaError_t* err) {
    static std::mutex mu;
    static RangePartial* addr[64] = {nullptr};
    static CUcontext owner[64] = {nullptr};
    *err = cudaSuccess;
    if (dev < 0 || dev >= 64) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    // no context may be current yet before the runtime's first use of the
    // device; the lookup below then creates the primary context
    CUcontext ctx = nullptr;
    current_context(&ctx);
    std::lock_guard<std::mutex> lock(mu);
    if (ctx && addr[dev] && owner[dev] == ctx) return addr[dev];
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !current_context(&ctx)) {
        *err = e != cudaSuccess ? e : cudaErrorDeviceUninitialized;
        addr[dev] = nullptr;
        owner[dev] = nullptr;
        return nullptr;
    }
    addr[dev] = static_cast<RangePartial*>(p);
    owner[dev] = ctx;
    return addr[dev];
}

}  // namespace cpt

extern "C" cpt_status cpt_fixed_point_noalloc(const float* uv, const cpt_dims* dims, int32_t* q, int32_t* scale_log2,
                                              void* cuda_stream) {
    using namespace cpt;
    constexpr size_t kMaxValues = (size_t)kNoAllocMaxBlocks * kNoAllocPerBlock;  // 2^28 floats
    if (!uv || !dims || !q || !scale_log2) return CPT_ERR_ARG;
    if (dims->H < 1 || dims->W < 1 || dims->T < 1) return CPT_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(uv) | reinterpret_cast<uintptr_t>(q)) & 15u) return CPT_ERR_ARG;
    // 2*H*W*T without wrap-around: every factor and partial product is checked
    // against the limit before the next multiplication
    const size_t H = (size_t)dims->H, W = (size_t)dims->W, T = (size_t)dims->T;
    if (H > kMaxValues || W > kMaxValues || T > kMaxValues) return CPT_ERR_ARG;
    if (H * W > kMaxValues) return CPT_ERR_ARG;
    if (H * W * T > kMaxValues / 2) return CPT_ERR_ARG;
    const size_t nvals = 2 * H * W * T;
    const size_t nblocks = (nvals + kNoAllocPerBlock - 1) / kNoAllocPerBlock;
    if (nblocks > (size_t)kNoAllocMaxBlocks) return CPT_ERR_ARG;  // beyond the scratch array
    // an error left pending by earlier work stays the caller's to see
    if (cudaPeekAtLastError() != cudaSuccess) return CPT_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CPT_ERR_CUDA;
    cudaError_t e;
    RangePartial* part = noalloc_scratch(dev, &e);
    if (!part) return CPT_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const size_t n4 = nvals / 4;            // whole float4 groups
    const int ntail = (int)(nvals - 4 * n4);  // 0 or 2 trailing values
    // stop at the first launch that fails: a later kernel would read partials
    // the failed one never wrote
    noalloc_range_kernel<<<(unsigned)nblocks, kNoAllocThreads, 0, s>>>(reinterpret_cast<const float4*>(uv), n4,
                                                                      uv + 4 * n4, ntail, part);
    if (cudaGetLastError() != cudaSuccess) return CPT_ERR_CUDA;
    noalloc_scale_kernel<<<1, 256, 0, s>>>(part, (int)nblocks, scale_log2);
    if (cudaGetLastError() != cudaSuccess) return CPT_ERR_CUDA;
    noalloc_fixed_kernel<<<1216, 256, 0, s>>>(reinterpret_cast<const float4*>(uv), n4, uv + 4 * n4, ntail, scale_log2,
                                              reinterpret_cast<int4*>(q), q + 4 * n4);
    if (cudaGetLastError() != cudaSuccess) return CPT_ERR_CUDA;
    return CPT_OK;
}
