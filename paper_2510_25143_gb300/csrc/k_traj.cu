// Critical-point trajectories (Sec. III-D, Thm. 2): crossed faces joined
// through the tetrahedra that contain two of them (Lemma 1: a tetrahedron has
// 0 or 2 crossed faces).  Kernels: compaction of the crossed faces in
// increasing id (owner vertex id * 12 + type), one thread per owner vertex
// over its six tetrahedra (Lemma 1 check, union-find hooking, adjacency), and
// the crossing point of each face (Eq. 3).
#include "cpt_dev.cuh"
#include "cpt_internal.h"

namespace cpt {

// Six tetrahedra owned by vertex A = (t,i,j) (t<T-1, i<H-1, j<W-1), as four
// faces each: (owner dt, di, dj, type).  The prism over triangle (A,R,G) is
// split into (A R G G'), (A R R' G'), (A A' R' G'); the prism over (A,D,G)
// into (A D G G'), (A D D' G'), (A A' D' G').
__device__ __constant__ const int8_t kTets[6][4][4] = {
    {{0, 0, 0, 0}, {0, 0, 0, 2}, {0, 0, 0, 10}, {0, 0, 1, 8}},
    {{0, 0, 0, 6}, {0, 0, 0, 2}, {0, 0, 0, 3}, {0, 0, 1, 9}},
    {{0, 0, 0, 7}, {0, 0, 0, 11}, {0, 0, 0, 3}, {1, 0, 0, 0}},
    {{0, 0, 0, 1}, {0, 0, 0, 4}, {0, 0, 0, 10}, {0, 1, 0, 6}},
    {{0, 0, 0, 8}, {0, 0, 0, 4}, {0, 0, 0, 5}, {0, 1, 0, 7}},
    {{0, 0, 0, 9}, {0, 0, 0, 11}, {0, 0, 0, 5}, {1, 0, 0, 1}},
};

// corner offsets (dt, di, dj) of the three vertices of each owned face type
__device__ __constant__ const int8_t kFaceCorner[12][3] = {
    {0, 1, 3}, {0, 2, 3}, {0, 1, 7}, {0, 5, 7}, {0, 2, 7}, {0, 6, 7},
    {0, 1, 5}, {0, 4, 5}, {0, 2, 6}, {0, 4, 6}, {0, 3, 7}, {0, 4, 7},
};

__global__ void __launch_bounds__(256) face_count_kernel(const uint16_t* __restrict__ mask, size_t N,
                                                         unsigned long long* __restrict__ cnt) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x)
        cnt[v] = (unsigned long long)__popc(mask[v]);
}

__global__ void __launch_bounds__(256) face_compact_kernel(const uint16_t* __restrict__ mask,
                                                           const unsigned long long* __restrict__ off, size_t N,
                                                           unsigned long long* __restrict__ fid) {
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N; v += (size_t)gridDim.x * blockDim.x) {
        unsigned m = mask[v];
        unsigned long long o = off[v];
        while (m) {
            const int ty = __ffs(m) - 1;
            m &= m - 1;
            fid[o++] = (unsigned long long)v * 12ull + (unsigned long long)ty;
        }
    }
}

// Parent links change under other thread blocks while the kernel runs: read
// them through L2 so that a failed hook always sees the new parent.
__device__ __forceinline__ unsigned uf_find(unsigned* par, unsigned x) {
    unsigned p = __ldcg(par + x);
    while (p != x) {
        const unsigned g = __ldcg(par + p);
        if (g != p) par[x] = g;  // path halving: g is an ancestor of x
        x = p;
        p = __ldcg(par + x);
    }
    return x;
}

__device__ __forceinline__ void uf_union(unsigned* par, unsigned a, unsigned b) {
    for (int it = 0; it < 1 << 20; ++it) {  // bounded: each retry follows a successful hook elsewhere
        a = uf_find(par, a);
        b = uf_find(par, b);
        if (a == b) return;
        if (a < b) { const unsigned t = a; a = b; b = t; }
        // hook the larger root under the smaller one
        if (atomicCAS(&par[a], a, b) == a) return;
    }
}

// One thread per owner vertex: its six tetrahedra.  idx(face) = off[owner] +
// number of crossed lower types of the owner.
__global__ void __launch_bounds__(256) tet_link_kernel(const uint16_t* __restrict__ mask,
                                                       const unsigned long long* __restrict__ off, int H, int W, int T,
                                                       unsigned* __restrict__ par, unsigned* __restrict__ deg,
                                                       unsigned* __restrict__ adj,
                                                       unsigned long long* __restrict__ bad) {
    const int j = blockIdx.x * 32 + (threadIdx.x & 31);
    const int i = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int t = blockIdx.z;
    unsigned nbad = 0;
    if (i + 1 < H && j + 1 < W && t + 1 < T) {
        for (int k = 0; k < 6; ++k) {
            unsigned hit[4];
            int nh = 0;
            for (int f = 0; f < 4; ++f) {
                const size_t ow = ((size_t)(t + kTets[k][f][0]) * H + (i + kTets[k][f][1])) * W + (j + kTets[k][f][2]);
                const int ty = kTets[k][f][3];
                const unsigned m = mask[ow];
                if ((m >> ty) & 1u) hit[nh++] = (unsigned)off[ow] + __popc(m & ((1u << ty) - 1u));
            }
            if (nh == 0) continue;
            if (nh != 2) { ++nbad; continue; }
            uf_union(par, hit[0], hit[1]);
            const unsigned s0 = atomicAdd(&deg[hit[0]], 1u), s1 = atomicAdd(&deg[hit[1]], 1u);
            if (s0 < 2) adj[2 * hit[0] + s0] = hit[1];
            if (s1 < 2) adj[2 * hit[1] + s1] = hit[0];
            if (s0 >= 2 || s1 >= 2) ++nbad;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nbad += __shfl_xor_sync(0xffffffffu, nbad, o);
    if ((threadIdx.x & 31) == 0 && nbad) atomicAdd(bad, (unsigned long long)nbad);
}

__global__ void __launch_bounds__(256) uf_flatten_kernel(unsigned* __restrict__ par, size_t n) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x)
        par[x] = uf_find(par, (unsigned)x);
}

// Crossing point of a crossed face (Eq. 3): barycentric weights
// (det(b,c), det(c,a), det(a,b)) / D_f over its vertices (a,b,c by id) applied
// to their (x = column, y = row, t); D_f = 0 gives the centroid.
__global__ void __launch_bounds__(256) crossing_point_kernel(const int2* __restrict__ q,
                                                             const unsigned long long* __restrict__ fid, size_t n,
                                                             int H, int W, double* __restrict__ xyt) {
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x) {
        const unsigned long long f = fid[x];
        const size_t owner = (size_t)(f / 12ull);
        const int ty = (int)(f % 12ull);
        const int j = (int)(owner % W), i = (int)((owner / W) % H), t = (int)(owner / ((size_t)W * H));
        int2 p[3];
        int ci[3], cj[3], ct[3];
        for (int k = 0; k < 3; ++k) {
            const int c = kFaceCorner[ty][k];
            cj[k] = j + (c & 1);
            ci[k] = i + ((c >> 1) & 1);
            ct[k] = t + ((c >> 2) & 1);
            p[k] = q[((size_t)ct[k] * H + ci[k]) * W + cj[k]];
        }
        const long long dbc = (long long)p[1].x * p[2].y - (long long)p[1].y * p[2].x;
        const long long dca = (long long)p[2].x * p[0].y - (long long)p[2].y * p[0].x;
        const long long dab = (long long)p[0].x * p[1].y - (long long)p[0].y * p[1].x;
        const long long D = dbc + dca + dab;
        double w[3];
        if (D == 0) {
            w[0] = w[1] = w[2] = __ddiv_rn(1.0, 3.0);
        } else {
            w[0] = __ddiv_rn((double)dbc, (double)D);
            w[1] = __ddiv_rn((double)dca, (double)D);
            w[2] = __ddiv_rn((double)dab, (double)D);
        }
        double px = 0.0, py = 0.0, pt = 0.0;
        for (int k = 0; k < 3; ++k) {
            px = __dadd_rn(px, __dmul_rn(w[k], (double)cj[k]));
            py = __dadd_rn(py, __dmul_rn(w[k], (double)ci[k]));
            pt = __dadd_rn(pt, __dmul_rn(w[k], (double)ct[k]));
        }
        xyt[3 * x] = px;
        xyt[3 * x + 1] = py;
        xyt[3 * x + 2] = pt;
    }
}

__global__ void __launch_bounds__(256) iota_kernel(unsigned* __restrict__ x, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        x[k] = (unsigned)k;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
void launch_iota(unsigned* x, size_t n, cudaStream_t s) {
    if (n) iota_kernel<<<1216, 256, 0, s>>>(x, n);
}
void launch_face_count(const uint16_t* mask, size_t N, unsigned long long* cnt, cudaStream_t s) {
    face_count_kernel<<<1216, 256, 0, s>>>(mask, N, cnt);
}
void launch_face_compact(const uint16_t* mask, const unsigned long long* off, size_t N, unsigned long long* fid,
                         cudaStream_t s) {
    face_compact_kernel<<<1216, 256, 0, s>>>(mask, off, N, fid);
}
void launch_tet_link(const uint16_t* mask, const unsigned long long* off, int H, int W, int T, unsigned* par,
                     unsigned* deg, unsigned* adj, unsigned long long* bad, cudaStream_t s) {
    dim3 grid((W + 31) / 32, (H + 7) / 8, T);
    tet_link_kernel<<<grid, 256, 0, s>>>(mask, off, H, W, T, par, deg, adj, bad);
}
void launch_uf_flatten(unsigned* par, size_t n, cudaStream_t s) {
    if (n) uf_flatten_kernel<<<1216, 256, 0, s>>>(par, n);
}
void launch_crossing_points(const int32_t* q, const unsigned long long* fid, size_t n, int H, int W, double* xyt,
                            cudaStream_t s) {
    if (n) crossing_point_kernel<<<1216, 256, 0, s>>>(reinterpret_cast<const int2*>(q), fid, n, H, W, xyt);
}

}  // namespace cpt
