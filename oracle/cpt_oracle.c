/*
 * CPU oracle for the critical-point-trajectory-preserving compressor of
 * "Time-Varying Vector Field Compression with Preserved Critical Point
 * Trajectories" (Xia, Li, Jiao, Wang, Liang, Guo).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded
 * restatement of the method, written step by step in the paper's order.  It is
 * used by the test-suite, by the smoke check and by the CPU-baseline leg of the
 * benchmark; no product code path may link, load or call it.  It shares no code
 * with the CUDA library: every table, helper and format routine below is
 * written here a second time from the same specification.
 *
 * Readings taken where the paper is silent (each is listed with the reason in
 * the design notes of the repository):
 *   R1  fixed point: S = 2^k, k = 23 - e, max|x| < 2^e (frexp); q = rint(x*S).
 *   R2  eps (absolute data units; relative: eb * (max - min) over u and v);
 *       eps' = floor(eps*S - 0.5), clamped to [0, 2^23].
 *   R3  SoS: every vertex value is perturbed symbolically by its global id, the
 *       origin is exact; predicate = the three 2x2 SoS signs agree.
 *   R4  quads split along the main diagonal (i,j)-(i+1,j+1); a<b<c by id.
 *   R5  Alg. 2 evaluated exactly in integers with strict bounds.
 *   R6  xi_q = 2^floor(log2 xi), code floor(log2 xi)+1, code 0 = lossless.
 *   R7  w = 2 xi_q + 1, c = floor((r + xi_q)/w), |c| < 32768 else unpredictable.
 *   R8  3-D Lorenzo with out-of-domain terms 0.
 *   R9  semi-Lagrangian: x (column) moves by u*CFL_x, y (row) by v*CFL_y; FP64
 *       with a fixed evaluation order and no contraction; floor(p + 0.5).
 *   R11 MoP: B = 16, stride n = 2, integer log2 (repeated squaring), switch
 *       iff 1000*R_SL < 997*R_3DL.
 *   R12 stream v1, canonical length-limited (24-bit) Huffman by package-merge.
 *   R13 trajectories = connected components of crossed faces joined by tets.
 *   L1  learned predictor (not in the paper; predictor 3): a 3-layer 3x3 conv
 *       net, bfloat16 weights, float32 fused multiply-add chains in a fixed
 *       order, prediction = qhat(t-1) + rint(clamp(y, -2, 2) * 2^23).
 *
 * The paper fixes no byte layout for the stream; R12 is this project's.  The
 * tests pin the writer to R12's description with a decoder written from it
 * alone, besides the round trip, the invariants and the optimality of the
 * Huffman code lengths.  Every step has a pin of its own.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math, no FMA).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_OK 0
#define O_ERR_ARG -1
#define O_ERR_OOM -3
#define O_ERR_CORRUPT -4

#define QRADIUS 32768
#define HUFF_MAXLEN 24
#define HUFF_CHUNK 16384u

typedef int64_t i64;
typedef uint64_t u64;

/* ------------------------------------------------------------------------ */
/* Mesh: space-time extrusion and the three-tetrahedron split (Sec. III-C).   */
/* Face types owned by vertex (t,i,j); spatial corners A=(i,j), R=(i,j+1),    */
/* D=(i+1,j), G=(i+1,j+1).  Triangles (A,R,G) and (A,D,G) (main diagonal).    */
/* For a triangle a<b<c the prism [t,t+1] is split into                        */
/*   tau1=(a_t,b_t,c_t,c_t+1) tau2=(a_t,b_t,b_t+1,c_t+1) tau3=(a_t,a_t+1,b_t+1,c_t+1) */
/* whose faces are the slice triangles, two interior faces per prism and two  */
/* faces per vertical quad (diagonal from the lower-id vertex at t to the      */
/* higher-id vertex at t+1).  Each face lists its vertices by increasing id.   */
/* ------------------------------------------------------------------------ */
static const int O_FACE[12][3][3] = {
    /* 0: slice triangle (A,R,G) at t */ {{0, 0, 0}, {0, 0, 1}, {0, 1, 1}},
    /* 1: slice triangle (A,D,G) at t */ {{0, 0, 0}, {0, 1, 0}, {0, 1, 1}},
    /* 2: (A_t, R_t, G_t+1)          */ {{0, 0, 0}, {0, 0, 1}, {1, 1, 1}},
    /* 3: (A_t, R_t+1, G_t+1)        */ {{0, 0, 0}, {1, 0, 1}, {1, 1, 1}},
    /* 4: (A_t, D_t, G_t+1)          */ {{0, 0, 0}, {0, 1, 0}, {1, 1, 1}},
    /* 5: (A_t, D_t+1, G_t+1)        */ {{0, 0, 0}, {1, 1, 0}, {1, 1, 1}},
    /* 6: edge A-R (A_t, R_t, R_t+1) */ {{0, 0, 0}, {0, 0, 1}, {1, 0, 1}},
    /* 7: edge A-R (A_t, A_t+1, R_t+1)*/ {{0, 0, 0}, {1, 0, 0}, {1, 0, 1}},
    /* 8: edge A-D (A_t, D_t, D_t+1) */ {{0, 0, 0}, {0, 1, 0}, {1, 1, 0}},
    /* 9: edge A-D (A_t, A_t+1, D_t+1)*/ {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}},
    /* 10: edge A-G (A_t, G_t, G_t+1)*/ {{0, 0, 0}, {0, 1, 1}, {1, 1, 1}},
    /* 11: edge A-G (A_t, A_t+1, G_t+1)*/ {{0, 0, 0}, {1, 0, 0}, {1, 1, 1}},
};

/* The six tetrahedra owned by vertex (t,i,j) for t<T-1, i<H-1, j<W-1, each as
 * four faces (owner offset dt,di,dj ; face type).  Derived from the split of
 * the two prisms over triangles (A,R,G) and (A,D,G). */
static const int O_TET[6][4][4] = {
    /* (A,R,G) tau1 = A_t R_t G_t G_t+1 */
    {{0, 0, 0, 0}, {0, 0, 0, 2}, {0, 0, 0, 10}, {0, 0, 1, 8}},
    /* (A,R,G) tau2 = A_t R_t R_t+1 G_t+1 */
    {{0, 0, 0, 6}, {0, 0, 0, 2}, {0, 0, 0, 3}, {0, 0, 1, 9}},
    /* (A,R,G) tau3 = A_t A_t+1 R_t+1 G_t+1 */
    {{0, 0, 0, 7}, {0, 0, 0, 11}, {0, 0, 0, 3}, {1, 0, 0, 0}},
    /* (A,D,G) tau1 = A_t D_t G_t G_t+1 */
    {{0, 0, 0, 1}, {0, 0, 0, 4}, {0, 0, 0, 10}, {0, 1, 0, 6}},
    /* (A,D,G) tau2 = A_t D_t D_t+1 G_t+1 */
    {{0, 0, 0, 8}, {0, 0, 0, 4}, {0, 0, 0, 5}, {0, 1, 0, 7}},
    /* (A,D,G) tau3 = A_t A_t+1 D_t+1 G_t+1 */
    {{0, 0, 0, 9}, {0, 0, 0, 11}, {0, 0, 0, 5}, {1, 0, 0, 1}},
};

static inline i64 vid(int H, int W, int t, int i, int j) {
    return ((i64)t * H + i) * W + j;
}

static int face_valid(int H, int W, int T, int t, int i, int j, int type) {
    if (t < 0 || i < 0 || j < 0) return 0;
    for (int k = 0; k < 3; ++k) {
        int tt = t + O_FACE[type][k][0], ii = i + O_FACE[type][k][1], jj = j + O_FACE[type][k][2];
        if (tt >= T || ii >= H || jj >= W) return 0;
    }
    return 1;
}

/* Number of faces of the mesh that contain vertex (t,i,j) (Alg. 4 iterates
 * over these; at most 36 for an interior vertex, Sec. V-B). */
int o_incident_face_count(int H, int W, int T, int t, int i, int j) {
    int n = 0;
    for (int type = 0; type < 12; ++type)
        for (int k = 0; k < 3; ++k) {
            int ot = t - O_FACE[type][k][0], oi = i - O_FACE[type][k][1], oj = j - O_FACE[type][k][2];
            n += face_valid(H, W, T, ot, oi, oj, type);
        }
    return n;
}

i64 o_face_count(int H, int W, int T) {
    i64 n = 0;
    for (int t = 0; t < T; ++t)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j)
                for (int type = 0; type < 12; ++type) n += face_valid(H, W, T, t, i, j, type);
    return n;
}

/* Copies the face and tetrahedron tables (for tests that rebuild the mesh
 * from the paper's definition and compare). */
void o_face_table(int* out /* 12*3*3 */) { memcpy(out, O_FACE, sizeof(O_FACE)); }
void o_tet_table(int* out /* 6*4*4 */) { memcpy(out, O_TET, sizeof(O_TET)); }

/* ------------------------------------------------------------------------ */
/* Fixed point (Alg. 3 Convert_FixedPoint; reading R1) and eps' (R2).         */
/* ------------------------------------------------------------------------ */
int o_range(const float* uv, i64 nvals, double* vmin, double* vmax, double* amax) {
    double mn = 0, mx = 0, am = 0;
    for (i64 n = 0; n < nvals; ++n) {
        double x = uv[n];
        if (!isfinite(x)) return O_ERR_ARG;
        if (n == 0 || x < mn) mn = x;
        if (n == 0 || x > mx) mx = x;
        if (fabs(x) > am) am = fabs(x);
    }
    *vmin = mn;
    *vmax = mx;
    *amax = am;
    return O_OK;
}

int o_scale_exponent(double amax) {
    if (amax == 0.0) return 0;
    int e;
    frexp(amax, &e); /* amax = m 2^e, m in [0.5,1): amax < 2^e */
    return 23 - e;
}

void o_to_fixed(const float* uv, i64 nvals, int k, int32_t* q) {
    for (i64 n = 0; n < nvals; ++n) q[n] = (int32_t)rint(ldexp((double)uv[n], k));
}

int32_t o_eps_int(double eps, int k) {
    double e = floor(ldexp(eps, k) - 0.5);
    if (!(e > 0)) return 0;
    if (e > 8388608.0) e = 8388608.0;
    return (int32_t)e;
}

/* ------------------------------------------------------------------------ */
/* Simulation of Simplicity (Sec. III-F, Alg. 1; reading R3).                 */
/* Vertex of global rank r carries (u,v) + (eps^(2^(2r-1)), eps^(2^(2r-2))).  */
/* The sign of det(a,b) for rank(a) < rank(b) is the sign of the first nonzero */
/* entry of  [a.u b.v - a.v b.u,  -b.u,  b.v,  a.u,  1].                       */
/* ------------------------------------------------------------------------ */
int o_sos_det2(i64 au, i64 av, i64 bu, i64 bv) {
    i64 d = au * bv - av * bu;
    if (d != 0) return d > 0 ? 1 : -1;
    if (bu != 0) return bu > 0 ? -1 : 1;
    if (bv != 0) return bv > 0 ? 1 : -1;
    if (au != 0) return au > 0 ? 1 : -1;
    return 1;
}

/* Face predicate (Eq. 2 under SoS): the origin lies inside the perturbed
 * triangle iff det(p1,p2), det(p2,p0), det(p0,p1) have one sign.  p0,p1,p2 are
 * given in increasing global id; det(p2,p0) = -det(p0,p2). */
int o_face_crossed(const i64* p /* u0 v0 u1 v1 u2 v2 */) {
    int s12 = o_sos_det2(p[2], p[3], p[4], p[5]);
    int s20 = -o_sos_det2(p[0], p[1], p[4], p[5]);
    int s01 = o_sos_det2(p[0], p[1], p[2], p[3]);
    return (s12 == s20) && (s20 == s01);
}

void o_face_crossed_batch(const i64* p, i64 n, uint8_t* out) {
    for (i64 k = 0; k < n; ++k) out[k] = (uint8_t)o_face_crossed(p + 6 * k);
}

static void face_values(const int32_t* q, int H, int W, int t, int i, int j, int type, i64* p) {
    for (int k = 0; k < 3; ++k) {
        i64 v = vid(H, W, t + O_FACE[type][k][0], i + O_FACE[type][k][1], j + O_FACE[type][k][2]);
        p[2 * k] = q[2 * v];
        p[2 * k + 1] = q[2 * v + 1];
    }
}

/* The crossed-face set C of Alg. 3, as a 12-bit mask per owner vertex. */
void o_face_masks(const int32_t* q, int H, int W, int T, uint16_t* mask) {
    i64 p[6];
    for (int t = 0; t < T; ++t)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                uint16_t m = 0;
                for (int type = 0; type < 12; ++type) {
                    if (!face_valid(H, W, T, t, i, j, type)) continue;
                    face_values(q, H, W, t, i, j, type, p);
                    if (o_face_crossed(p)) m |= (uint16_t)(1u << type);
                }
                mask[vid(H, W, t, i, j)] = m;
            }
}

/* ------------------------------------------------------------------------ */
/* Alg. 2 (error bound that keeps a triangle free of critical points when the */
/* third vertex (u2,v2) moves), evaluated exactly in integers (reading R5).    */
/* A ratio num/den becomes the largest integer e with e < num/den.            */
/* ------------------------------------------------------------------------ */
static inline i64 iabs64(i64 x) { return x < 0 ? -x : x; }
static inline i64 strict_ratio(i64 num, i64 den) { return num > 0 ? (num - 1) / den : 0; }
static inline int same_sign(i64 a, i64 b, i64 c) {
    return (a > 0 && b > 0 && c > 0) || (a < 0 && b < 0 && c < 0);
}

i64 o_alg2(i64 u0, i64 v0, i64 u1, i64 v1, i64 u2, i64 v2) {
    i64 M0 = u2 * v0 - u0 * v2;
    i64 M1 = u1 * v2 - u2 * v1;
    i64 M2 = u0 * v1 - u1 * v0;
    i64 M = M0 + M1 + M2;
    if (M == 0) return 0;
    i64 eb = strict_ratio(iabs64(M), iabs64(u1 - u0) + iabs64(v0 - v1));
    if (iabs64(u1) + iabs64(v1) != 0) {
        i64 e = strict_ratio(iabs64(M1), iabs64(u1) + iabs64(v1));
        if (e < eb) eb = e;
    } else {
        return 0;
    }
    if (iabs64(u0) + iabs64(v0) != 0) {
        i64 e = strict_ratio(iabs64(M0), iabs64(u0) + iabs64(v0));
        if (e < eb) eb = e;
    } else {
        return 0;
    }
    if (same_sign(u0, u1, u2) && iabs64(u2) - 1 > eb) eb = iabs64(u2) - 1;
    if (same_sign(v0, v1, v2) && iabs64(v2) - 1 > eb) eb = iabs64(v2) - 1;
    return eb;
}

/* Alg. 4: minimum bound over the faces containing v, with the current values
 * in Q (already-processed vertices hold their reconstruction).  Returns 0 when
 * an incident face is in C (the vertex is then stored losslessly). */
static i64 derive_min_eb(const int32_t* Q, const uint16_t* mask, int H, int W, int T, int t, int i,
                         int j, i64 eps_int, int* crossed) {
    i64 xi = eps_int;
    *crossed = 0;
    i64 self = vid(H, W, t, i, j);
    for (int type = 0; type < 12; ++type)
        for (int k = 0; k < 3; ++k) {
            int ot = t - O_FACE[type][k][0], oi = i - O_FACE[type][k][1], oj = j - O_FACE[type][k][2];
            if (!face_valid(H, W, T, ot, oi, oj, type)) continue;
            if (mask[vid(H, W, ot, oi, oj)] & (1u << type)) {
                *crossed = 1;
                return 0;
            }
            i64 nb[4];
            int m = 0;
            for (int kk = 0; kk < 3; ++kk) {
                if (kk == k) continue;
                i64 w = vid(H, W, ot + O_FACE[type][kk][0], oi + O_FACE[type][kk][1], oj + O_FACE[type][kk][2]);
                nb[m++] = Q[2 * w];
                nb[m++] = Q[2 * w + 1];
            }
            i64 e = o_alg2(nb[0], nb[1], nb[2], nb[3], Q[2 * self], Q[2 * self + 1]);
            if (e < xi) xi = e;
        }
    return xi;
}

/* ------------------------------------------------------------------------ */
/* Quantisation of the bound (R6) and of the residual (R7).                   */
/* ------------------------------------------------------------------------ */
static inline int floor_log2_u64(u64 x) {
    int e = -1;
    while (x) {
        x >>= 1;
        ++e;
    }
    return e;
}

int o_xi_code(i64 xi) { return xi >= 1 ? floor_log2_u64((u64)xi) + 1 : 0; }

static inline i64 floor_div(i64 a, i64 b) { /* b > 0 */
    i64 q = a / b;
    if ((a % b) != 0 && a < 0) --q;
    return q;
}

/* Returns the symbol (0 = unpredictable) and writes the reconstruction. */
static inline int quantize(i64 q, i64 p, i64 xiq, i64* qhat) {
    i64 w = 2 * xiq + 1;
    i64 c = floor_div(q - p + xiq, w);
    if (c > -QRADIUS && c < QRADIUS) {
        *qhat = p + c * w;
        return (int)(c + QRADIUS);
    }
    *qhat = q;
    return 0;
}

int o_quantize(i64 q, i64 p, i64 xiq, i64* qhat) { return quantize(q, p, xiq, qhat); }

/* ------------------------------------------------------------------------ */
/* Predictors.                                                                */
/* ------------------------------------------------------------------------ */
/* First-order 3-D Lorenzo predictor (Sec. VI; reading R8), component c, on   */
/* the current array Q. */
static inline i64 qat(const int32_t* Q, int H, int W, int t, int i, int j, int c) {
    if (t < 0 || i < 0 || j < 0) return 0;
    return Q[2 * vid(H, W, t, i, j) + c];
}

i64 o_lorenzo(const int32_t* Q, int H, int W, int t, int i, int j, int c) {
    return qat(Q, H, W, t, i - 1, j, c) + qat(Q, H, W, t, i, j - 1, c) + qat(Q, H, W, t - 1, i, j, c) -
           qat(Q, H, W, t, i - 1, j - 1, c) - qat(Q, H, W, t - 1, i - 1, j, c) -
           qat(Q, H, W, t - 1, i, j - 1, c) + qat(Q, H, W, t - 1, i - 1, j - 1, c);
}

/* The SL predictor runs in IEEE binary32 (reading R9): Sec. VI-A fixes no
 * precision, the fields are single precision (Sec. V), and the prediction is
 * an integer guess both sides reproduce.  Every float operation below is one
 * correctly rounded IEEE operation (built with -ffp-contract=off; binary32
 * arithmetic has no excess precision on x86-64 or AArch64). */

/* Bilinear interpolation I_bil of one component of slice P (Eq. 6), at a
 * position already clamped to [0,W-1]x[0,H-1].  x is the column, y the row. */
static float bilinear(const int32_t* P, int H, int W, int c, float x, float y) {
    float xf = floorf(x), yf = floorf(y);
    int x0 = (int)xf, y0 = (int)yf;
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
    int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    float fx = x - xf, fy = y - yf;
    float gx = 1.0f - fx, gy = 1.0f - fy;
    float f00 = (float)P[2 * ((i64)y0 * W + x0) + c];
    float f10 = (float)P[2 * ((i64)y0 * W + x1) + c];
    float f01 = (float)P[2 * ((i64)y1 * W + x0) + c];
    float f11 = (float)P[2 * ((i64)y1 * W + x1) + c];
    float w00 = gx * gy, w10 = fx * gy, w01 = gx * fy, w11 = fx * fy;
    float p = w00 * f00 + w10 * f10;
    p = p + w01 * f01;
    p = p + w11 * f11;
    return p;
}

static inline float clampf(float x, float hi) {
    if (x < 0.0f) return 0.0f;
    if (x > hi) return hi;
    return x;
}

/* Semi-Lagrangian predictor (Sec. VI-A, Eqs. 5-9; reading R9).  P is the
 * reconstructed slice t-1 ([H][W][2]); the departure point of grid point
 * (i,j) is traced back with the velocity of slice t-1 and both components are
 * sampled there.  Returns the mode used: 0 RK2, N>0 number of Euler substeps. */
int o_sl_predict(const int32_t* P, int H, int W, int i, int j, float cfl_x, float cfl_y,
                 i64* pu, i64* pv) {
    const int32_t* g = P + 2 * ((i64)i * W + j);
    float du = (float)g[0] * cfl_x;
    float dv = (float)g[1] * cfl_y;
    float dinf = fabsf(du) > fabsf(dv) ? fabsf(du) : fabsf(dv);
    float xs, ys;
    int mode;
    if (dinf <= 2.0f) {
        /* RK2 midpoint (Eqs. 7-8) */
        float xh = clampf((float)j - 0.5f * du, (float)(W - 1));
        float yh = clampf((float)i - 0.5f * dv, (float)(H - 1));
        float uh = bilinear(P, H, W, 0, xh, yh);
        float vh = bilinear(P, H, W, 1, xh, yh);
        xs = clampf((float)j - uh * cfl_x, (float)(W - 1));
        ys = clampf((float)i - vh * cfl_y, (float)(H - 1));
        mode = 0;
    } else {
        /* adaptive Euler substepping (Eq. 9) */
        float nd = ceilf(dinf / 2.0f);
        int N = nd > 32.0f ? 32 : (int)nd;
        float sx = cfl_x / (float)N, sy = cfl_y / (float)N;
        xs = (float)j;
        ys = (float)i;
        for (int s = 0; s < N; ++s) {
            float us = bilinear(P, H, W, 0, xs, ys);
            float vs = bilinear(P, H, W, 1, xs, ys);
            xs = clampf(xs - us * sx, (float)(W - 1));
            ys = clampf(ys - vs * sy, (float)(H - 1));
        }
        mode = N;
    }
    *pu = (i64)floorf(bilinear(P, H, W, 0, xs, ys) + 0.5f);
    *pv = (i64)floorf(bilinear(P, H, W, 1, xs, ys) + 0.5f);
    return mode;
}

/* CFL number dt / (dx * S), S = 2^k, rounded once to binary32 */
float o_cfl(double d_t, double d_x, int k) { return (float)ldexp(d_t / d_x, -k); }

/* ------------------------------------------------------------------------ */
/* MoP scoring (Sec. VI-B; reading R11).                                       */
/* ------------------------------------------------------------------------ */
/* log2(x) in Q32 by repeated squaring of the mantissa (the classic binary    */
/* logarithm algorithm): integer part from the bit length, then one fraction   */
/* bit per squaring.  x >= 1. */
u64 o_ilog2_q32(uint32_t x) {
    int e = floor_log2_u64(x);
    u64 y = ((u64)x << 31) >> e; /* mantissa in [2^31, 2^32), Q31 */
    u64 r = (u64)e << 32;
    for (int b = 31; b >= 0; --b) {
        y = (y * y) >> 31;
        if (y >= (1ull << 32)) {
            y >>= 1;
            r |= 1ull << b;
        }
    }
    return r;
}

/* Estimated rate R_p(B) in Q32 bits per sample (Eq. 10 plus penalty and
 * metadata): H0 + 16 L/(n+L) + 1/(2 B^2).  hist has 65536 bins. */
i64 o_score_q32(const uint32_t* hist, uint32_t n_valid, uint32_t n_fail, int B) {
    i64 h0 = 0;
    if (n_valid > 0) {
        i64 s = (i64)n_valid * (i64)o_ilog2_q32(n_valid);
        for (int k = 0; k < 2 * QRADIUS; ++k)
            if (hist[k] > 0) s -= (i64)hist[k] * (i64)o_ilog2_q32(hist[k]);
        h0 = s / (i64)n_valid;
    }
    i64 pen = 0;
    if (n_valid + n_fail > 0) pen = (i64)(((u64)16 * n_fail << 32) / (u64)(n_valid + n_fail));
    i64 meta = (i64)((1ull << 32) / (u64)(2 * B * B));
    return h0 + pen + meta;
}

/* ------------------------------------------------------------------------ */
/* Canonical length-limited Huffman code (R12): package-merge.                */
/* ------------------------------------------------------------------------ */
typedef struct {
    u64 w;
    uint32_t sym;
} o_leaf;

static int leaf_cmp(const void* a, const void* b) {
    const o_leaf* x = (const o_leaf*)a;
    const o_leaf* y = (const o_leaf*)b;
    if (x->w != y->w) return x->w < y->w ? -1 : 1;
    return x->sym < y->sym ? -1 : (x->sym > y->sym);
}

/* Code lengths (<= maxlen) of an optimal length-limited prefix code.  Leaves
 * sorted by (weight, symbol); at each level the list is the merge of the
 * leaves with the pairwise packages of the previous level, a leaf going first
 * on equal weight; the first 2n-2 items of the last list are selected. */
int o_huff_lengths(const u64* freq, uint32_t nsym, int maxlen, uint8_t* len) {
    memset(len, 0, nsym);
    uint32_t n = 0;
    for (uint32_t s = 0; s < nsym; ++s) n += freq[s] > 0;
    if (n == 0) return O_OK;
    o_leaf* lv = (o_leaf*)malloc(sizeof(o_leaf) * n);
    if (!lv) return O_ERR_OOM;
    n = 0;
    for (uint32_t s = 0; s < nsym; ++s)
        if (freq[s] > 0) {
            lv[n].w = freq[s];
            lv[n].sym = s;
            ++n;
        }
    if (n == 1) {
        len[lv[0].sym] = 1;
        free(lv);
        return O_OK;
    }
    qsort(lv, n, sizeof(o_leaf), leaf_cmp);
    /* per level: weights and the leaf/package flag of each list position */
    size_t cap = 2 * (size_t)n;
    u64* w_prev = (u64*)malloc(sizeof(u64) * cap);
    u64* w_cur = (u64*)malloc(sizeof(u64) * cap);
    uint8_t* isleaf = (uint8_t*)malloc(cap * (size_t)maxlen);
    size_t* cnt = (size_t*)malloc(sizeof(size_t) * maxlen);
    if (!w_prev || !w_cur || !isleaf || !cnt) {
        free(lv); free(w_prev); free(w_cur); free(isleaf); free(cnt);
        return O_ERR_OOM;
    }
    /* level 0 (deepest): the leaves alone */
    for (uint32_t a = 0; a < n; ++a) {
        w_prev[a] = lv[a].w;
        isleaf[a] = 1;
    }
    cnt[0] = n;
    for (int lvl = 1; lvl < maxlen; ++lvl) {
        size_t np = cnt[lvl - 1] / 2, a = 0, b = 0, m = 0;
        uint8_t* fl = isleaf + cap * (size_t)lvl;
        while (a < n || b < np) {
            u64 pw = b < np ? w_prev[2 * b] + w_prev[2 * b + 1] : 0;
            if (a < n && (b >= np || lv[a].w <= pw)) {
                w_cur[m] = lv[a].w;
                fl[m++] = 1;
                ++a;
            } else {
                w_cur[m] = pw;
                fl[m++] = 0;
                ++b;
            }
        }
        cnt[lvl] = m;
        u64* tmp = w_prev;
        w_prev = w_cur;
        w_cur = tmp;
    }
    /* backtrack the selection */
    size_t take = 2 * (size_t)n - 2;
    for (int lvl = maxlen - 1; lvl >= 0 && take > 0; --lvl) {
        const uint8_t* fl = isleaf + cap * (size_t)lvl;
        size_t leaves = 0, packs = 0;
        for (size_t x = 0; x < take; ++x) {
            if (fl[x]) ++leaves; else ++packs;
        }
        for (size_t x = 0; x < leaves; ++x) len[lv[x].sym]++;
        take = 2 * packs;
    }
    free(lv); free(w_prev); free(w_cur); free(isleaf); free(cnt);
    return O_OK;
}

/* Canonical codes: symbols ordered by (length, symbol), consecutive codes. */
static void canonical_codes(const uint8_t* len, uint32_t nsym, uint32_t* code) {
    uint32_t nl[HUFF_MAXLEN + 2] = {0};
    for (uint32_t s = 0; s < nsym; ++s) nl[len[s]]++;
    uint32_t next[HUFF_MAXLEN + 2] = {0};
    uint32_t c = 0;
    nl[0] = 0;
    for (int l = 1; l <= HUFF_MAXLEN; ++l) {
        c = (c + nl[l - 1]) << 1;
        next[l] = c;
    }
    for (uint32_t s = 0; s < nsym; ++s)
        if (len[s]) code[s] = next[len[s]]++;
}

/* ------------------------------------------------------------------------ */
/* Byte buffer helpers (little-endian).                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint8_t* p;
    size_t n, cap;
    int err;
} o_buf;

static void buf_put(o_buf* b, const void* src, size_t n) {
    if (b->err) return;
    if (b->n + n > b->cap) {
        size_t c = b->cap ? b->cap : 4096;
        while (c < b->n + n) c *= 2;
        uint8_t* q = (uint8_t*)realloc(b->p, c);
        if (!q) { b->err = 1; return; }
        b->p = q;
        b->cap = c;
    }
    memcpy(b->p + b->n, src, n);
    b->n += n;
}
static void put_u32(o_buf* b, uint32_t x) {
    uint8_t t[4] = {(uint8_t)x, (uint8_t)(x >> 8), (uint8_t)(x >> 16), (uint8_t)(x >> 24)};
    buf_put(b, t, 4);
}
static void put_u64(o_buf* b, u64 x) {
    put_u32(b, (uint32_t)x);
    put_u32(b, (uint32_t)(x >> 32));
}
static void put_f64(o_buf* b, double d) {
    u64 x;
    memcpy(&x, &d, 8);
    put_u64(b, x);
}
static uint32_t rd_u32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static u64 rd_u64(const uint8_t* p) { return (u64)rd_u32(p) | ((u64)rd_u32(p + 4) << 32); }
static double rd_f64(const uint8_t* p) {
    u64 x = rd_u64(p);
    double d;
    memcpy(&d, &x, 8);
    return d;
}

/* Huffman stream: n_sym u64, n_used u32, chunk u32, table[n_used] u32
 * ((symbol << 8) | length, increasing symbol), chunk_off[ceil(n_sym/chunk)]
 * u64 (bit offset of each chunk's first symbol), n_words u64, words u32 with
 * the code bits packed most-significant bit first. */
static int huff_write(o_buf* b, const uint32_t* sym, u64 nsym_in, uint32_t alpha) {
    u64* freq = (u64*)calloc(alpha, sizeof(u64));
    uint8_t* len = (uint8_t*)malloc(alpha);
    uint32_t* code = (uint32_t*)calloc(alpha, sizeof(uint32_t));
    if (!freq || !len || !code) { free(freq); free(len); free(code); return O_ERR_OOM; }
    for (u64 x = 0; x < nsym_in; ++x) freq[sym[x]]++;
    int rc = o_huff_lengths(freq, alpha, HUFF_MAXLEN, len);
    if (rc) { free(freq); free(len); free(code); return rc; }
    canonical_codes(len, alpha, code);
    uint32_t nused = 0;
    for (uint32_t s = 0; s < alpha; ++s) nused += len[s] > 0;
    put_u64(b, nsym_in);
    put_u32(b, nused);
    put_u32(b, HUFF_CHUNK);
    for (uint32_t s = 0; s < alpha; ++s)
        if (len[s]) put_u32(b, (s << 8) | len[s]);
    u64 nbits = 0;
    for (u64 x = 0; x < nsym_in; ++x) {
        if (x % HUFF_CHUNK == 0) put_u64(b, nbits);
        nbits += len[sym[x]];
    }
    u64 nwords = (nbits + 31) / 32;
    uint32_t* words = (uint32_t*)calloc(nwords ? nwords : 1, sizeof(uint32_t));
    if (!words) { free(freq); free(len); free(code); return O_ERR_OOM; }
    u64 pos = 0;
    for (u64 x = 0; x < nsym_in; ++x) {
        uint32_t c = code[sym[x]];
        int l = len[sym[x]];
        for (int k = l - 1; k >= 0; --k) {
            if ((c >> k) & 1u) words[pos >> 5] |= 1u << (31 - (pos & 31));
            ++pos;
        }
    }
    put_u64(b, nwords);
    for (u64 x = 0; x < nwords; ++x) put_u32(b, words[x]);
    free(words); free(freq); free(len); free(code);
    return b->err ? O_ERR_OOM : O_OK;
}

/* Decodes one Huffman stream; *used = bytes consumed. */
static int huff_read(const uint8_t* p, size_t avail, uint32_t alpha, uint32_t* out, u64 nsym_expect,
                     size_t* used) {
    if (avail < 16) return O_ERR_CORRUPT;
    u64 nsym = rd_u64(p);
    uint32_t nused = rd_u32(p + 8);
    uint32_t chunk = rd_u32(p + 12);
    if (nsym != nsym_expect || nused > alpha || chunk == 0) return O_ERR_CORRUPT;
    size_t off = 16;
    if (avail < off + 4 * (size_t)nused) return O_ERR_CORRUPT;
    uint8_t* len = (uint8_t*)calloc(alpha, 1);
    uint32_t* code = (uint32_t*)calloc(alpha, sizeof(uint32_t));
    if (!len || !code) { free(len); free(code); return O_ERR_OOM; }
    for (uint32_t x = 0; x < nused; ++x) {
        uint32_t e = rd_u32(p + off + 4 * x);
        uint32_t s = e >> 8, l = e & 255u;
        if (s >= alpha || l == 0 || l > HUFF_MAXLEN) { free(len); free(code); return O_ERR_CORRUPT; }
        len[s] = (uint8_t)l;
    }
    off += 4 * (size_t)nused;
    u64 nchunks = (nsym + chunk - 1) / chunk;
    if (avail < off + 8 * nchunks + 8) { free(len); free(code); return O_ERR_CORRUPT; }
    off += 8 * nchunks;
    u64 nwords = rd_u64(p + off);
    off += 8;
    if ((avail - off) / 4 < nwords) { free(len); free(code); return O_ERR_CORRUPT; }
    const uint8_t* wp = p + off;
    canonical_codes(len, alpha, code);
    /* plain bit-by-bit decode against the canonical table */
    uint32_t first[HUFF_MAXLEN + 2], count[HUFF_MAXLEN + 2], base[HUFF_MAXLEN + 2];
    memset(count, 0, sizeof(count));
    for (uint32_t s = 0; s < alpha; ++s) count[len[s]]++;
    uint32_t* sorted = (uint32_t*)malloc(sizeof(uint32_t) * (nused ? nused : 1));
    if (!sorted) { free(len); free(code); return O_ERR_OOM; }
    uint32_t idx = 0;
    for (int l = 1; l <= HUFF_MAXLEN; ++l) {
        base[l] = idx;
        for (uint32_t s = 0; s < alpha; ++s)
            if (len[s] == l) sorted[idx++] = s;
    }
    uint32_t c = 0;
    count[0] = 0;
    for (int l = 1; l <= HUFF_MAXLEN; ++l) {
        c = (c + count[l - 1]) << 1;
        first[l] = c;
    }
    u64 pos = 0, total = nwords * 32;
    int rc = O_OK;
    for (u64 x = 0; x < nsym && rc == O_OK; ++x) {
        uint32_t v = 0;
        int l = 0;
        for (;;) {
            if (pos >= total) { rc = O_ERR_CORRUPT; break; }
            uint32_t word = rd_u32(wp + 4 * (pos >> 5));
            v = (v << 1) | ((word >> (31 - (pos & 31))) & 1u);
            ++pos;
            ++l;
            if (l > HUFF_MAXLEN) { rc = O_ERR_CORRUPT; break; }
            if (count[l] && v >= first[l] && v - first[l] < count[l]) {
                out[x] = sorted[base[l] + (v - first[l])];
                break;
            }
        }
    }
    free(sorted); free(len); free(code);
    *used = off + 4 * nwords;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Compression (Alg. 3 with Alg. 4 and the MoP pass).                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t k, eps_int;
    double eps, vmin, vmax;
    u64 crossed_faces, lossless_vertices, unpredictable, sl_blocks, blocks, n_ld, n_qd;
    u64 substep_vertices, substeps_total;
} o_stats;

/* Micro-encodes block (by,bx) of slice t under 3DL or SL and returns its Q32
 * score (Sec. VI-B).  Qcur is the current array (slice t-1 reconstructed,
 * slice t original), q the original field, xiq the quantiser half width. */
/* ------------------------------------------------------------------------ */
/* Learned predictor (predictor 3; an extension, the paper has none).  A     */
/* 3-layer 3x3 convolutional net, 2 -> 32 -> 32 -> 2 channels, ReLU after    */
/* the first two layers, zero padding at the field boundary, maps the        */
/* reconstructed slice t-1 scaled by 2^-23 to the change y of each component. */
/* Parameters are bfloat16: w1[32][2][3][3] b1[32] w2[32][32][3][3] b2[32]     */
/* w3[2][32][3][3] b3[2].  Every output is a chain of float32 fused           */
/* multiply-adds starting from the bias, over (input channel, ky, kx) in that */
/* order, padding included as zero inputs, so any IEEE implementation gives   */
/* the same bits.  Prediction: qhat(t-1) + rint(clamp(y, -2, 2) * 2^23).      */
/* ------------------------------------------------------------------------ */
#define NET_C 32
#define NET_PARAMS (NET_C * 2 * 9 + NET_C + NET_C * NET_C * 9 + NET_C + 2 * NET_C * 9 + 2)

int o_net_params(void) { return NET_PARAMS; }

static float bf16f(uint16_t h) {
    uint32_t x = (uint32_t)h << 16;
    float f;
    memcpy(&f, &x, 4);
    return f;
}

/* out[co][i][j] = act(b[co] + sum over (ci, ky, kx) of w[co][ci][ky][kx] * in[ci][i+ky-1][j+kx-1]) */
static void net_conv(const float* in, int cin, int H, int W, const uint16_t* w, const uint16_t* b, int cout,
                     int relu, float* out) {
    for (int co = 0; co < cout; ++co)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                float acc = bf16f(b[co]);
                for (int ci = 0; ci < cin; ++ci)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            int ii = i + ky - 1, jj = j + kx - 1;
                            float v = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? in[((i64)ci * H + ii) * W + jj] : 0.0f;
                            acc = fmaf(bf16f(w[((co * cin + ci) * 3 + ky) * 3 + kx]), v, acc);
                        }
                out[((i64)co * H + i) * W + j] = relu ? (acc > 0.0f ? acc : 0.0f) : acc;
            }
}

/* y = net(prev * 2^-23) for a whole slice: y[2][H][W] (float). */
void o_net_forward(const uint16_t* model, const int32_t* prev, int H, int W, float* y) {
    const uint16_t* w1 = model;
    const uint16_t* b1 = w1 + NET_C * 2 * 9;
    const uint16_t* w2 = b1 + NET_C;
    const uint16_t* b2 = w2 + NET_C * NET_C * 9;
    const uint16_t* w3 = b2 + NET_C;
    const uint16_t* b3 = w3 + 2 * NET_C * 9;
    i64 hw = (i64)H * W;
    float* x = (float*)malloc(sizeof(float) * 2 * hw);
    float* h1 = (float*)malloc(sizeof(float) * NET_C * hw);
    float* h2 = (float*)malloc(sizeof(float) * NET_C * hw);
    if (!x || !h1 || !h2) { free(x); free(h1); free(h2); for (i64 k = 0; k < 2 * hw; ++k) y[k] = 0.0f; return; }
    for (i64 v = 0; v < hw; ++v) {  /* 2^-23 scaling of |q| < 2^24: exact */
        x[v] = (float)prev[2 * v] * 0x1p-23f;
        x[hw + v] = (float)prev[2 * v + 1] * 0x1p-23f;
    }
    net_conv(x, 2, H, W, w1, b1, NET_C, 1, h1);
    net_conv(h1, NET_C, H, W, w2, b2, NET_C, 1, h2);
    net_conv(h2, NET_C, H, W, w3, b3, 2, 0, y);
    free(x); free(h1); free(h2);
}

/* The learned prediction of every vertex of a slice: pred[H][W][2]. */
void o_net_predict(const uint16_t* model, const int32_t* prev, int H, int W, int32_t* pred) {
    i64 hw = (i64)H * W;
    float* y = (float*)malloc(sizeof(float) * 2 * hw);
    if (!y) { for (i64 v = 0; v < 2 * hw; ++v) pred[v] = prev[v]; return; }
    o_net_forward(model, prev, H, W, y);
    for (i64 v = 0; v < hw; ++v)
        for (int c = 0; c < 2; ++c) {
            float d = y[c * hw + v];
            if (!(d == d)) d = 0.0f;
            d = d < -2.0f ? -2.0f : (d > 2.0f ? 2.0f : d);
            pred[2 * v + c] = prev[2 * v + c] + (int32_t)rintf(d * 0x1p23f);
        }
    free(y);
}

/* Score of one block (Sec. VI) with mode 0 = 3DL, 1 = SL, 2 = the learned
 * predictions npred of the slice (the learned mixture). */
static i64 mop_block_score(const int32_t* Q, int H, int W, int t, int by, int bx, int B, int n,
                           int mode, i64 xiq, float cfl_x, float cfl_y, const int32_t* npred,
                           int32_t* cand, uint32_t* hist) {
    int i0 = by * B, j0 = bx * B;
    int i1 = i0 + B < H ? i0 + B : H, j1 = j0 + B < W ? j0 + B : W;
    const int32_t* prev = Q + 2 * vid(H, W, t - 1, 0, 0);
    const int32_t* orig = Q + 2 * vid(H, W, t, 0, 0);
    /* candidate buffer for rows i0-1..i1-1, cols j0-1..j1-1 (halo = original) */
    int bw = j1 - j0 + 1;
    for (int i = i0 - 1; i < i1; ++i)
        for (int j = j0 - 1; j < j1; ++j)
            for (int c = 0; c < 2; ++c) {
                int32_t val = (i >= 0 && j >= 0) ? orig[2 * ((i64)i * W + j) + c] : 0;
                cand[2 * ((i - i0 + 1) * bw + (j - j0 + 1)) + c] = val;
            }
    uint32_t nv = 0, nf = 0;
    for (int i = i0; i < i1; ++i)
        for (int j = j0; j < j1; ++j) {
            int sampled = (i % n == 0) && (j % n == 0);
            i64 pu = 0, pv = 0;
            if (mode == 1) o_sl_predict(prev, H, W, i, j, cfl_x, cfl_y, &pu, &pv);
            if (mode == 2) {
                pu = npred[2 * ((i64)i * W + j)];
                pv = npred[2 * ((i64)i * W + j) + 1];
            }
            for (int c = 0; c < 2; ++c) {
                i64 p;
                if (mode != 0) {
                    p = c == 0 ? pu : pv;
                } else {
                    /* Lorenzo on the candidate buffer (slice t) and slice t-1 */
#define CB(ii, jj) ((i64)cand[2 * (((ii) - i0 + 1) * bw + ((jj) - j0 + 1)) + c])
#define PV(ii, jj) (((ii) < 0 || (jj) < 0) ? 0 : (i64)prev[2 * ((i64)(ii) * W + (jj)) + c])
                    p = CB(i - 1, j) + CB(i, j - 1) + PV(i, j) - CB(i - 1, j - 1) - PV(i - 1, j) -
                        PV(i, j - 1) + PV(i - 1, j - 1);
#undef PV
                }
                i64 qv = orig[2 * ((i64)i * W + j) + c], qh;
                int sym = quantize(qv, p, xiq, &qh);
                cand[2 * ((i - i0 + 1) * bw + (j - j0 + 1)) + c] = (int32_t)qh;
                if (sampled) {
                    if (sym) { hist[sym]++; ++nv; } else { ++nf; }
                }
#undef CB
            }
        }
    return o_score_q32(hist, nv, nf, B);
}

static void mop_modes(const int32_t* Q, int H, int W, int t, int B, int n, i64 xiq, float cfl_x,
                      float cfl_y, const int32_t* npred /* NULL: SL */, uint8_t* modes /* nby*nbx */,
                      o_stats* st) {
    int nby = (H + B - 1) / B, nbx = (W + B - 1) / B;
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * 2 * (B + 1) * (B + 1));
    uint32_t* hist = (uint32_t*)calloc(2 * QRADIUS, sizeof(uint32_t));
    for (int by = 0; by < nby; ++by)
        for (int bx = 0; bx < nbx; ++bx) {
            i64 r3, rs;
            memset(hist, 0, sizeof(uint32_t) * 2 * QRADIUS);
            r3 = mop_block_score(Q, H, W, t, by, bx, B, n, 0, xiq, cfl_x, cfl_y, npred, cand, hist);
            memset(hist, 0, sizeof(uint32_t) * 2 * QRADIUS);
            rs = mop_block_score(Q, H, W, t, by, bx, B, n, npred ? 2 : 1, xiq, cfl_x, cfl_y, npred, cand, hist);
            uint8_t m = (1000 * rs < 997 * r3) ? 1 : 0;
            modes[by * nbx + bx] = m;
            st->sl_blocks += m;
            st->blocks++;
        }
    free(cand);
    free(hist);
}

/* Full compressor.  Optional outputs (nullable): q (fixed point input),
 * qhat (reconstruction), xi (per-vertex integer bound), qxi (codes), modes
 * (T*nby*nbx block modes), mask (crossed faces), qd (N*2 per-vertex symbols,
 * 0xFFFFFFFF where absent).  t_end < T stops after slice t_end-1 (the bytes
 * are then not produced). */
int o_compress2(const float* uv, int H, int W, int T, double d_x, double d_y, double d_t,
                int eb_mode, double eb, int pred, int B, int n, int t_end, const uint16_t* model,
                uint8_t** out, size_t* out_bytes, int32_t* q_out, int32_t* qhat_out, int64_t* xi_out,
                uint8_t* qxi_out, uint8_t* modes_out, uint16_t* mask_out, uint32_t* qd_out, o_stats* st,
                const uint8_t* force) {
    if (H < 2 || W < 2 || T < 1 || B < 1 || n < 1 || pred < 0 || pred > 4) return O_ERR_ARG;
    const int has_net = pred == 3 || pred == 4, has_modes = pred == 2 || pred == 4;
    if (has_net && !model) return O_ERR_ARG;
    if (!(d_x > 0) || !(d_y > 0) || !(d_t > 0) || !(eb >= 0)) return O_ERR_ARG;
    i64 N = (i64)H * W * T;
    o_stats S;
    memset(&S, 0, sizeof(S));
    double amax;
    if (o_range(uv, 2 * N, &S.vmin, &S.vmax, &amax)) return O_ERR_ARG;
    S.k = o_scale_exponent(amax);
    S.eps = eb_mode == 1 ? eb * (S.vmax - S.vmin) : eb;
    S.eps_int = o_eps_int(S.eps, S.k);
    i64 eps_int = S.eps_int;
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * 2 * N);
    int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * 2 * N);
    uint16_t* mask = (uint16_t*)malloc(sizeof(uint16_t) * N);
    uint8_t* qxi = (uint8_t*)malloc(N);
    uint32_t* qd = (uint32_t*)malloc(sizeof(uint32_t) * 2 * N);
    int32_t* ld = (int32_t*)malloc(sizeof(int32_t) * 2 * N);
    int nby = (H + B - 1) / B, nbx = (W + B - 1) / B;
    uint8_t* modes = (uint8_t*)calloc((size_t)T * nby * nbx, 1);
    int32_t* npred = has_net ? (int32_t*)malloc(sizeof(int32_t) * 2 * H * W) : NULL;
    if (!q || !Q || !mask || !qxi || !qd || !ld || !modes || (has_net && !npred)) {
        free(q); free(Q); free(mask); free(qxi); free(qd); free(ld); free(modes); free(npred);
        return O_ERR_OOM;
    }
    o_to_fixed(uv, 2 * N, S.k, q);
    memcpy(Q, q, sizeof(int32_t) * 2 * N);
    o_face_masks(q, H, W, T, mask);
    for (i64 v = 0; v < N; ++v)
        for (int b = 0; b < 12; ++b) S.crossed_faces += (mask[v] >> b) & 1u;
    float cfl_x = o_cfl(d_t, d_x, S.k), cfl_y = o_cfl(d_t, d_y, S.k);
    i64 xiq_eps = eps_int >= 1 ? (i64)1 << floor_log2_u64((u64)eps_int) : 0;
    if (t_end > T || t_end < 0) t_end = T;
    u64 nqd = 0, nld = 0;
    if (xi_out) for (i64 v = 0; v < N; ++v) xi_out[v] = -1;
    if (qd_out) for (i64 v = 0; v < 2 * N; ++v) qd_out[v] = 0xFFFFFFFFu;
    for (int t = 0; t < t_end; ++t) {
        uint8_t* tm = modes + (size_t)t * nby * nbx;
        const int32_t* prev = t >= 1 ? Q + 2 * vid(H, W, t - 1, 0, 0) : NULL;
        /* learned: the whole slice's predictions from the finished slice t-1 */
        if (has_net && t >= 1) o_net_predict(model, prev, H, W, npred);
        if (has_modes && t >= 1 && xiq_eps >= 1)
            mop_modes(Q, H, W, t, B, n, xiq_eps, cfl_x, cfl_y, pred == 4 ? npred : NULL, tm, &S);
        else if (has_modes)
            S.blocks += (u64)nby * nbx;
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                i64 v = vid(H, W, t, i, j);
                int crossed;
                i64 xi = derive_min_eb(Q, mask, H, W, T, t, i, j, eps_int, &crossed);
                /* reading R14 (repair of a failed verification): a forced vertex is
                 * stored losslessly */
                if (force && force[v]) xi = 0;
                if (xi_out) xi_out[v] = xi;
                int code = o_xi_code(xi);
                qxi[v] = (uint8_t)code;
                if (code == 0) {
                    ld[nld++] = Q[2 * v];
                    ld[nld++] = Q[2 * v + 1];
                    S.lossless_vertices++;
                    continue;
                }
                i64 xiq = (i64)1 << (code - 1);
                const int blk = has_modes && tm[(i / B) * nbx + (j / B)];
                int use_sl = t >= 1 && (pred == 1 || (pred == 2 && blk));
                i64 pu = 0, pv = 0;
                if (t >= 1 && (pred == 3 || (pred == 4 && blk))) {
                    pu = npred[2 * ((i64)i * W + j)];
                    pv = npred[2 * ((i64)i * W + j) + 1];
                } else if (use_sl) {
                    int md = o_sl_predict(prev, H, W, i, j, cfl_x, cfl_y, &pu, &pv);
                    if (md > 0) { S.substep_vertices++; S.substeps_total += (u64)md; }
                } else {
                    pu = o_lorenzo(Q, H, W, t, i, j, 0);
                    pv = o_lorenzo(Q, H, W, t, i, j, 1);
                }
                for (int c = 0; c < 2; ++c) {
                    i64 qh;
                    int sym = quantize(Q[2 * v + c], c == 0 ? pu : pv, xiq, &qh);
                    qd[nqd++] = (uint32_t)sym;
                    if (qd_out) qd_out[2 * v + c] = (uint32_t)sym;
                    if (sym == 0) {
                        ld[nld++] = Q[2 * v + c];
                        S.unpredictable++;
                    }
                    Q[2 * v + c] = (int32_t)qh;
                }
            }
    }
    S.n_ld = nld;
    S.n_qd = nqd;
    int rc = O_OK;
    if (out && out_bytes && t_end == T) {
        o_buf b = {0};
        buf_put(&b, "CPT1", 4);
        put_u32(&b, 1);
        put_u32(&b, (uint32_t)H);
        put_u32(&b, (uint32_t)W);
        put_u32(&b, (uint32_t)T);
        put_u32(&b, (uint32_t)S.k);
        put_u32(&b, (uint32_t)S.eps_int);
        put_u32(&b, (uint32_t)pred);
        put_u32(&b, (uint32_t)B);
        put_u32(&b, (uint32_t)n);
        put_u32(&b, QRADIUS);
        put_u32(&b, 0);
        put_f64(&b, d_x);
        put_f64(&b, d_y);
        put_f64(&b, d_t);
        put_f64(&b, S.eps);
        put_u64(&b, nld);
        u64 nblk = has_modes ? (u64)T * nby * nbx : 0;
        u64 mode_bytes = (nblk + 7) / 8;
        put_u64(&b, mode_bytes);
        for (u64 x = 0; x < mode_bytes; ++x) {
            uint8_t byte = 0;
            for (int bit = 0; bit < 8; ++bit) {
                u64 idx = x * 8 + bit;
                if (idx < nblk && modes[idx]) byte |= (uint8_t)(1u << bit);
            }
            buf_put(&b, &byte, 1);
        }
        if (has_net) {  /* the model: parameter count, then the bfloat16 parameters (4-byte padded) */
            put_u32(&b, NET_PARAMS);
            for (int x = 0; x < NET_PARAMS; x += 2)
                put_u32(&b, (uint32_t)model[x] | (x + 1 < NET_PARAMS ? (uint32_t)model[x + 1] << 16 : 0u));
        }
        uint32_t* xs = (uint32_t*)malloc(sizeof(uint32_t) * (N ? N : 1));
        if (!xs) rc = O_ERR_OOM;
        if (!rc) {
            for (i64 v = 0; v < N; ++v) xs[v] = qxi[v];
            rc = huff_write(&b, xs, (u64)N, 33);
        }
        free(xs);
        if (!rc) rc = huff_write(&b, qd, nqd, 2 * QRADIUS);
        for (u64 x = 0; x < nld && !rc; ++x) put_u32(&b, (uint32_t)ld[x]);
        if (!rc && b.err) rc = O_ERR_OOM;
        if (rc) {
            free(b.p);
        } else {
            *out = b.p;
            *out_bytes = b.n;
        }
    }
    if (q_out) memcpy(q_out, q, sizeof(int32_t) * 2 * N);
    if (qhat_out) memcpy(qhat_out, Q, sizeof(int32_t) * 2 * N);
    if (qxi_out) memcpy(qxi_out, qxi, N);
    if (mask_out) memcpy(mask_out, mask, sizeof(uint16_t) * N);
    if (modes_out) memcpy(modes_out, modes, (size_t)T * nby * nbx);
    if (st) *st = S;
    free(q); free(Q); free(mask); free(qxi); free(qd); free(ld); free(modes); free(npred);
    return rc;
}

int o_compress(const float* uv, int H, int W, int T, double d_x, double d_y, double d_t,
               int eb_mode, double eb, int pred, int B, int n, int t_end, uint8_t** out,
               size_t* out_bytes, int32_t* q_out, int32_t* qhat_out, int64_t* xi_out,
               uint8_t* qxi_out, uint8_t* modes_out, uint16_t* mask_out, uint32_t* qd_out,
               o_stats* st) {
    if (pred == 3 || pred == 4) return O_ERR_ARG;
    return o_compress2(uv, H, W, T, d_x, d_y, d_t, eb_mode, eb, pred, B, n, t_end, NULL, out, out_bytes, q_out,
                       qhat_out, xi_out, qxi_out, modes_out, mask_out, qd_out, st, NULL);
}

void o_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Decompression: the inverse raster loop (decoded bounds, no derivation).     */
/* ------------------------------------------------------------------------ */
int o_decompress(const uint8_t* in, size_t nbytes, int* dims /* H W T k */, int32_t* qhat_out,
                 float* uv_out) {
    if (nbytes < 96 || memcmp(in, "CPT1", 4) != 0 || rd_u32(in + 4) != 1) return O_ERR_CORRUPT;
    int H = (int)rd_u32(in + 8), W = (int)rd_u32(in + 12), T = (int)rd_u32(in + 16);
    int k = (int)rd_u32(in + 20);
    int pred = (int)rd_u32(in + 28), B = (int)rd_u32(in + 32);
    double d_x = rd_f64(in + 48), d_y = rd_f64(in + 56), d_t = rd_f64(in + 64);
    u64 nld = rd_u64(in + 80), mode_bytes = rd_u64(in + 88);
    if (H < 2 || W < 2 || T < 1 || B < 1 || pred < 0 || pred > 4) return O_ERR_CORRUPT;
    const int has_net = pred == 3 || pred == 4;
    if (dims) { dims[0] = H; dims[1] = W; dims[2] = T; dims[3] = k; }
    if (!qhat_out && !uv_out) return O_OK;
    i64 N = (i64)H * W * T;
    int nby = (H + B - 1) / B, nbx = (W + B - 1) / B;
    size_t off = 96;
    if (nbytes - off < mode_bytes) return O_ERR_CORRUPT;
    const uint8_t* mb = in + off;
    off += mode_bytes;
    uint16_t model[NET_PARAMS];
    if (has_net) {
        if (nbytes - off < 4 || rd_u32(in + off) != NET_PARAMS) return O_ERR_CORRUPT;
        off += 4;
        size_t mbytes = 4 * (size_t)((NET_PARAMS + 1) / 2);
        if (nbytes - off < mbytes) return O_ERR_CORRUPT;
        for (int x = 0; x < NET_PARAMS; ++x) model[x] = (uint16_t)(rd_u32(in + off + 4 * (x / 2)) >> (16 * (x & 1)));
        off += mbytes;
    }
    uint32_t* xs = (uint32_t*)malloc(sizeof(uint32_t) * N);
    int32_t* Q = (int32_t*)malloc(sizeof(int32_t) * 2 * N);
    if (!xs || !Q) { free(xs); free(Q); return O_ERR_OOM; }
    size_t used;
    int rc = huff_read(in + off, nbytes - off, 33, xs, (u64)N, &used);
    if (rc) { free(xs); free(Q); return rc; }
    off += used;
    u64 nqd = 0;
    for (i64 v = 0; v < N; ++v) nqd += xs[v] ? 2 : 0;
    uint32_t* qd = (uint32_t*)malloc(sizeof(uint32_t) * (nqd ? nqd : 1));
    if (!qd) { free(xs); free(Q); return O_ERR_OOM; }
    rc = huff_read(in + off, nbytes - off, 2 * QRADIUS, qd, nqd, &used);
    if (rc) { free(xs); free(Q); free(qd); return rc; }
    off += used;
    if ((nbytes - off) / 4 < nld) { free(xs); free(Q); free(qd); return O_ERR_CORRUPT; }
    const uint8_t* ldp = in + off;
    float cfl_x = o_cfl(d_t, d_x, k), cfl_y = o_cfl(d_t, d_y, k);
    u64 iq = 0, il = 0;
    int32_t* npred = has_net ? (int32_t*)malloc(sizeof(int32_t) * 2 * H * W) : NULL;
    if (has_net && !npred) rc = O_ERR_OOM;
    for (int t = 0; t < T && !rc; ++t) {
        const int32_t* prev = t >= 1 ? Q + 2 * vid(H, W, t - 1, 0, 0) : NULL;
        if (has_net && t >= 1) o_net_predict(model, prev, H, W, npred);
        for (int i = 0; i < H && !rc; ++i)
            for (int j = 0; j < W; ++j) {
                i64 v = vid(H, W, t, i, j);
                uint32_t code = xs[v];
                if (code > 24) { rc = O_ERR_CORRUPT; break; }
                if (code == 0) {
                    if (il + 2 > nld) { rc = O_ERR_CORRUPT; break; }
                    Q[2 * v] = (int32_t)rd_u32(ldp + 4 * il);
                    Q[2 * v + 1] = (int32_t)rd_u32(ldp + 4 * (il + 1));
                    il += 2;
                    continue;
                }
                i64 xiq = (i64)1 << (code - 1), w = 2 * xiq + 1;
                u64 bidx = ((u64)t * nby + (u64)(i / B)) * nbx + (u64)(j / B);
                int blk = (pred == 2 || pred == 4) && ((mb[bidx >> 3] >> (bidx & 7)) & 1u);
                int use_sl = t >= 1 && (pred == 1 || (pred == 2 && blk));
                i64 pu, pv;
                if (t >= 1 && (pred == 3 || (pred == 4 && blk))) {
                    pu = npred[2 * ((i64)i * W + j)];
                    pv = npred[2 * ((i64)i * W + j) + 1];
                } else if (use_sl) {
                    o_sl_predict(prev, H, W, i, j, cfl_x, cfl_y, &pu, &pv);
                } else {
                    pu = o_lorenzo(Q, H, W, t, i, j, 0);
                    pv = o_lorenzo(Q, H, W, t, i, j, 1);
                }
                for (int c = 0; c < 2; ++c) {
                    uint32_t sym = qd[iq++];
                    if (sym == 0) {
                        if (il + 1 > nld) { rc = O_ERR_CORRUPT; break; }
                        Q[2 * v + c] = (int32_t)rd_u32(ldp + 4 * il);
                        ++il;
                    } else {
                        Q[2 * v + c] = (int32_t)((c == 0 ? pu : pv) + ((i64)sym - QRADIUS) * w);
                    }
                }
            }
    }
    if (!rc) {
        if (qhat_out) memcpy(qhat_out, Q, sizeof(int32_t) * 2 * N);
        if (uv_out)
            for (i64 x = 0; x < 2 * N; ++x) uv_out[x] = (float)ldexp((double)Q[x], -k);
    }
    free(xs); free(Q); free(qd); free(npred);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Trajectories (Sec. IV, Thm. 2; reading R13).                                */
/* ------------------------------------------------------------------------ */
static i64 lower_bound_u64(const u64* a, i64 n, u64 key) {
    i64 lo = 0, hi = n;
    while (lo < hi) {
        i64 mid = (lo + hi) / 2;
        if (a[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Crossing point of a crossed face (Eq. 3): barycentric weights
 * (det(b,c), det(c,a), det(a,b)) / D_f applied to the (x=j, y=i, t) of its
 * vertices; D_f = 0 gives the centroid. */
static void crossing_point(const int32_t* q, int H, int W, u64 fid, double* xyt) {
    i64 owner = (i64)(fid / 12);
    int type = (int)(fid % 12);
    int j = (int)(owner % W), i = (int)((owner / W) % H), t = (int)(owner / ((i64)W * H));
    i64 p[6];
    face_values(q, H, W, t, i, j, type, p);
    i64 dbc = p[2] * p[5] - p[3] * p[4];
    i64 dca = p[4] * p[1] - p[5] * p[0];
    i64 dab = p[0] * p[3] - p[1] * p[2];
    i64 D = dbc + dca + dab;
    double wa, wb, wc;
    if (D == 0) {
        wa = wb = wc = 1.0 / 3.0;
    } else {
        wa = (double)dbc / (double)D;
        wb = (double)dca / (double)D;
        wc = (double)dab / (double)D;
    }
    double w3[3] = {wa, wb, wc};
    xyt[0] = xyt[1] = xyt[2] = 0.0;
    for (int k = 0; k < 3; ++k) {
        xyt[0] += w3[k] * (double)(j + O_FACE[type][k][2]);
        xyt[1] += w3[k] * (double)(i + O_FACE[type][k][1]);
        xyt[2] += w3[k] * (double)(t + O_FACE[type][k][0]);
    }
}

/* Links the crossed faces of q into trajectories.  Outputs (library-allocated
 * with malloc, freed by o_free): face ids in trajectory order, offsets
 * (n_traj+1), xyt (3 per face).  Each trajectory starts at its lowest-id
 * endpoint (or its lowest-id face for a closed loop, walking to the lower-id
 * neighbour first); trajectories are ordered by their starting face id.
 * Returns the number of tets whose crossed-face count is not 0 or 2 in
 * *bad_tets (Lemma 1 check). */
int o_trajectories(const int32_t* q, int H, int W, int T, u64* n_traj_out, u64* n_faces_out,
                   u64** faces_out, u64** offsets_out, double** xyt_out, u64* bad_tets) {
    i64 N = (i64)H * W * T;
    uint16_t* mask = (uint16_t*)malloc(sizeof(uint16_t) * N);
    if (!mask) return O_ERR_OOM;
    o_face_masks(q, H, W, T, mask);
    i64 nf = 0;
    for (i64 v = 0; v < N; ++v)
        for (int b = 0; b < 12; ++b) nf += (mask[v] >> b) & 1u;
    u64* fid = (u64*)malloc(sizeof(u64) * (nf ? nf : 1));
    i64* nb = (i64*)malloc(sizeof(i64) * 2 * (nf ? nf : 1));
    if (!fid || !nb) { free(mask); free(fid); free(nb); return O_ERR_OOM; }
    i64 x = 0;
    for (i64 v = 0; v < N; ++v)
        for (int b = 0; b < 12; ++b)
            if ((mask[v] >> b) & 1u) fid[x++] = (u64)v * 12 + (u64)b;
    for (i64 a = 0; a < nf; ++a) nb[2 * a] = nb[2 * a + 1] = -1;
    u64 bad = 0;
    for (int t = 0; t + 1 < T; ++t)
        for (int i = 0; i + 1 < H; ++i)
            for (int j = 0; j + 1 < W; ++j)
                for (int tet = 0; tet < 6; ++tet) {
                    i64 hit[4];
                    int nh = 0;
                    for (int f = 0; f < 4; ++f) {
                        const int* e = O_TET[tet][f];
                        i64 ow = vid(H, W, t + e[0], i + e[1], j + e[2]);
                        if ((mask[ow] >> e[3]) & 1u)
                            hit[nh++] = lower_bound_u64(fid, nf, (u64)ow * 12 + (u64)e[3]);
                    }
                    if (nh == 0) continue;
                    if (nh != 2) { ++bad; continue; }
                    i64 a = hit[0], c = hit[1];
                    if (nb[2 * a] < 0) nb[2 * a] = c; else nb[2 * a + 1] = c;
                    if (nb[2 * c] < 0) nb[2 * c] = a; else nb[2 * c + 1] = a;
                }
    /* walk each component */
    uint8_t* seen = (uint8_t*)calloc(nf ? nf : 1, 1);
    u64* order = (u64*)malloc(sizeof(u64) * (nf ? nf : 1));
    u64* offs = (u64*)malloc(sizeof(u64) * (nf + 1));
    double* xyt = (double*)malloc(sizeof(double) * 3 * (nf ? nf : 1));
    if (!seen || !order || !offs || !xyt) {
        free(mask); free(fid); free(nb); free(seen); free(order); free(offs); free(xyt);
        return O_ERR_OOM;
    }
    u64 ntraj = 0, pos = 0;
    /* pass 1: endpoints (degree <= 1) in id order start open paths; pass 2: loops */
    for (int pass = 0; pass < 2; ++pass)
        for (i64 a = 0; a < nf; ++a) {
            if (seen[a]) continue;
            int deg = (nb[2 * a] >= 0) + (nb[2 * a + 1] >= 0);
            if (pass == 0 && deg == 2) continue;
            offs[ntraj++] = pos;
            i64 prevf = -1, cur = a;
            while (cur >= 0 && !seen[cur]) {
                seen[cur] = 1;
                order[pos++] = fid[cur];
                i64 n0 = nb[2 * cur], n1 = nb[2 * cur + 1], nxt = -1;
                if (pass == 1 && prevf < 0) {
                    /* closed loop: leave towards the lower-id neighbour */
                    nxt = (n0 >= 0 && (n1 < 0 || n0 < n1)) ? n0 : n1;
                } else {
                    if (n0 >= 0 && n0 != prevf && !seen[n0]) nxt = n0;
                    else if (n1 >= 0 && n1 != prevf && !seen[n1]) nxt = n1;
                }
                prevf = cur;
                cur = nxt;
            }
        }
    offs[ntraj] = pos;
    /* trajectories were produced endpoints-first then loops; order them by
     * their starting face id */
    {
        u64* idx = (u64*)malloc(sizeof(u64) * (ntraj ? ntraj : 1));
        u64* order2 = (u64*)malloc(sizeof(u64) * (nf ? nf : 1));
        u64* offs2 = (u64*)malloc(sizeof(u64) * (ntraj + 1));
        for (u64 a = 0; a < ntraj; ++a) idx[a] = a;
        /* insertion sort is too slow for many trajectories: simple merge sort */
        for (u64 width = 1; width < ntraj; width *= 2) {
            u64* tmp = (u64*)malloc(sizeof(u64) * ntraj);
            for (u64 lo = 0; lo < ntraj; lo += 2 * width) {
                u64 mid = lo + width < ntraj ? lo + width : ntraj;
                u64 hi = lo + 2 * width < ntraj ? lo + 2 * width : ntraj;
                u64 a = lo, b = mid, m = lo;
                while (a < mid || b < hi) {
                    if (a < mid && (b >= hi || order[offs[idx[a]]] <= order[offs[idx[b]]]))
                        tmp[m++] = idx[a++];
                    else
                        tmp[m++] = idx[b++];
                }
            }
            memcpy(idx, tmp, sizeof(u64) * ntraj);
            free(tmp);
        }
        u64 p2 = 0;
        for (u64 a = 0; a < ntraj; ++a) {
            offs2[a] = p2;
            for (u64 s = offs[idx[a]]; s < offs[idx[a] + 1]; ++s) order2[p2++] = order[s];
        }
        offs2[ntraj] = p2;
        memcpy(order, order2, sizeof(u64) * p2);
        memcpy(offs, offs2, sizeof(u64) * (ntraj + 1));
        free(idx); free(order2); free(offs2);
    }
    for (u64 a = 0; a < pos; ++a) crossing_point(q, H, W, order[a], xyt + 3 * a);
    *n_traj_out = ntraj;
    *n_faces_out = (u64)nf;
    if (bad_tets) *bad_tets = bad;
    if (faces_out) *faces_out = order; else free(order);
    if (offsets_out) *offsets_out = offs; else free(offs);
    if (xyt_out) *xyt_out = xyt; else free(xyt);
    free(mask); free(fid); free(nb); free(seen);
    return O_OK;
}

/* Stats struct size, for the binding's sanity check. */
int o_stats_size(void) { return (int)sizeof(o_stats); }
