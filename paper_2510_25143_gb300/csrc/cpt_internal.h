// Internal declarations of the library: small device structs and the host-side
// launchers of every kernel (one translation unit per kernel family).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "cpt_net.cuh"

namespace cpt {

struct RangePartial {
    float mn, mx, amax;
    unsigned bad;
};

struct VerifyOut {
    unsigned long long mismatch_slice;
    unsigned long long mismatch_slab;
    unsigned long long linf_bits;  // double bits of max |x_hat - x|
    double sq_err;
};

// The encoder's reconstruction array holds (x, y ^ kQhatTag) per vertex: a
// written word is told from the zeroed array by bits 30 and 31 of y.
constexpr int kQhatTag = 0x40000000;

// Arguments of the encoder pipeline (one persistent launch over all slices).
struct SliceArgs {
    const int2* q;          // original fixed point [T][H][W]
    int2* qhat;             // reconstruction words [T][H][W] (tagged, zeroed before the launch)
    const uint16_t* mask;   // crossed-face masks [T][H][W]
    // Strip-diagonal layout [T][nstrips][W + 31][32] (zero padding): element
    // (t, s, k, l) holds vertex (32 s + l, k - l), the vertex lane l of
    // wave(t, s) handles at step k, so that a wave's loads are contiguous.
    const int2* cls;        // (bound over certain faces, faces needing the full Alg. 2)
    const unsigned* cls_m;  // faces needing only the M = 0 check
    const int2* qd;         // the original fixed point q
    int2* psl;              // [T][H][W] semi-Lagrangian predictions (where needed)
    uint8_t* modes;         // [T][nby][nbx] block modes (1 = SL)
    uint8_t* qxi;           // [T][H][W] bound codes
    uint32_t* sym;          // [T][H][W] residual symbols, u | v << 16
    int* xi_out;            // optional [T][H][W] integer bounds
    unsigned* qslot;        // [queue_len] ready queue of prep units of the launch (global unit id + 1, 0 = not yet filled)
    unsigned* qtail;        // next queue position to fill
    int* status;            // device status word of the launch (0 = ok)
    unsigned long long* counters;  // [4]: substep vertices, substeps, SL blocks, spare
    int H, W, T;
    int eps_int;
    int pred;               // 0 3DL, 1 SL, 2 MoP, 3 learned
    NetDev net;             // learned predictor parameters (pred 3)
    int B, n;               // MoP block side (divides 32) and sampling stride
    int nby, nbx;
    int nchunks;            // ceil(W / 32)
    int U;                  // side of a prep unit (8 for SL; 16, or 32 for MoP blocks of 32)
    int nur, nuc;           // prep units per slice: rows, columns
    unsigned n_units;       // prep units of this field ((T - 1) * nur * nuc), 0 = no prep stage
    unsigned unit_base;     // global id of this field's first prep unit in the launch's queue
    unsigned queue_len;     // prep units of the whole launch (every field)
    const unsigned long long* log2tab;  // [kLog2Tab] Q32 binary logarithms
    int R;                  // rows/columns of slice t-1 a prep tile may read beyond itself
    float cfl_x, cfl_y;  // binary32 CFL numbers of the SL predictor
    int t_end;              // slices >= t_end are not encoded (their units are not queued)
    long long timeout_ns;
    // Decoding: the same pipeline rebuilds qhat from a stream.  cls then holds
    // (bound code, residual symbols u | v << 16) and qd the verbatim values,
    // both strip-diagonal; MoP block modes come from the stream's bits.
    int decode;
    const uint8_t* mode_bits;  // [ceil(T * nby * nbx / 8)] 1 = SL block (decode)
};

// One launch of the encoder pipeline over one or more fields (a batch): the
// wavefront items of every field in one ticket order and one ready queue of
// prep units.  Each field's items keep their relative order, so every item
// still waits only for items with smaller tickets.
struct PipeArgs {
    SliceArgs one;            // the field of a single-field launch (read from parameter space)
    const SliceArgs* fields;  // [nfields] device copies
    int nfields;
    const int4* order;        // [total_items] (field, t, s, 0) in ticket order
    unsigned total_items;
    unsigned* ticket;         // wavefront item counter
    unsigned* qhead;          // next queue position to take
    unsigned queue_len;       // prep units of every field
    int* status;              // device status word (0 = ok)
    long long timeout_ns;
    int prep_warps;           // layout 0: warps working the prep queue (the first ones of the grid)
    int prep_per_cta;         // layout 1: warps of each CTA working the prep queue (the first ones)
    int mixed;                // 0: every warp has a slot of one size, whole CTAs per role;
                              // 1: prep and wave slots of their own sizes in every CTA
    unsigned slot_bytes;      // layout 0: bytes of a warp's slot
    int wave_cap;             // layout 0: wave warps per CTA at most (0 = all; the others idle)
    unsigned skip_item;       // failure injection: the ticket of a wave that never runs (~0u = none)
};

// Scheduling parameters of the encoder pipeline.  They order and place the
// work only; the output does not depend on them.
struct PipeTuning {
    int prep_share;    // percent of the warps working prep units (0 = default for the predictor)
    int sl_unit;       // side of a pure-SL prep unit: 8 or 16 (0 = default 8)
    int slice_weight;  // slice weight of the ticket order without prep units (0 = default)
    int slack;         // extra slice weight of the ticket order with prep units (0 = default)
    int warps_per_sm;  // worker warps per SM (0 = as many as shared memory and registers allow)
    int mixed;         // 1: prep and wave warps in every CTA, each with a slot of its own size;
                       // 0: whole CTAs per role, every slot the size of the larger one;
                       // w >= 2: as 0 with at most w wave warps working in a CTA
};

// Canonical Huffman decoding tables of one stream (device pointers).
struct HuffDecode {
    const uint32_t* words;          // code words, two zero words of padding after nwords
    unsigned long long nwords;
    unsigned long long nsym;
    const unsigned long long* chunk_off;  // bit offset of every kChunkSyms-th symbol
    const uint32_t* lut;            // [4096] (symbol << 5) | length for codes of <= 12 bits, else 0
    const uint32_t* first;          // [25] first code of each length
    const uint32_t* count;          // [25] codes of each length
    const uint32_t* base;           // [25] index of the first symbol of each length in `sorted`
    const uint32_t* sorted;         // symbols ordered by (length, symbol)
    // [4096] for each 12-bit window, the complete codes at its start (up to
    // three): count | total length << 2 | symbol k << (7 + 16 k); count 0 =
    // the first code is longer than 12 bits
    const unsigned long long* lut3;
};

// k_field.cu
void launch_range(const float* uv, size_t n, RangePartial* part, int nblocks, cudaStream_t s);
void launch_to_fixed(const float* uv, size_t n, int k, int32_t* q, int nblocks, cudaStream_t s);  // q = rint(x 2^k)
// over slices [t_first, t_first + t_count) of a [T][H][W] field (default: all)
void launch_face_masks(const int32_t* q, int H, int W, int T, uint16_t* mask, unsigned long long* ncrossed,
                       cudaStream_t s, int t_first = 0, int t_count = -1);
void launch_verify(const int32_t* qhat, const uint16_t* mask, const float* uv, int H, int W, int T, int k,
                   VerifyOut* out, cudaStream_t s, int t_first = 0, int t_count = -1);
// repair of a failed verification: flags (zeroed before) of the vertices of
// changed faces and of vertices past the bound (qhat untagged); the flagged
// vertices' classification set to lossless (strip-diagonal cls)
void launch_repair_flags(const int32_t* qhat, const float* uv, const uint16_t* m_orig, const uint16_t* m_rec, int H,
                         int W, int T, int k, double bound, uint8_t* flags, cudaStream_t s);
void launch_force_lossless(const uint8_t* flags, int H, int W, int T, int2* cls, cudaStream_t s);

// k_encode.cu
// out, out_m and qd in the strip-diagonal layout (see SliceArgs), zeroed before
void launch_classify(const int32_t* q, const uint16_t* mask, int H, int W, int T, int eps_int, int2* out,
                     unsigned* out_m, int2* qd, cudaStream_t s, int t_first = 0, int t_count = -1);
inline size_t diag_elems(int H, int W, int T) { return (size_t)T * ((H + 31) / 32) * (W + 31) * 32; }
// zeroes the entries of launch_classify's three strip-diagonal outputs that
// hold no vertex (slices [0, T)); launch_classify over [0, T) writes the rest
void launch_diag_pad(int2* cls, unsigned* cls_m, int2* qd, int H, int W, int T, cudaStream_t s);
cudaError_t launch_encode_pipeline(const PipeArgs& p, int pred, int nsm, const PipeTuning& tune, cudaStream_t s);
void launch_log2_table(unsigned long long* tab, int n, cudaStream_t s);
constexpr int kLog2Tab = 4097;  // counts of at most 2 * 32 * 32 sampled symbols

// k_entropy.cu
size_t scan_temp_elems(size_t n);
void launch_exclusive_scan_u64(unsigned long long* data, size_t n, unsigned long long* tmp, cudaStream_t s);
// compaction in tiles: counts per tile, then (after an exclusive scan of the
// tile counts, with one extra element for the total) the scatter
size_t compact_tiles(size_t N);
void launch_tile_count(const uint8_t* qxi, const uint32_t* sym, size_t N, unsigned long long* tile_cnt,
                       cudaStream_t s);
void launch_pack_bits(const uint8_t* in, size_t n, uint8_t* out, cudaStream_t s);
// decoder: tiled expansion of Q_d and L_d, then the strip-diagonal layout
void launch_dec_tile_qd(const uint8_t* qxi, size_t N, unsigned long long* tile_cnt, int* status, cudaStream_t s);
void launch_dec_tile_sym(const uint8_t* qxi, size_t N, const uint16_t* qd, size_t n_qd,
                         const unsigned long long* qd_off, uint32_t* sym, unsigned long long* tile_ld, int* status,
                         cudaStream_t s);
void launch_dec_tile_raw(const uint8_t* qxi, const uint32_t* sym, size_t N, const int32_t* ld, size_t n_ld,
                         const unsigned long long* ld_off, int2* dcs, int2* raw, int* status, cudaStream_t s);
void launch_diag_transpose(const int2* a_in, const int2* b_in, int H, int W, int T, int2* a_out, int2* b_out,
                           cudaStream_t s);
void launch_tile_scatter(const uint8_t* qxi, const uint32_t* sym, const int32_t* q,
                         const unsigned long long* tile_off, size_t N, uint16_t* qd_out, int32_t* ld_out,
                         cudaStream_t s);
void launch_hist_u8(const uint8_t* x, size_t n, unsigned* hist /*33*/, cudaStream_t s);
void launch_hist_u16(const uint16_t* x, size_t n, unsigned* hist /*65536*/, cudaStream_t s);
// code table entries: (code << 5) | len, len <= 24
void launch_tile_bits_u8(const uint8_t* x, size_t n, const uint32_t* table, unsigned long long* tile_bits,
                         cudaStream_t s);
void launch_tile_bits_u16(const uint16_t* x, size_t n, const uint32_t* table, unsigned long long* tile_bits,
                          cudaStream_t s);
void launch_encode_u8(const uint8_t* x, size_t n, const uint32_t* table, const unsigned long long* tile_off,
                      uint32_t* words, cudaStream_t s);
void launch_encode_u16(const uint16_t* x, size_t n, const uint32_t* table, const unsigned long long* tile_off,
                       uint32_t* words, cudaStream_t s);
// k_decode.cu
void launch_huff_decode_u8(const HuffDecode& h, uint8_t* out, int* status, cudaStream_t s);
void launch_huff_decode_u16(const HuffDecode& h, uint16_t* out, int* status, cudaStream_t s);
void launch_untag(int2* qhat, size_t N, cudaStream_t s);  // reconstruction words -> values
// q_hat 2^-k; tagged: the words still carry the reconstruction tag
void launch_to_float(const int2* qhat, size_t N, int k, float* out, cudaStream_t s, bool tagged = false);

// k_traj.cu
void launch_iota(unsigned* x, size_t n, cudaStream_t s);
void launch_face_count(const uint16_t* mask, size_t N, unsigned long long* cnt, cudaStream_t s);
void launch_face_compact(const uint16_t* mask, const unsigned long long* off, size_t N, unsigned long long* fid,
                         cudaStream_t s);
void launch_tet_link(const uint16_t* mask, const unsigned long long* off, int H, int W, int T, unsigned* par,
                     unsigned* deg, unsigned* adj, unsigned long long* bad, cudaStream_t s);
void launch_uf_flatten(unsigned* par, size_t n, cudaStream_t s);
void launch_crossing_points(const int32_t* q, const unsigned long long* fid, size_t n, int H, int W, double* xyt,
                            cudaStream_t s);

// learned predictor (an extension; the paper has none)
struct NetTrainPtrs {
    float* fwd;      // kNetDevFloats: bfloat16-rounded weights in the NetDev layout
    float* bwd2;     // [32][9][32]: transposed, flipped layer-2 weights (input gradient)
    float* bwd3;     // [2][9][32]: the same for layer 3
    uint16_t* bits;  // kNetParams: the bfloat16 model
};
constexpr int kNetPartRec = kNetC * kNetC * 9 + kNetC;  // largest per-block gradient record
void launch_net_predict(const NetDev& nd, const int32_t* prev, int H, int W, int32_t* out, cudaStream_t s);
size_t net_train_floats(int n, int H, int W);
int net_wgrad_blocks(int n, int H, int W, int nsm);
cudaError_t launch_net_inputs(const int32_t* prev, const int32_t* next, int n, int H, int W, float* x0, float* d,
                              cudaStream_t s);
cudaError_t net_train_pass(const float* P, float* ws, int n, int H, int W, int nblk, float* part, double* lpart,
                           const NetTrainPtrs& w, float* grad, float* loss_dev, cudaStream_t s);
cudaError_t launch_adam(float* P, float* m, float* v, const float* g, float lr, int step, cudaStream_t s);
cudaError_t launch_net_prep_weights(const float* P, const NetTrainPtrs& w, cudaStream_t s);
NetDev net_dev_view(const float* fwd);

// k_rates.cu (rate diagnostics): bins [L] = maximal zero-code runs of length L
// (1 <= L <= kRunMax), [kRunMax + 1] = longer runs, [0] = their total length
constexpr int kRunMax = 4096;
constexpr int kRunBins = kRunMax + 2;
size_t zero_runs_ws_bytes(size_t n);
cudaError_t launch_zero_runs(const uint16_t* qd, size_t n, unsigned zero_sym, unsigned long long* bins, void* ws,
                             int nsm, cudaStream_t s);

constexpr int kTileSyms = 4096;     // symbols per encode tile
constexpr int kChunkSyms = 16384;   // symbols per decode chunk (stream sync points)

}  // namespace cpt
