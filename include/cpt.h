/*
 * cpt.h - C ABI of the GB300 (sm_103a) critical-point-trajectory-preserving
 * compressor for time-varying 2-D vector fields.
 *
 * The method is that of "Time-Varying Vector Field Compression with Preserved
 * Critical Point Trajectories" (Xia, Li, Jiao, Wang, Liang, Guo): a lossy
 * compressor C and decompressor D (Sec. IV-A) with a pointwise bound
 * ||D(C(x)) - x||_inf <= eps and the face-level critical-point predicate of
 * every space-time face preserved (Eq. 4), hence the track set T(.) of
 * critical-point trajectories preserved (Thm. 1, Thm. 2).
 *
 * Data layout everywhere: float32 [T][H][W][2], u and v interleaved, row
 * major; j (the x axis, column) is the fastest index, then i (y, row), then t.
 * The global space-time vertex id is (t*H + i)*W + j; it orders the vertices
 * for the symbolic perturbation of Sec. III-F.
 *
 * Every function returns a cpt_status (0 = CPT_OK, negative = error); none
 * aborts or traps.  The text of the last error of the calling thread is
 * available from cpt_last_error().  All compute runs in the library's CUDA
 * kernels on the current CUDA device; there is no CPU fallback: without a
 * usable device every compute call returns CPT_ERR_CUDA.
 */
#ifndef CPT_H
#define CPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CPT_OK = 0,
    CPT_ERR_ARG = -1,         /* invalid argument (sizes, bound, non-finite input) */
    CPT_ERR_CUDA = -2,        /* a CUDA call failed or no device is usable */
    CPT_ERR_OOM = -3,         /* host or device allocation failed */
    CPT_ERR_CORRUPT = -4,     /* malformed or truncated stream */
    CPT_ERR_VERIFY = -5,      /* reconstruction changed a face predicate or broke the bound */
    CPT_ERR_TIMEOUT = -6,     /* a kernel's bounded inter-block wait ran out */
    CPT_ERR_UNSUPPORTED = -7  /* option not available in this build */
} cpt_status;

/* Grid of the field.  dx, dy, dt are the spacings used by the semi-Lagrangian
 * predictor (Sec. VI-A, CFL_x = dt/dx * 1/S); 0 means 1. */
typedef struct {
    int32_t H, W, T;
    double dx, dy, dt;
} cpt_dims;

typedef enum { CPT_EB_ABS = 0, CPT_EB_REL = 1 } cpt_eb_mode;

/* Predictors: 3-D Lorenzo (3DL), semi-Lagrangian (SL, Sec. VI-A), the
 * block-wise mixture of both (MoP, Sec. VI), and a learned predictor (an
 * extension; the paper has none): a 3-layer 3x3 convolutional net,
 * 2 -> 32 -> 32 -> 2 channels with ReLU after the first two layers and zero
 * padding at the field boundary, maps the reconstructed slice t-1 scaled by
 * 2^-23 to y, and the prediction of a component is qhat(t-1) +
 * rint(clamp(y, -2, 2) * 2^23).  Its CPT_NET_PARAMS parameters are bfloat16,
 * laid out w1[32][2][3][3] b1[32] w2[32][32][3][3] b2[32] w3[2][32][3][3] b3[2];
 * every output is a chain of float32 fused multiply-adds from the bias over
 * (input channel, ky, kx) in that order, so the encoder, the decoder and any
 * IEEE reimplementation agree bit for bit.  Slice 0 uses 3DL.  The model is
 * stored in the stream.  The learned mixture (CPT_PRED_LEARNED_MOP) chooses
 * per block between 3DL and the net by the MoP rule (Sec. VI-B) with the net
 * in the place of SL: the plain predictor stays the fallback of every block. */
typedef enum {
    CPT_PRED_LORENZO = 0,
    CPT_PRED_SL = 1,
    CPT_PRED_MOP = 2,
    CPT_PRED_LEARNED = 3,
    CPT_PRED_LEARNED_MOP = 4
} cpt_pred;
#define CPT_NET_PARAMS 10434

/* Compression parameters.
 *   mode/eb  : eps = eb (ABS, data units) or eb * (max - min over u and v) (REL)
 *   pred     : predictor
 *   block    : MoP block side B (0 = 16; 4, 8, 16 or 32; also the learned
 *              mixture's); stride: MoP sampling
 *              stride n (0 = 2)
 *   cuda_stream : cudaStream_t to run on (NULL = the legacy default stream)
 *   verify   : nonzero = recompute every face predicate on the reconstruction
 *              and check the pointwise bound before returning (Thm. 1/2)
 *   model    : the learned predictor's parameters (CPT_PRED_LEARNED and
 *              CPT_PRED_LEARNED_MOP; copied by the call)
 *   tune     : nonzero = pick the encoder pipeline's schedule by timing a
 *              few candidates on the first call of each size class (the
 *              choice is cached for the process); 0 = use `schedule`
 *   schedule : the encoder pipeline's schedule when tune is 0; zeros give the
 *              defaults.  [0] percent of the warps that compute predictions
 *              (SL, MoP, learned), [1] side of a pure-SL prediction unit (8
 *              or 16), [2] slice weight of the wave order without prediction
 *              units (3DL), [3] extra slice weight of the wave order with
 *              them, [4] worker warps per SM (0 = as many as shared memory
 *              and registers allow), [5] warp layout: 0 = whole CTAs per role
 *              (every warp slot the larger role's size), 1 = prediction and
 *              wave warps in every CTA, each slot of its own size, w >= 2 =
 *              as 0 with at most w wave warps working per CTA.  The
 *              schedule orders and places work only: the stream does not
 *              depend on it.                                                  */
typedef struct {
    cpt_eb_mode mode;
    double eb;
    cpt_pred pred;
    int32_t block;
    int32_t stride;
    int32_t verify;
    void* cuda_stream;
    const uint16_t* model;  /* host bfloat16 [CPT_NET_PARAMS]: the learned predictor (CPT_PRED_LEARNED) */
    int32_t tune;
    int32_t schedule[6];
    int32_t zstd_level;     /* 0 = off; 1..ZSTD_maxCLevel(): the finished stream is wrapped in a
                             * ZSTD frame on the host (the lossless stage after the Huffman coder,
                             * Alg. 3 lossless_comp); see cpt_zstd_wrap.  The stream inside is
                             * byte for byte the stream without the option. */
    int32_t repair;         /* nonzero: when the verification finds a changed face predicate or a
                             * value past the bound (which exact integer bounds rule out; only a
                             * fault can cause it), the vertices of the changed faces and the
                             * vertices past the bound are stored losslessly and the field is
                             * encoded again, up to 3 rounds (reading R14 of the verification
                             * policy the paper leaves open); the stream returned then verifies.
                             * The slices before the earliest forced vertex encode as before. */
    uint64_t device_budget; /* 0 = no limit; else the device bytes the call may allocate (the
                             * caller's input not counted).  A field whose working set (about
                             * 90 B per vertex) exceeds it is compressed slab by slab: a window of
                             * S + 2 slices (S chosen from the budget, about 70 B per vertex of a
                             * slice) holds the slab, the reconstructed slice before it and the
                             * original slice after it; the bound and residual codes of each
                             * slab go to host memory and the Huffman streams are built from
                             * them in chunks.  The stream is byte for byte the stream of the
                             * in-memory call.  Not with cpt_debug outputs or repair
                             * (CPT_ERR_UNSUPPORTED); CPT_ERR_OOM when one slice does not fit. */
} cpt_params;

/* Statistics of one compression.  ms_stage (CUDA-event time on the library's
 * stream, summed over launches): 0 range+fixed point, 1 face predicates,
 * 2 MoP selection + SL prediction, 3 incident-face bounds, 4 wavefront
 * encode, 5 entropy coding, 6 verification, 7 host (codebook, stream).
 * launches[s] counts the kernels launched for stage s. */
typedef struct {
    double ms_total;
    double ms_stage[8];
    uint32_t launches[8];
    int32_t scale_log2;       /* k: S = 2^k (fixed point) */
    int32_t eps_int;          /* eps' = floor(eps*S - 0.5) */
    double eps;               /* absolute bound in data units */
    uint64_t faces;           /* faces of the space-time mesh */
    uint64_t crossed_faces;   /* |C| */
    uint64_t lossless_vertices;
    uint64_t unpredictable;
    uint64_t sl_blocks, blocks;
    uint64_t n_ld, n_qd;
    uint64_t verify_mismatch_slice;  /* FC_t: slice faces whose predicate changed */
    uint64_t verify_mismatch_slab;   /* FC_s: slab faces whose predicate changed */
    double linf;              /* max |x_hat - x| over both components: the exact largest
                                 difference of the float32 values, rounded once to double
                                 (0 without params->verify) */
    double psnr;              /* 20 log10(value range) - 10 log10(mean squared difference); the
                                 squares are summed in float32 per thread (a statistic, not
                                 bit-reproducible) */
    double ratio;             /* input bytes / output bytes */
    uint64_t out_bytes;
    uint64_t raw_bytes;       /* bytes of the stream before the optional ZSTD frame */
    uint64_t forced_vertices; /* vertices stored losslessly by the repair (cpt_params.repair) */
    int32_t repair_rounds;    /* encodings repeated by the repair (0 = none needed) */
    int32_t reserved0;
} cpt_stats;

/* Optional host outputs of cpt_compress_ex (each pointer may be NULL).
 *   q     int32 [T][H][W][2]  fixed-point input (Alg. 3, Convert_FixedPoint)
 *   qhat  int32 [T][H][W][2]  reconstruction in fixed point
 *   xi    int32 [T][H][W]     per-vertex integer bound of Alg. 4 (0 = lossless)
 *   qxi   uint8 [T][H][W]     bound codes Q_xi
 *   sym   uint16 [T][H][W][2] residual symbols Q_d (0 = unpredictable;
 *                             unspecified where qxi == 0)
 *   mask  uint16 [T][H][W]    crossed-face bits of the 12 faces owned by each vertex
 *   modes uint8 [T][ceil(H/B)][ceil(W/B)]  1 = SL block
 * Rate diagnostics (the code distributions behind the ratios, Sec. VII-E):
 *   qxi_hist  uint32 [33]     counts of the bound codes Q_xi
 *   qd_hist   uint32 [65536]  counts of the residual symbols Q_d (symbol = code
 *                             + 32768; 0 = unpredictable)
 *   zero_runs uint64 [4098]   maximal runs of the zero code (symbol 32768) in
 *                             the Q_d stream (raster order, u then v of each
 *                             vertex that has symbols): [L] runs of length L
 *                             for 1 <= L <= 4096, [4097] longer runs, [0]
 *                             their total length                            */
typedef struct {
    int32_t* q;
    int32_t* qhat;
    int32_t* xi;
    uint8_t* qxi;
    uint16_t* sym;
    uint16_t* mask;
    uint8_t* modes;
    uint32_t* qxi_hist;
    uint32_t* qd_hist;
    uint64_t* zero_runs;
} cpt_debug;

/* Compresses uv (Alg. 3 with Alg. 1, 2, 4 and Sec. VI).
 *   uv        : float32 [T][H][W][2], host or device memory (detected); host
 *               input is copied to the device inside the call
 *   out       : receives a library-allocated host buffer with the stream;
 *               release it with cpt_free
 *   stats     : nullable
 * Errors: CPT_ERR_ARG (H or W < 2, T < 1, eb < 0 or non-finite input),
 * CPT_ERR_OOM, CPT_ERR_CUDA, CPT_ERR_TIMEOUT, CPT_ERR_VERIFY (only when
 * params->verify is set; *out is still produced). */
cpt_status cpt_compress(const float* uv, const cpt_dims* dims, const cpt_params* params,
                        uint8_t** out, size_t* out_bytes, cpt_stats* stats);

/* Statistics of a batch (cpt_compress_batch). */
typedef struct {
    double ms_total;          /* the whole call (CUDA events on the stream) */
    double ms_pipeline;       /* the encoder pipeline launches, summed over groups */
    double ms_tune;           /* schedule candidates timed by the autotuner (0 when cached or off) */
    uint32_t groups;          /* groups of fields (one pipeline launch each) */
    uint32_t launches;        /* kernels launched, autotuning runs excluded */
    int32_t schedule[6];      /* the schedule used (cpt_params.schedule) */
    uint64_t device_budget;   /* device bytes a group may hold */
    uint64_t in_bytes, out_bytes;
    double ms_phase[8];       /* host wall time of each phase up to its synchronisation: 0 input and
                                 range, 1 fixed point, masks and classification, 2 pipeline (and
                                 autotuning), 3 compaction, 4 histograms, 5 code books and tile
                                 counts, 6 stream layout, words and verification, 7 unused */
} cpt_batch_stats;

/* Compresses nfields independent fields with one set of parameters.  Each
 * field's stream is byte for byte the one cpt_compress gives for it alone.
 * The fields are taken in order into groups whose device memory fits
 * device_budget (0 = 60 % of the free device memory; a group holds at least
 * one field); every phase of the method runs for all fields of a group
 * between the same host synchronisations, and the encoder pipeline (Alg. 3's
 * raster loop with its prediction units) of all fields of a group is one
 * persistent launch whose wave items and prediction units come from one
 * ticket order and one ready queue, so small and short fields fill the
 * warps that one field's slice-to-slice dependencies leave idle.
 *   uv[f]       : float32 [T][H][W][2] of field f, host or device
 *   dims[f]     : its grid
 *   out[f]      : receives a library-allocated host buffer (cpt_free each)
 *   stats       : nullable [nfields]; ms_total is the whole call's time,
 *                 ms_stage[4] the shared pipeline launch of the field's group;
 *                 the other ms_stage entries are event intervals on the
 *                 group's one stream, which also hold the other fields'
 *                 launches of the same phase and the host waits between
 *                 phases (ms_phase of batch_stats is the per-phase split)
 *   batch_stats : nullable
 * Errors: as cpt_compress; on any error but CPT_ERR_VERIFY no output is
 * returned (every out[f] is NULL).  CPT_ERR_VERIFY: every stream is
 * returned, and stats tell which field failed. */
cpt_status cpt_compress_batch(const float* const* uv, const cpt_dims* dims, int32_t nfields, const cpt_params* params,
                              size_t device_budget, uint8_t** out, size_t* out_bytes, cpt_stats* stats,
                              cpt_batch_stats* batch_stats);

/* cpt_compress plus optional copies of the intermediate arrays (dbg nullable). */
cpt_status cpt_compress_ex(const float* uv, const cpt_dims* dims, const cpt_params* params,
                           uint8_t** out, size_t* out_bytes, cpt_stats* stats,
                           const cpt_debug* dbg);

/* Decompresses a stream produced by cpt_compress: the decompressor D of the
 * problem statement (Sec. IV-A), whose output x_hat = D(C(x)) keeps every
 * face predicate of the original (the face invariance of Eq. 4) and the
 * pointwise error constraint |x_hat - x| <= eps of the same section.  It
 * repeats Alg. 3's raster loop: each vertex gets the compressor's prediction
 * (Sec. VI) from the values already reconstructed plus its dequantised
 * residual, or its verbatim value.
 *   uv_out : caller-allocated float32 [T][H][W][2], host or device; NULL only
 *            fills dims_out (a cheap header query)
 *   qhat_out : nullable host int32 [T][H][W][2] copy of the fixed-point values
 * Errors: CPT_ERR_CORRUPT for a malformed or truncated stream. */
cpt_status cpt_decompress(const uint8_t* in, size_t in_bytes, float* uv_out, int32_t* qhat_out,
                          cpt_dims* dims_out, void* cuda_stream);

/* Critical-point trajectories of a field (Sec. III-D, Thm. 2): the crossed
 * faces of the space-time mesh joined through the tetrahedra they share.
 *   scale_log2 : fixed-point exponent k to use (as stored in a stream), or
 *                CPT_SCALE_AUTO to derive it from the data
 * Each trajectory lists its faces in path order from its lowest-id end (a
 * closed loop starts at its lowest-id face, towards the lower-id neighbour);
 * trajectories are ordered by their first face id.  Face id = owner vertex id
 * * 12 + face type.  xyt holds the crossing point of each face (Eq. 3) as
 * (x = column, y = row, t).  *out is library-allocated (cpt_free). */
#define CPT_SCALE_AUTO INT32_MIN
typedef struct {
    uint64_t n_traj, n_points;
    uint64_t* offsets;  /* n_traj + 1 */
    uint64_t* face_ids; /* n_points */
    double* xyt;        /* 3 * n_points */
    uint64_t bad_tets;  /* tets with a crossed-face count other than 0 or 2 (Lemma 1) */
} cpt_trajs;

cpt_status cpt_extract_trajectories(const float* uv, const cpt_dims* dims, int32_t scale_log2,
                                    cpt_trajs** out, void* cuda_stream);

/* Range reduction and fixed-point conversion (the first step of
 * cpt_compress) without any device allocation.  The paper has no counterpart:
 * this entry point serves callers that cannot allocate device memory when
 * they call it (a pre-reserved memory pool, an allocator that forbids foreign
 * allocations, a context where cudaMalloc would synchronise the device).
 *   uv         : device float32 [T][H][W][2], 16-byte aligned (read)
 *   q          : device int32 [T][H][W][2], 16-byte aligned (written):
 *                q = rint(x * 2^k)
 *   scale_log2 : device int32 (written): k = 23 - e with max|x| < 2^e, 0 for
 *                an all-zero field, INT32_MIN when a value is not finite (q is
 *                then left untouched)
 * Runs asynchronously on cuda_stream.  Its scratch is a 256 KiB array in
 * device memory that every GPU loading the library holds until the process
 * exits; inputs of more than 16384 * 16384 float values (2*H*W*T) are
 * rejected with CPT_ERR_ARG.  Calls share that array: calls whose kernels
 * overlap on the GPU race and must be serialised by the caller.  The first
 * call on a device looks up the array's address; make it before capturing a
 * stream into a CUDA graph.
 * Errors: CPT_ERR_ARG (null or misaligned pointer, empty or oversized field),
 * CPT_ERR_CUDA. */
cpt_status cpt_fixed_point_noalloc(const float* uv, const cpt_dims* dims, int32_t* q, int32_t* scale_log2,
                                   void* cuda_stream);

/* Learned predictor (an extension; the paper has none).
 *
 * cpt_net_predict: the predictions int32 [H][W][2] of a slice from the
 * reconstructed previous slice prev int32 [H][W][2] (host arrays), computed
 * by the same device code as the compressor's prep units.
 *
 * cpt_net_gradients: loss and gradients of the training objective at the
 * float32 parameters params [CPT_NET_PARAMS] (host): the network runs with
 * params rounded to bfloat16, and the loss is the mean over the n pairs, the
 * H*W vertices and both components of (y - d)^2, where
 * d = clamp((next - prev) * 2^-23, -2, 2); prev and next are int32
 * [n][H][W][2] fixed-point slices (host).  grad_out: host float
 * [CPT_NET_PARAMS] (d loss / d parameter, through the rounding as if it
 * were the identity).
 *
 * cpt_train_predictor: trains the network on the n pairs with Adam
 * (learning rate lr, beta1 0.9, beta2 0.999, epsilon 1e-8) for `steps` full
 * batches, entirely on the GPU, starting from init (host bfloat16, or NULL
 * for a seeded initialisation); writes the bfloat16 model to model_out (host)
 * and, when loss_out is not NULL, the loss before each step (host float
 * [steps]).
 * Errors: CPT_ERR_ARG (sizes < 1, null pointers), CPT_ERR_OOM, CPT_ERR_CUDA. */
cpt_status cpt_net_predict(const uint16_t* model, const int32_t* prev, int32_t H, int32_t W, int32_t* pred_out,
                           void* cuda_stream);
cpt_status cpt_net_gradients(const float* params, const int32_t* prev, const int32_t* next, int32_t n, int32_t H,
                             int32_t W, float* grad_out, float* loss_out, void* cuda_stream);
cpt_status cpt_train_predictor(const int32_t* prev, const int32_t* next, int32_t n, int32_t H, int32_t W,
                               int32_t steps, float lr, uint32_t seed, const uint16_t* init, uint16_t* model_out,
                               float* loss_out, void* cuda_stream);

/* Failure injection for tests of the bounded waits (the paper has no
 * counterpart).  The next compression on the calling thread runs its encoder
 * pipeline without the wave item of this ticket (an index into the pipeline's
 * ticket order) and with every wait limited to timeout_ns: the items that
 * depend on the skipped one wait until the limit, set the kernel's status
 * word and stop, and the call returns CPT_ERR_TIMEOUT with the device left
 * usable.  No fault, trap or unbounded wait is involved.  ticket < 0 clears a
 * pending injection.
 * Errors: CPT_ERR_ARG (ticket >= 2^32 - 1, limit outside [1 ms, 10 s]). */
cpt_status cpt_inject_wave_stall(int64_t ticket, int64_t timeout_ns);

/* Failure injection for tests of the verification (the paper has no
 * counterpart).  The next single-field compression with verification on the
 * calling thread adds delta to the u component of the reconstruction of
 * vertex `vertex` (global id (t*H + i)*W + j) after the encoder pipeline and
 * before the verification, which must then report the changed predicates or
 * the broken bound (CPT_ERR_VERIFY); the stream itself is unaffected.
 * vertex < 0 clears a pending injection.  Always CPT_OK. */
cpt_status cpt_inject_verify_fault(int64_t vertex, int32_t delta);

/* Inspection of the encoder pipeline's schedule (host only, no device work):
 * the order in which the wave items of one launch over nfields fields take
 * their tickets.  A wave item (f, t, s) encodes rows 32s..32s+31 of slice t of
 * field f (Alg. 3's raster loop, one strip); it waits only for items with
 * smaller tickets: the strip above, the strips of slice t-1 under its faces
 * and its Lorenzo stencil, and those that complete the footprint of the
 * prediction units it reads (rows up to 32s + 31 + R of slice t-1).
 *   fields   : [nfields][4] int32: T, H, R (the units' reach, 0 without
 *              units), with_units (0 / 1)
 *   schedule : cpt_params.schedule or NULL (defaults)
 *   items    : [n_items][3] int32 (field, t, s) in ticket order, or NULL to
 *              query n_items only
 * Errors: CPT_ERR_ARG (null fields or n_items, T or H < 1, R < 0, 2^31 items
 * or more). */
cpt_status cpt_pipeline_order(int32_t nfields, const int32_t* fields, const int32_t* schedule, int32_t* items,
                              uint64_t* n_items);

/* The code lengths of the library's entropy stage (host only): an optimal
 * prefix code with no code longer than maxlen for the symbol frequencies
 * freq[nsym] (package-merge; symbols of frequency 0 get length 0, a single
 * used symbol length 1).  The stream's canonical codes follow from these
 * lengths (Sec. VII-E, the Huffman stage of the lossless back end).
 * Errors: CPT_ERR_ARG (null arrays with nsym > 0, maxlen outside [1, 32], more
 * used symbols than 2^maxlen). */
cpt_status cpt_huffman_lengths(const uint64_t* freq, uint32_t nsym, int32_t maxlen, uint8_t* len);

/* Releases a buffer returned by cpt_compress(_ex) or a cpt_trajs (deep). */
/* Optional lossless back end (Alg. 3, lossless_comp: the general-purpose
 * lossless stage after the Huffman coder; the paper uses ZSTD).  Host only,
 * no GPU needed.  libzstd.so.1 is loaded at run time; without it both calls
 * return CPT_ERR_UNSUPPORTED.
 * cpt_zstd_wrap: in (any bytes, normally a stream of cpt_compress) becomes
 *   the container "CPTZ", u32 version 1, u64 in_bytes, one ZSTD frame
 *   (little-endian); level 1..ZSTD_maxCLevel(), else CPT_ERR_ARG.
 * cpt_zstd_unwrap: the bytes inside such a container; CPT_ERR_CORRUPT when
 *   in is not one or its frame does not decode to the stated size.
 * *out is library-allocated (cpt_free).  cpt_decompress accepts containers
 * directly.  Compression with cpt_params.zstd_level > 0 returns the
 * container; cpt_stats.raw_bytes is then the size of the stream inside. */
cpt_status cpt_zstd_wrap(const uint8_t* in, size_t in_bytes, int32_t level, uint8_t** out, size_t* out_bytes);
cpt_status cpt_zstd_unwrap(const uint8_t* in, size_t in_bytes, uint8_t** out, size_t* out_bytes);

void cpt_free(void* p);
void cpt_free_trajs(cpt_trajs* t);

const char* cpt_error_string(cpt_status s);
const char* cpt_last_error(void);

/* Library version (stream format version in the low byte). */
uint32_t cpt_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CPT_H */
