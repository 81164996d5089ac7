// Host side of the library: the C ABI (include/cpt.h), argument checks, device
// buffers, the launch schedule of the compressor (Alg. 3), the canonical
// Huffman codebooks and the byte stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <tuple>
#include <mutex>
#include <unordered_map>
#include <string>
#include <thread>
#include <vector>

#include "cpt.h"
#include "cpt_internal.h"

namespace cpt {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static cpt_status fail(cpt_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}
cpt_status fail_status(cpt_status s, const char* msg) { return fail(s, msg); }

// cpt_zstd.cu: the optional ZSTD container of a finished stream (host only)
bool is_zstd_container(const uint8_t* in, size_t n);
cpt_status zstd_wrap(const uint8_t* in, size_t n, int level, uint8_t** out, size_t* out_n);
cpt_status zstd_unwrap(const uint8_t* in, size_t n, uint8_t** out, size_t* out_n);

#define CPT_CUDA(call)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) {                                                                        \
            return fail(e_ == cudaErrorMemoryAllocation ? CPT_ERR_OOM : CPT_ERR_CUDA,                   \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                            \
        }                                                                                               \
    } while (0)

// ---------------------------------------------------------------------------
// stream-ordered device buffers
// ---------------------------------------------------------------------------
struct DevArena {
    cudaStream_t s;
    std::vector<void*> ptrs;
    explicit DevArena(cudaStream_t st) : s(st) {}
    ~DevArena() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t n) {
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(n * sizeof(T), 16), s);
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = static_cast<T*>(q);
        return e;
    }
};

static void retain_pool_memory() {
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return;
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    });
}

// ---------------------------------------------------------------------------
// stage timing with CUDA events on the library stream
// ---------------------------------------------------------------------------
struct StageTimer {
    cudaStream_t s;
    bool on;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    int open_stage = -1;
    cudaEvent_t open_ev = nullptr;
    StageTimer(cudaStream_t st, bool enable) : s(st), on(enable) {}
    ~StageTimer() {
        for (auto& r : recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
        if (open_ev) cudaEventDestroy(open_ev);
    }
    void begin(int stage) {
        if (!on) return;
        end();  // a stage still open ends here
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
        cudaEventRecord(e, s);
        open_stage = stage;
        open_ev = e;
    }
    void end() {
        if (!on || open_stage < 0) return;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
        cudaEventRecord(e, s);
        recs.push_back({open_stage, open_ev, e});
        open_stage = -1;
        open_ev = nullptr;
    }
    void collect(cpt_stats* st) {
        if (!on || !st) return;
        for (auto& r : recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) st->ms_stage[r.stage] += ms;
        }
    }
};

// ---------------------------------------------------------------------------
// canonical length-limited Huffman codebook (package-merge)
// ---------------------------------------------------------------------------
// Leaves are ordered by (weight, symbol).  Level 0 holds the leaves; level l
// merges the leaves with the pairwise sums of level l-1 (a leaf before a
// package of equal weight).  Selecting the 2n-2 cheapest items of the last
// level, a leaf's code length is the number of levels whose selection reaches
// it; the selection of level l-1 is twice the packages selected at level l.
static bool huffman_lengths(const std::vector<uint64_t>& freq, int maxlen, std::vector<uint8_t>& len) {
    const size_t A = freq.size();
    len.assign(A, 0);
    std::vector<uint32_t> order;
    for (uint32_t s = 0; s < A; ++s)
        if (freq[s]) order.push_back(s);
    const size_t n = order.size();
    if (n == 0) return true;
    if (n == 1) { len[order[0]] = 1; return true; }
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) {
        return freq[a] != freq[b] ? freq[a] < freq[b] : a < b;
    });
    if ((size_t)1 << maxlen < n) return false;
    std::vector<std::vector<uint8_t>> is_leaf(maxlen);
    std::vector<uint64_t> lvl_w, next_w;
    lvl_w.reserve(2 * n);
    next_w.reserve(2 * n);
    for (size_t a = 0; a < n; ++a) lvl_w.push_back(freq[order[a]]);
    is_leaf[0].assign(n, 1);
    for (int l = 1; l < maxlen; ++l) {
        const size_t npk = lvl_w.size() / 2;
        next_w.clear();
        std::vector<uint8_t>& fl = is_leaf[l];
        fl.clear();
        size_t a = 0, b = 0;
        while (a < n || b < npk) {
            const bool take_leaf = a < n && (b == npk || freq[order[a]] <= lvl_w[2 * b] + lvl_w[2 * b + 1]);
            if (take_leaf) { next_w.push_back(freq[order[a]]); fl.push_back(1); ++a; }
            else { next_w.push_back(lvl_w[2 * b] + lvl_w[2 * b + 1]); fl.push_back(0); ++b; }
        }
        lvl_w.swap(next_w);
    }
    size_t sel = 2 * n - 2;
    for (int l = maxlen - 1; l >= 0 && sel > 0; --l) {
        size_t leaves = 0;
        for (size_t x = 0; x < sel; ++x) leaves += is_leaf[l][x];
        for (size_t x = 0; x < leaves; ++x) len[order[x]]++;
        sel = 2 * (sel - leaves);
    }
    return true;
}

// table entry (code << 5) | len; symbols of one length get consecutive codes
// in symbol order, shorter lengths first
static void canonical_table(const std::vector<uint8_t>& len, std::vector<uint32_t>& table) {
    table.assign(len.size(), 0);
    uint32_t count[33] = {0};
    for (uint8_t l : len) count[l]++;
    count[0] = 0;
    uint32_t next[33] = {0};
    uint32_t code = 0;
    for (int l = 1; l <= 32; ++l) {
        code = (code + count[l - 1]) << 1;
        next[l] = code;
    }
    for (size_t s = 0; s < len.size(); ++s)
        if (len[s]) table[s] = (next[len[s]]++ << 5) | len[s];
}

// ---------------------------------------------------------------------------
// byte stream (little endian)
// ---------------------------------------------------------------------------
// Little-endian writer into a buffer sized in advance.
struct Writer {
    uint8_t* p;
    size_t n = 0;
    void u32(uint32_t x) { for (int k = 0; k < 4; ++k) p[n++] = (uint8_t)(x >> (8 * k)); }
    void u64(uint64_t x) { u32((uint32_t)x); u32((uint32_t)(x >> 32)); }
    void f64(double d) { uint64_t x; std::memcpy(&x, &d, 8); u64(x); }
    void raw(const void* src, size_t m) { std::memcpy(p + n, src, m); n += m; }
};

// CFL number of the SL predictor: dt / (dx * S) with S = 2^k, rounded once to
// binary32 (the precision of the back-trace).
static float sl_cfl(double dt, double dx, int k) { return (float)std::ldexp(dt / dx, -k); }

// Reach of the SL back-trace into slice t-1 (rows and columns around a unit)
// when no reconstruction exceeds qmax in magnitude.  The exact displacement
// is at most qmax * CFL; the binary32 evaluation adds at most a few units in
// the last place to the bilinear sums (relative < 2^-20 altogether) and to
// the positions (< 2^-8 of a cell over 32 substeps); the bilinear stencil
// adds one cell and one more cell covers those roundings.  A clamped position
// never leaves the domain, so max(H, W) + 2 always suffices.
static int sl_reach(double qmax, float cfl_x, float cfl_y, int H, int W) {
    const double c = std::max((double)cfl_x, (double)cfl_y);
    const double reach = std::ceil(qmax * c * (1.0 + std::ldexp(1.0, -20))) + 2.0;
    return (int)std::min(reach, (double)std::max(H, W) + 2.0);
}

static constexpr uint32_t kMaxCodeLen = 24;
static constexpr long long kOrderStrip = 32;         // wave ticket order: strip weight
static constexpr long long kOrderSliceLorenzo = 2;   // slice weight without prep units
static constexpr long long kOrderSlackPrep = 64;     // extra slice weight with prep units
static constexpr int kRadius = 32768;  // quantisation radius (symbol = c + kRadius)
static constexpr uint32_t kFormat = 1;

// ---------------------------------------------------------------------------
// Pinned host memory.  Streams returned to the caller live in page-locked
// blocks the library keeps (device copies into them run at full speed and
// touch no fresh pages); cpt_free hands a block back for the next call.  A
// per-thread staging block carries the small host <-> device exchanges of the
// entropy stage.
// ---------------------------------------------------------------------------
class PinnedPool {
    std::mutex mu_;
    std::unordered_map<void*, size_t> live_;
    std::multimap<size_t, void*> idle_;
    size_t idle_bytes_ = 0;
    static constexpr size_t kKeepIdle = (size_t)8 << 30;  // a batch's streams are reused by the next batch

  public:
    void* get(size_t n) {
        n = (n + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
        std::lock_guard<std::mutex> g(mu_);
        auto it = idle_.lower_bound(n);
        if (it != idle_.end() && it->first <= 2 * n) {
            void* p = it->second;
            live_[p] = it->first;
            idle_bytes_ -= it->first;
            idle_.erase(it);
            return p;
        }
        void* p = nullptr;
        if (cudaMallocHost(&p, n) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        live_[p] = n;
        return p;
    }
    bool put(void* p) {
        std::lock_guard<std::mutex> g(mu_);
        auto it = live_.find(p);
        if (it == live_.end()) return false;
        idle_.emplace(it->second, p);
        idle_bytes_ += it->second;
        live_.erase(it);
        while (idle_bytes_ > kKeepIdle && !idle_.empty()) {  // release the smallest idle blocks
            auto f = idle_.begin();
            idle_bytes_ -= f->first;
            cudaFreeHost(f->second);
            idle_.erase(f);
        }
        return true;
    }
};
static PinnedPool& pinned_pool() {
    static PinnedPool* pool = new PinnedPool();  // never destroyed: may outlive the CUDA context
    return *pool;
}

struct Staging {
    void* p = nullptr;
    size_t n = 0;
    void* get(size_t need) {
        if (need <= n) return p;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        if (cudaMallocHost(&p, need) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return nullptr;
        }
        n = need;
        return p;
    }
};
static thread_local Staging t_staging;

// A CUDA event owned by a host thread (created on first use).
struct EventHolder {
    cudaEvent_t ev = nullptr;
};

// The decoder's second stream and its fork/join events, one set per host
// thread (created on first use, kept for the thread's lifetime).
struct DecodeSide {
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool ready() {
        if (!s2 && cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) s2 = nullptr;
        if (!ev_fork && cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess) ev_fork = nullptr;
        if (!ev_join && cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess) ev_join = nullptr;
        if (!s2 || !ev_fork || !ev_join) {
            cudaGetLastError();
            return false;
        }
        return true;
    }
};

// One Huffman stream: host-side code book and the device buffers of its
// tile offsets and words.
struct StreamPlan {
    size_t nsym = 0;
    uint32_t alphabet = 0;
    std::vector<uint32_t> entries;  // (symbol << 8) | length of the used symbols, in symbol order
    uint32_t* d_table = nullptr;    // [alphabet] (code << 5) | length
    unsigned long long* d_tiles = nullptr;
    unsigned long long* d_tmp = nullptr;
    size_t nt = 0;
    uint64_t nwords = 0;
    std::vector<uint64_t> chunk_off;
    uint32_t* d_words = nullptr;
    size_t header_bytes() const { return 8 + 4 + 4 + 4 * entries.size() + 8 * chunk_off.size() + 8; }
};

// Code lengths, the code book entries and the code table (into table_h:
// pinned [alphabet], later copied to the device) of a stream from its
// histogram.  Host only, touches nothing but sp and table_h (thread safe).
static bool build_codebook(StreamPlan& sp, const unsigned* hist, uint32_t* table_h) {
    std::vector<uint64_t> freq(sp.alphabet);
    for (uint32_t k = 0; k < sp.alphabet; ++k) freq[k] = hist[k];
    std::vector<uint8_t> len;
    if (!huffman_lengths(freq, kMaxCodeLen, len)) return false;
    std::vector<uint32_t> table;
    canonical_table(len, table);
    sp.entries.clear();
    for (uint32_t sy = 0; sy < sp.alphabet; ++sy)
        if (len[sy]) sp.entries.push_back((sy << 8) | len[sy]);
    std::memcpy(table_h, table.data(), sizeof(uint32_t) * sp.alphabet);
    return true;
}

static void write_stream_header(Writer& w, const StreamPlan& sp) {
    w.u64(sp.nsym);
    w.u32((uint32_t)sp.entries.size());
    w.u32((uint32_t)kChunkSyms);
    for (uint32_t e : sp.entries) w.u32(e);
    for (uint64_t o : sp.chunk_off) w.u64(o);
    w.u64(sp.nwords);
}

// bfloat16 bits -> float (exact)
static float bf16_to_float(uint16_t h) {
    const uint32_t x = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &x, 4);
    return f;
}

// The learned predictor's parameters on the device: float, each layer's
// weights transposed to [ci][ky][kx][co] (see NetDev).  d: kNetDevFloats.
static cpt_status upload_net_f32(const float* m, float* d, NetDev* nd, cudaStream_t s) {
    std::vector<float> h(kNetDevFloats);
    size_t o = 0, src = 0;
    auto layer = [&](int cin, int cout, const float** wt, const float** b) {
        const size_t wo = o;
        for (int co = 0; co < cout; ++co)
            for (int ci = 0; ci < cin; ++ci)
                for (int k = 0; k < 9; ++k) h[wo + ((size_t)ci * 9 + k) * cout + co] = m[src++];
        o += (size_t)cin * 9 * cout;
        const size_t bo = o;
        for (int co = 0; co < cout; ++co) h[o++] = m[src++];
        *wt = d + wo;
        *b = d + bo;
    };
    layer(2, kNetC, &nd->w1t, &nd->b1);
    layer(kNetC, kNetC, &nd->w2t, &nd->b2);
    layer(kNetC, 2, &nd->w3t, &nd->b3);
    CPT_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(float) * kNetDevFloats, cudaMemcpyHostToDevice, s));
    CPT_CUDA(cudaStreamSynchronize(s));  // h is released on return
    return CPT_OK;
}

static cpt_status upload_net(const uint16_t* model, float* d, NetDev* nd, cudaStream_t s) {
    std::vector<float> m(kNetParams);
    for (int x = 0; x < kNetParams; ++x) m[x] = bf16_to_float(model[x]);
    return upload_net_f32(m.data(), d, nd, s);
}

static bool is_device_pointer(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------------------
// the encoder pipeline's ticket order (also used to decode)
// ---------------------------------------------------------------------------
// Ticket keys of a field's wavefront items (t, s): Ks s + Kt t, then t.  A
// wave depends on the waves above it and, through its prep units, on slice
// t-1 down to (31 + R) / 32 strips below it, so Kt exceeds Ks times that with
// prep units (Kt > Ks * strips below); without them any Kt > 0 keeps
// dependencies at smaller tickets, and a small Kt lets consecutive slices run
// a few steps apart.
static void pipeline_keys(int T, int nstrips, int R, unsigned n_units, const PipeTuning& tune,
                          std::vector<long long>& key) {
    const long long below = (31 + R) / 32;
    const long long slack = tune.slack > 0 ? tune.slack : kOrderSlackPrep;
    const long long kl = tune.slice_weight > 0 ? tune.slice_weight : kOrderSliceLorenzo;
    const long long Kt = n_units > 0 ? kOrderStrip * below + slack : kl;
    key.resize((size_t)T * nstrips);
    for (int t = 0; t < T; ++t)
        for (int sx = 0; sx < nstrips; ++sx) key[(size_t)t * nstrips + sx] = kOrderStrip * sx + Kt * t;
}

// The wave items of one pipeline launch in ticket order: each field's items
// by its own key, merged by key (then field, then t), so every field keeps
// its own relative order.  Item x is (field, t, strip, 0).
struct OrderField {
    int T, nstrips, R;
    unsigned n_units;
};
static void merged_order(const std::vector<OrderField>& fs, const PipeTuning& tune, std::vector<int4>& order) {
    struct Item { long long key; int f, t, sx; };
    std::vector<Item> items;
    size_t total = 0;
    for (const OrderField& g : fs) total += (size_t)g.T * g.nstrips;
    items.reserve(total);
    std::vector<long long> key;
    for (int f = 0; f < (int)fs.size(); ++f) {
        const OrderField& g = fs[f];
        pipeline_keys(g.T, g.nstrips, g.R, g.n_units, tune, key);
        for (int t = 0; t < g.T; ++t)
            for (int sx = 0; sx < g.nstrips; ++sx) items.push_back({key[(size_t)t * g.nstrips + sx], f, t, sx});
    }
    std::stable_sort(items.begin(), items.end(), [](const Item& p, const Item& q) {
        if (p.key != q.key) return p.key < q.key;
        if (p.f != q.f) return p.f < q.f;
        return p.t < q.t;
    });
    order.resize(items.size());
    for (size_t x = 0; x < items.size(); ++x) order[x] = make_int4(items[x].f, items[x].t, items[x].sx, 0);
}

// The decoder's schedule (its prediction units carry no MoP decisions and its
// waves no face work).
static const PipeTuning kDecodeSchedule = {0, 0, 0, 0, 0, 0};

// ---------------------------------------------------------------------------
// compression (Alg. 3)
// ---------------------------------------------------------------------------
// Argument checks shared by the in-memory and the slab-by-slab compressor.
static cpt_status check_args(const cpt_dims& d, const cpt_params* prm) {
    if (d.H < 2 || d.W < 2 || d.T < 1) return fail(CPT_ERR_ARG, "need H >= 2, W >= 2, T >= 1");
    if ((long long)d.H * d.W > (1ll << 31) / 4) return fail(CPT_ERR_ARG, "slice too large");
    if (!(prm->eb >= 0) || !std::isfinite(prm->eb)) return fail(CPT_ERR_ARG, "error bound must be finite and >= 0");
    if (prm->pred < CPT_PRED_LORENZO || prm->pred > CPT_PRED_LEARNED_MOP) return fail(CPT_ERR_ARG, "unknown predictor");
    const bool net = prm->pred == CPT_PRED_LEARNED || prm->pred == CPT_PRED_LEARNED_MOP;
    const bool modes = prm->pred == CPT_PRED_MOP || prm->pred == CPT_PRED_LEARNED_MOP;
    if (net && !prm->model) return fail(CPT_ERR_ARG, "the learned predictor needs a model");
    const int B = prm->block > 0 ? prm->block : 16;
    if (B < 2 || B > 32) return fail(CPT_ERR_ARG, "block side must be in [2, 32]");
    if (modes && (32 % B != 0 || B < 4)) return fail(CPT_ERR_UNSUPPORTED, "MoP block side must be 4, 8, 16 or 32");
    return CPT_OK;
}

// Failure injection for tests (per host thread): the next compression adds
// delta to the u component of one reconstructed vertex before verification.
struct VerifyFault {
    long long vertex = -1;
    int delta = 0;
};
static thread_local VerifyFault t_vfault;

// One field of a compression call.  Its work is split at the host
// synchronisations of the method (range -> fixed-point scale; compaction
// totals; histograms -> code books; tile offsets -> stream layout), so that a
// call over many fields runs each phase for every field before it waits once,
// and runs the encoder pipeline of all its fields in one launch.  A field's
// kernels, their order and their arguments are the same whether it is
// compressed alone or in a batch.
struct FieldJob {
    // inputs
    const float* uv = nullptr;
    cpt_dims dims{};
    const cpt_params* prm = nullptr;
    const cpt_debug* dbg = nullptr;
    cudaStream_t s = nullptr;
    DevArena ar;
    StageTimer tm;
    cpt_stats st{};
    // derived sizes and options
    int H = 0, W = 0, T = 0, B = 16, nstride = 2;
    double dx = 1, dy = 1, dt = 1;
    size_t N = 0, NV = 0;
    bool has_net = false, has_modes = false, want_sl = false;
    // pinned small host values (assigned by run_jobs)
    RangePartial* part_h = nullptr;  // [rblocks]
    unsigned long long* small_h = nullptr;  // [0] last count, [1] last offset, [2..9] counters
    VerifyOut* vo_h = nullptr;
    // phase results
    const float* d_uv = nullptr;
    RangePartial* d_part = nullptr;
    int rblocks = 0;
    float mn = 0, mx = 0, am = 0;
    int k = 0, eps_int = 0;
    double eps = 0;
    int32_t *d_q = nullptr, *d_qhat = nullptr;
    uint16_t* d_mask = nullptr;
    unsigned long long* d_cnt64 = nullptr;  // [0] crossed faces, [1..4] encoder counters
    uint8_t *d_qxi = nullptr, *d_modes = nullptr, *d_mbits = nullptr;
    uint32_t* d_sym = nullptr;
    int* d_xiout = nullptr;
    int2 *d_psl = nullptr, *d_cls = nullptr, *d_qdiag = nullptr;
    unsigned* d_clsm = nullptr;
    size_t nprep_alloc = 0;
    int nby = 0, nbx = 0, nstrips = 0;
    double qmax = 0;  // bound on |reconstruction| for the semi-Lagrangian reach
    SliceArgs a{};
    unsigned long long *d_off = nullptr, *d_stmp = nullptr;
    size_t n_qd = 0, n_ld = 0, nblk = 0, mode_bytes = 0;
    uint16_t* d_qd = nullptr;
    int32_t* d_ld = nullptr;
    StreamPlan sx, sd;
    unsigned* d_hist = nullptr;
    size_t st_hist = 0, st_modes = 0, st_tab = 0, st_toff = 0;
    uint8_t* stage_h = nullptr;  // pinned staging of the entropy stage (assigned by run_jobs)
    VerifyOut* d_vo = nullptr;
    uint8_t* obuf = nullptr;
    bool obuf_pinned = false;
    size_t total = 0;
    VerifyFault vfault;  // failure injection (tests)
    const uint8_t* force_h = nullptr;  // repair: [N] host flags of vertices to store losslessly

    FieldJob(cudaStream_t st_, bool timing) : s(st_), ar(st_), tm(st_, timing) { std::memset(&st, 0, sizeof(st)); }
    ~FieldJob() { release_output(); }
    void release_output() {
        if (obuf && !(obuf_pinned && pinned_pool().put(obuf))) std::free(obuf);
        obuf = nullptr;
    }
    size_t staging_bytes() const { return st_hist + st_modes + st_tab + st_toff + 64; }
    // device bytes a field holds at its peak (for grouping a batch)
    static size_t device_bytes(const cpt_dims& d, bool host_input) {
        const size_t n = (size_t)d.H * d.W * d.T;
        return n * (84 + (host_input ? 8 : 0)) + ((size_t)64 << 20);
    }

    // ---- phase 0: argument checks, input on the device, range partials
    cpt_status begin(int nsm) {
        if (!uv) return fail(CPT_ERR_ARG, "null argument");
        H = dims.H; W = dims.W; T = dims.T;
        const cpt_status ca = check_args(dims, prm);
        if (ca != CPT_OK) return ca;
        has_net = prm->pred == CPT_PRED_LEARNED || prm->pred == CPT_PRED_LEARNED_MOP;
        has_modes = prm->pred == CPT_PRED_MOP || prm->pred == CPT_PRED_LEARNED_MOP;
        B = prm->block > 0 ? prm->block : 16;
        nstride = prm->stride > 0 ? prm->stride : 2;
        dx = dims.dx > 0 ? dims.dx : 1.0;
        dy = dims.dy > 0 ? dims.dy : 1.0;
        dt = dims.dt > 0 ? dims.dt : 1.0;
        N = (size_t)H * W * T;
        NV = 2 * N;
        // input on the device, 16-byte aligned
        d_uv = uv;
        if (!is_device_pointer(uv) || (reinterpret_cast<uintptr_t>(uv) & 15u)) {
            float* tmp;
            CPT_CUDA(ar.alloc(&tmp, NV));
            CPT_CUDA(cudaMemcpyAsync(tmp, uv, NV * sizeof(float), cudaMemcpyDefault, s));
            d_uv = tmp;
        }
        // ---- stage 0: range, scale, fixed point
        tm.begin(0);
        rblocks = nsm * 4;
        CPT_CUDA(ar.alloc(&d_part, rblocks));
        launch_range(d_uv, NV, d_part, rblocks, s);
        st.launches[0]++;
        CPT_CUDA(cudaMemcpyAsync(part_h, d_part, sizeof(RangePartial) * rblocks, cudaMemcpyDeviceToHost, s));
        return CPT_OK;
    }

    // ---- phase 1 (after the range partials arrived): scale and bound,
    // fixed point, crossed-face masks, the pipeline's buffers and arguments,
    // incident-face classification
    cpt_status plan(int nsm, const unsigned long long* d_log2, const NetDev* net, const PipeTuning& tune) {
        mn = INFINITY; mx = -INFINITY; am = 0.f;
        unsigned bad = 0;
        for (int x = 0; x < rblocks; ++x) {
            const RangePartial& p = part_h[x];
            mn = std::min(mn, p.mn); mx = std::max(mx, p.mx); am = std::max(am, p.amax); bad |= p.bad;
        }
        if (bad) return fail(CPT_ERR_ARG, "input holds a non-finite value");
        k = 0;
        if (am > 0.f) { int e; std::frexp((double)am, &e); k = 23 - e; }
        eps = prm->mode == CPT_EB_REL ? prm->eb * ((double)mx - (double)mn) : prm->eb;
        const double ef = std::floor(std::ldexp(eps, k) - 0.5);
        eps_int = !(ef > 0) ? 0 : (ef > 8388608.0 ? 8388608 : (int)ef);
        st.scale_log2 = k;
        st.eps_int = eps_int;
        st.eps = eps;
        CPT_CUDA(ar.alloc(&d_q, NV));
        CPT_CUDA(ar.alloc(&d_qhat, NV));
        launch_to_fixed(d_uv, NV, k, d_q, nsm * 8, s);
        st.launches[0]++;
        tm.end();

        // ---- stage 1: crossed-face masks (C)
        tm.begin(1);
        CPT_CUDA(ar.alloc(&d_mask, N));
        CPT_CUDA(ar.alloc(&d_cnt64, 8));
        CPT_CUDA(cudaMemsetAsync(d_cnt64, 0, 8 * sizeof(unsigned long long), s));
        launch_face_masks(d_q, H, W, T, d_mask, d_cnt64, s);
        st.launches[1]++;
        tm.end();

        // ---- the encoder pipeline's buffers (MoP / SL, incident-face bounds, wavefront)
        nby = (H + B - 1) / B;
        nbx = (W + B - 1) / B;
        nstrips = (H + 31) / 32;
        const int nchunks = (W + 31) / 32;
        want_sl = prm->pred != CPT_PRED_LORENZO && T > 1 && eps_int > 0;
        CPT_CUDA(ar.alloc(&d_qxi, N));
        CPT_CUDA(ar.alloc(&d_modes, (size_t)T * nby * nbx));
        CPT_CUDA(ar.alloc(&d_sym, N));
        const size_t ND = diag_elems(H, W, T);  // strip-diagonal layout, zero padding
        CPT_CUDA(ar.alloc(&d_cls, ND));
        CPT_CUDA(ar.alloc(&d_clsm, ND));
        CPT_CUDA(ar.alloc(&d_qdiag, ND));
        // classification writes every vertex's entry; only the padding is zeroed
        launch_diag_pad(d_cls, d_clsm, d_qdiag, H, W, T, s);
        CPT_CUDA(ar.alloc(&d_psl, want_sl ? N : 1));
        if (dbg && dbg->xi) CPT_CUDA(ar.alloc(&d_xiout, N));
        CPT_CUDA(cudaMemsetAsync(d_modes, 0, (size_t)T * nby * nbx, s));
        SliceArgs& A = a;
        std::memset(&A, 0, sizeof(A));
        A.q = reinterpret_cast<const int2*>(d_q);
        A.qhat = reinterpret_cast<int2*>(d_qhat);
        A.mask = d_mask;
        A.cls = d_cls;
        A.cls_m = d_clsm;
        A.qd = d_qdiag;
        A.psl = d_psl;
        A.modes = d_modes;
        A.qxi = d_qxi;
        A.sym = d_sym;
        A.xi_out = d_xiout;
        A.counters = d_cnt64 + 1;
        A.H = H; A.W = W; A.T = T;
        A.t_end = T;
        A.eps_int = eps_int;
        A.pred = (int)prm->pred;
        A.B = B; A.n = nstride; A.nby = nby; A.nbx = nbx;
        A.nchunks = nchunks;
        A.cfl_x = sl_cfl(dt, dx, k);
        A.cfl_y = sl_cfl(dt, dy, k);
        // Reach of the semi-Lagrangian back-trace into slice t-1: no
        // reconstruction exceeds max|q| + E in magnitude, every displacement is
        // at most that times CFL, the bilinear stencil adds one cell, and one
        // more cell covers rounding of the positions.
        A.R = 0;
        if (want_sl && has_net) {
            A.R = kNetReach;  // the net's receptive field: 3 cells around a vertex
        } else if (want_sl) {
            qmax = std::ceil((double)am * std::ldexp(1.0, k)) +
                   (eps_int > 0 ? std::ldexp(1.0, (int)std::floor(std::log2((double)eps_int))) : 0.0);
            A.R = sl_reach(qmax, A.cfl_x, A.cfl_y, H, W);
        }
        if (has_net) A.net = *net;
        A.log2tab = d_log2;
        // prep units (SL and MoP): U x U squares of slices 1..T-1; the ready
        // queue is sized for the smallest unit a schedule may pick
        const int Umin = has_modes ? (B == 32 ? 32 : 16) : 8;
        nprep_alloc = (size_t)T * ((H + Umin - 1) / Umin) * ((W + Umin - 1) / Umin);
        cpt_status rc = set_units(tune);
        if (rc != CPT_OK) return rc;

        tm.begin(3);
        launch_classify(d_q, d_mask, H, W, T, eps_int, d_cls, d_clsm, d_qdiag, s);
        st.launches[3]++;
        if (force_h) {  // repair: the flagged vertices are stored losslessly
            uint8_t* d_force;
            CPT_CUDA(ar.alloc(&d_force, N));
            CPT_CUDA(cudaMemcpyAsync(d_force, force_h, N, cudaMemcpyHostToDevice, s));
            launch_force_lossless(d_force, H, W, T, d_cls, s);
            st.launches[3]++;
        }
        tm.end();
        return CPT_OK;
    }

    // Repair (after a failed verification): ORs into flags_h [N] the vertices
    // of the faces whose predicate the reconstruction changed and the
    // vertices past the pointwise bound.
    cpt_status repair_flags(uint8_t* flags_h) {
        int32_t* d_rec;
        uint16_t* d_mrec;
        uint8_t* d_fl;
        unsigned long long* d_n;
        CPT_CUDA(ar.alloc(&d_rec, NV));
        CPT_CUDA(ar.alloc(&d_mrec, N));
        CPT_CUDA(ar.alloc(&d_fl, N));
        CPT_CUDA(ar.alloc(&d_n, 1));
        CPT_CUDA(cudaMemcpyAsync(d_rec, d_qhat, NV * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        launch_untag(reinterpret_cast<int2*>(d_rec), N, s);
        CPT_CUDA(cudaMemsetAsync(d_n, 0, sizeof(unsigned long long), s));
        CPT_CUDA(cudaMemsetAsync(d_fl, 0, N, s));
        launch_face_masks(d_rec, H, W, T, d_mrec, d_n, s);
        const double bound = std::max(eps, std::ldexp(0.5, -k));
        launch_repair_flags(d_rec, d_uv, d_mask, d_mrec, H, W, T, k, bound, d_fl, s);
        std::vector<uint8_t> fl(N);
        CPT_CUDA(cudaMemcpyAsync(fl.data(), d_fl, N, cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaStreamSynchronize(s));
        for (size_t v = 0; v < N; ++v) flags_h[v] |= fl[v];
        return CPT_OK;
    }

    // Side of the prep units under a schedule: MoP blocks fit whole units
    // (16, or 32 for B = 32); pure SL and the learned predictor use 8 unless
    // the schedule asks for 16 (pure SL).
    cpt_status set_units(const PipeTuning& tune) {
        SliceArgs& A = a;
        int U = has_modes ? (B == 32 ? 32 : 16) : 8;
        if (prm->pred == CPT_PRED_SL && tune.sl_unit == 16) U = 16;
        A.U = U;
        A.nur = (H + U - 1) / U;
        A.nuc = (W + U - 1) / U;
        A.n_units = 0;
        if (want_sl) {
            const unsigned long long nu = (unsigned long long)(T - 1) * A.nur * A.nuc;
            if (nu >= 0x7FFFFFFFull) return fail(CPT_ERR_UNSUPPORTED, "too many prediction units");
            A.n_units = (unsigned)nu;
        }
        return CPT_OK;
    }

    // Resets what the encoder pipeline reads and writes back (before every launch).
    cpt_status reset_pipeline() {
        CPT_CUDA(cudaMemsetAsync(d_qhat, 0, NV * sizeof(int32_t), s));  // no reconstruction word present
        if (want_sl) CPT_CUDA(cudaMemsetAsync(d_psl, 0, N * sizeof(int2), s));  // no prediction word present
        CPT_CUDA(cudaMemsetAsync(d_cnt64 + 1, 0, 4 * sizeof(unsigned long long), s));
        return CPT_OK;
    }

    // ---- phase 2 (after the pipeline): compaction counts
    cpt_status compact() {
        tm.begin(5);
        const size_t nt = compact_tiles(N);
        CPT_CUDA(ar.alloc(&d_off, nt + 1));
        CPT_CUDA(ar.alloc(&d_stmp, scan_temp_elems(nt + 1)));
        CPT_CUDA(cudaMemsetAsync(d_off + nt, 0, sizeof(unsigned long long), s));
        launch_tile_count(d_qxi, d_sym, N, d_off, s);
        launch_exclusive_scan_u64(d_off, nt + 1, d_stmp, s);  // [nt]: the totals
        small_h[0] = 0;
        CPT_CUDA(cudaMemcpyAsync(&small_h[1], d_off + nt, 8, cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaMemcpyAsync(&small_h[2], d_cnt64, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        return CPT_OK;
    }

    // ---- phase 3 (after the totals arrived): scatter, histograms
    cpt_status scatter_hist() {
        const unsigned long long tot = small_h[1] + small_h[0];
        n_qd = (size_t)(tot >> 32);
        n_ld = (size_t)(tot & 0xFFFFFFFFull);
        CPT_CUDA(ar.alloc(&d_qd, n_qd));
        CPT_CUDA(ar.alloc(&d_ld, n_ld));
        launch_tile_scatter(d_qxi, d_sym, d_q, d_off, N, d_qd, d_ld, s);
        // both streams advance together: histograms (+ block modes) -> code books
        // and tile bit counts -> layout of the output -> words, copied straight
        // into the caller's buffer
        sx.nsym = N;
        sx.alphabet = 33;
        sd.nsym = n_qd;
        sd.alphabet = 2 * kRadius;
        nblk = has_modes ? (size_t)T * nby * nbx : 0;
        mode_bytes = (nblk + 7) / 8;
        if (nblk) {  // the stream's mode bits, packed on the device
            CPT_CUDA(ar.alloc(&d_mbits, mode_bytes));
            launch_pack_bits(d_modes, nblk, d_mbits, s);
        }
        CPT_CUDA(ar.alloc(&d_hist, sx.alphabet + sd.alphabet));
        CPT_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(unsigned) * (sx.alphabet + sd.alphabet), s));
        launch_hist_u8(d_qxi, N, d_hist, s);
        launch_hist_u16(d_qd, n_qd, d_hist + sx.alphabet, s);
        sx.nt = (sx.nsym + kTileSyms - 1) / kTileSyms;
        sd.nt = (sd.nsym + kTileSyms - 1) / kTileSyms;
        // staging: histograms | block modes | tables | tile offsets
        st_hist = sizeof(unsigned) * (sx.alphabet + sd.alphabet);
        st_modes = (mode_bytes + 15) & ~(size_t)15;
        st_tab = sizeof(uint32_t) * (sx.alphabet + sd.alphabet);
        st_toff = sizeof(unsigned long long) * (sx.nt + 1 + sd.nt + 1);
        return CPT_OK;
    }
    cpt_status copy_hist() {
        unsigned* hist_h = reinterpret_cast<unsigned*>(stage_h);
        uint8_t* modes_h = stage_h + st_hist;
        CPT_CUDA(cudaMemcpyAsync(hist_h, d_hist, st_hist, cudaMemcpyDeviceToHost, s));
        if (nblk) CPT_CUDA(cudaMemcpyAsync(modes_h, d_mbits, mode_bytes, cudaMemcpyDeviceToHost, s));
        return CPT_OK;
    }

    // ---- phase 4 (after the histograms arrived): code books, tile bit counts
    // host part (thread safe across fields): both code books from the histograms
    bool host_codebooks() {
        const unsigned* hist_h = reinterpret_cast<const unsigned*>(stage_h);
        uint32_t* tab_h = reinterpret_cast<uint32_t*>(stage_h + st_hist + st_modes);
        return build_codebook(sx, hist_h, tab_h) && build_codebook(sd, hist_h + sx.alphabet, tab_h + sx.alphabet);
    }
    cpt_status codebooks() {
        unsigned* hist_h = reinterpret_cast<unsigned*>(stage_h);
        uint32_t* tab_h = reinterpret_cast<uint32_t*>(stage_h + st_hist + st_modes);
        unsigned long long* toff_h = reinterpret_cast<unsigned long long*>(stage_h + st_hist + st_modes + st_tab);
        for (StreamPlan* sp : {&sx, &sd}) {
            CPT_CUDA(ar.alloc(&sp->d_table, sp->alphabet));
            CPT_CUDA(ar.alloc(&sp->d_tiles, sp->nt + 1));
            CPT_CUDA(ar.alloc(&sp->d_tmp, scan_temp_elems(sp->nt + 1)));
        }
        if (dbg && dbg->qxi_hist) std::memcpy(dbg->qxi_hist, hist_h, sizeof(unsigned) * sx.alphabet);
        if (dbg && dbg->qd_hist) std::memcpy(dbg->qd_hist, hist_h + sx.alphabet, sizeof(unsigned) * sd.alphabet);
        CPT_CUDA(cudaMemcpyAsync(sx.d_table, tab_h, sizeof(uint32_t) * sx.alphabet, cudaMemcpyHostToDevice, s));
        CPT_CUDA(cudaMemcpyAsync(sd.d_table, tab_h + sx.alphabet, sizeof(uint32_t) * sd.alphabet,
                                 cudaMemcpyHostToDevice, s));
        for (StreamPlan* sp : {&sx, &sd})
            CPT_CUDA(cudaMemsetAsync(sp->d_tiles, 0, sizeof(unsigned long long) * (sp->nt + 1), s));
        launch_tile_bits_u8(d_qxi, sx.nsym, sx.d_table, sx.d_tiles, s);
        launch_tile_bits_u16(d_qd, sd.nsym, sd.d_table, sd.d_tiles, s);
        launch_exclusive_scan_u64(sx.d_tiles, sx.nt + 1, sx.d_tmp, s);
        launch_exclusive_scan_u64(sd.d_tiles, sd.nt + 1, sd.d_tmp, s);
        CPT_CUDA(cudaMemcpyAsync(toff_h, sx.d_tiles, sizeof(unsigned long long) * (sx.nt + 1), cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaMemcpyAsync(toff_h + sx.nt + 1, sd.d_tiles, sizeof(unsigned long long) * (sd.nt + 1),
                                 cudaMemcpyDeviceToHost, s));
        return CPT_OK;
    }

    // ---- stage 6: verification (Eq. 4 on every face, pointwise bound),
    // launched once the histograms are on their way to the host, so that it
    // runs while the host builds the code books; its result is read after the
    // call's last synchronisation
    cpt_status verify_launch() {
        std::memset(vo_h, 0, sizeof(VerifyOut));
        if (prm->verify && vfault.vertex >= 0 && (size_t)vfault.vertex < N) {
            // failure injection (tests): one corrupted reconstruction word
            int2 w;
            int2* p = reinterpret_cast<int2*>(d_qhat) + vfault.vertex;
            CPT_CUDA(cudaMemcpyAsync(&w, p, sizeof(int2), cudaMemcpyDeviceToHost, s));
            CPT_CUDA(cudaStreamSynchronize(s));
            w.x += vfault.delta;
            CPT_CUDA(cudaMemcpyAsync(p, &w, sizeof(int2), cudaMemcpyHostToDevice, s));
            CPT_CUDA(cudaStreamSynchronize(s));
        }
        if (prm->verify) {
            const int open = tm.open_stage;  // the entropy stage, timed apart from the verification
            tm.begin(6);
            CPT_CUDA(ar.alloc(&d_vo, 1));
            CPT_CUDA(cudaMemsetAsync(d_vo, 0, sizeof(VerifyOut), s));
            launch_verify(d_qhat, d_mask, d_uv, H, W, T, k, d_vo, s);
            st.launches[6]++;
            CPT_CUDA(cudaMemcpyAsync(vo_h, d_vo, sizeof(VerifyOut), cudaMemcpyDeviceToHost, s));
            tm.end();
            if (open >= 0) tm.begin(open);
        }
        return CPT_OK;
    }

    // ---- phase 5 (after the tile offsets arrived): layout, header, words,
    // debug copies
    cpt_status write_stream() {
        const uint8_t* mbits_h = stage_h + st_hist;  // block modes as bits (packed on the device)
        const unsigned long long* toff_h =
            reinterpret_cast<const unsigned long long*>(stage_h + st_hist + st_modes + st_tab);
        for (size_t b = 0; b < mode_bytes; ++b) st.sl_blocks += (uint64_t)__builtin_popcount(mbits_h[b]);
        {
            const unsigned long long* to = toff_h;
            for (StreamPlan* sp : {&sx, &sd}) {
                sp->nwords = (to[sp->nt] + 31) / 32;
                const size_t per_chunk = kChunkSyms / kTileSyms;
                sp->chunk_off.clear();
                for (size_t c = 0; c * kChunkSyms < sp->nsym; ++c) sp->chunk_off.push_back(to[c * per_chunk]);
                to += sp->nt + 1;
            }
        }
        // layout: header | mode bits | model | stream Q_xi | stream Q_d | L_d
        const size_t kHeaderBytes = 4 + 11 * 4 + 4 * 8 + 8 + 8;
        const size_t model_bytes = has_net ? 4 + 4 * (size_t)((kNetParams + 1) / 2) : 0;
        const size_t off_x = kHeaderBytes + mode_bytes + model_bytes;
        const size_t off_xw = off_x + sx.header_bytes();
        const size_t off_d = off_xw + 4 * sx.nwords;
        const size_t off_dw = off_d + sd.header_bytes();
        const size_t off_ld = off_dw + 4 * sd.nwords;
        total = off_ld + 4 * n_ld;
        obuf = static_cast<uint8_t*>(pinned_pool().get(total));
        obuf_pinned = obuf != nullptr;
        if (!obuf) obuf = static_cast<uint8_t*>(std::malloc(total));
        if (!obuf) return fail(CPT_ERR_OOM, "host allocation failed");
        Writer w{obuf};
        w.raw("CPT1", 4);
        w.u32(kFormat);
        w.u32((uint32_t)H);
        w.u32((uint32_t)W);
        w.u32((uint32_t)T);
        w.u32((uint32_t)k);
        w.u32((uint32_t)eps_int);
        w.u32((uint32_t)prm->pred);
        w.u32((uint32_t)B);
        w.u32((uint32_t)nstride);
        w.u32((uint32_t)kRadius);
        w.u32(0);
        w.f64(dx);
        w.f64(dy);
        w.f64(dt);
        w.f64(eps);
        w.u64(n_ld);
        w.u64(mode_bytes);
        if (w.n != kHeaderBytes) return fail(CPT_ERR_ARG, "internal: header size");
        if (mode_bytes) w.raw(mbits_h, mode_bytes);
        if (model_bytes) {  // the model: parameter count, then the bfloat16 parameters two per word
            w.u32((uint32_t)kNetParams);
            for (int x = 0; x < kNetParams; x += 2)
                w.u32((uint32_t)prm->model[x] | (x + 1 < kNetParams ? (uint32_t)prm->model[x + 1] << 16 : 0u));
        }
        write_stream_header(w, sx);
        if (w.n != off_xw) return fail(CPT_ERR_ARG, "internal: stream layout");
        w.n = off_d;
        write_stream_header(w, sd);
        if (w.n != off_dw) return fail(CPT_ERR_ARG, "internal: stream layout");
        for (StreamPlan* sp : {&sx, &sd}) {
            CPT_CUDA(ar.alloc(&sp->d_words, sp->nwords + 1));
            CPT_CUDA(cudaMemsetAsync(sp->d_words, 0, sizeof(uint32_t) * (sp->nwords + 1), s));
        }
        launch_encode_u8(d_qxi, sx.nsym, sx.d_table, sx.d_tiles, sx.d_words, s);
        launch_encode_u16(d_qd, sd.nsym, sd.d_table, sd.d_tiles, sd.d_words, s);
        if (sx.nwords) CPT_CUDA(cudaMemcpyAsync(obuf + off_xw, sx.d_words, 4 * sx.nwords, cudaMemcpyDeviceToHost, s));
        if (sd.nwords) CPT_CUDA(cudaMemcpyAsync(obuf + off_dw, sd.d_words, 4 * sd.nwords, cudaMemcpyDeviceToHost, s));
        if (n_ld) CPT_CUDA(cudaMemcpyAsync(obuf + off_ld, d_ld, 4 * n_ld, cudaMemcpyDeviceToHost, s));
        st.launches[5] += 9;
        tm.end();

        // ---- debug copies and rate diagnostics
        if (dbg && dbg->zero_runs) {
            unsigned long long* d_bins;
            uint8_t* d_ws;
            CPT_CUDA(ar.alloc(&d_bins, kRunBins));
            CPT_CUDA(ar.alloc(&d_ws, zero_runs_ws_bytes(n_qd)));
            CPT_CUDA(launch_zero_runs(d_qd, n_qd, (unsigned)kRadius, d_bins, d_ws, sm_count(), s));
            CPT_CUDA(cudaMemcpyAsync(dbg->zero_runs, d_bins, sizeof(unsigned long long) * kRunBins,
                                     cudaMemcpyDeviceToHost, s));
        }
        if (dbg) {
            if (dbg->q) CPT_CUDA(cudaMemcpyAsync(dbg->q, d_q, NV * 4, cudaMemcpyDeviceToHost, s));
            if (dbg->qhat) CPT_CUDA(cudaMemcpyAsync(dbg->qhat, d_qhat, NV * 4, cudaMemcpyDeviceToHost, s));
            if (dbg->xi) CPT_CUDA(cudaMemcpyAsync(dbg->xi, d_xiout, N * 4, cudaMemcpyDeviceToHost, s));
            if (dbg->qxi) CPT_CUDA(cudaMemcpyAsync(dbg->qxi, d_qxi, N, cudaMemcpyDeviceToHost, s));
            if (dbg->mask) CPT_CUDA(cudaMemcpyAsync(dbg->mask, d_mask, N * 2, cudaMemcpyDeviceToHost, s));
            if (dbg->modes)
                CPT_CUDA(cudaMemcpyAsync(dbg->modes, d_modes, (size_t)T * nby * nbx, cudaMemcpyDeviceToHost, s));
            if (dbg->sym) {
                std::vector<uint32_t> tmp(N);
                CPT_CUDA(cudaMemcpyAsync(tmp.data(), d_sym, N * 4, cudaMemcpyDeviceToHost, s));
                CPT_CUDA(cudaStreamSynchronize(s));
                for (size_t v = 0; v < N; ++v) {
                    dbg->sym[2 * v] = (uint16_t)(tmp[v] & 0xFFFFu);
                    dbg->sym[2 * v + 1] = (uint16_t)(tmp[v] >> 16);
                }
            }
        }
        return CPT_OK;
    }

    // ---- phase 6 (after everything arrived): statistics and the verdict
    cpt_status finish(double ms_total, double ms_pipeline, uint8_t** out, size_t* out_bytes, cpt_stats* stats) {
        if (dbg && dbg->qhat)  // reconstruction words -> values
            for (size_t v = 0; v < N; ++v) dbg->qhat[2 * v + 1] ^= kQhatTag;
        tm.collect(&st);
        st.ms_stage[4] += ms_pipeline;
        st.launches[4]++;
        st.ms_total = ms_total;
        {
            const unsigned long long Hl = H, Wl = W, Tl = T;
            const unsigned long long E = Hl * (Wl - 1) + Wl * (Hl - 1) + (Hl - 1) * (Wl - 1);
            st.faces = 2 * (Hl - 1) * (Wl - 1) * Tl + (Tl - 1) * (2 * E + 4 * (Hl - 1) * (Wl - 1));
        }
        st.crossed_faces = small_h[2];
        st.blocks = has_modes ? (uint64_t)T * nby * nbx : 0;
        st.n_ld = n_ld;
        st.n_qd = n_qd;
        st.out_bytes = total;
        st.raw_bytes = total;
        st.ratio = (double)(NV * 4) / (double)total;
        const VerifyOut& vo = *vo_h;
        st.verify_mismatch_slice = vo.mismatch_slice;
        st.verify_mismatch_slab = vo.mismatch_slab;
        double linf;
        std::memcpy(&linf, &vo.linf_bits, 8);
        st.linf = linf;
        if (prm->verify) {
            const double mse = vo.sq_err / (double)NV;
            const double range = (double)mx - (double)mn;
            st.psnr = mse > 0 ? 20.0 * std::log10(range) - 10.0 * std::log10(mse) : INFINITY;
        }
        // lossless vertices: n_ld minus the unpredictable components; n_qd = 2 * (N - lossless)
        st.lossless_vertices = N - n_qd / 2;
        st.unpredictable = n_ld - 2 * st.lossless_vertices;
        if (stats) *stats = st;
        *out = obuf;
        *out_bytes = total;
        obuf = nullptr;  // handed to the caller
        // The pointwise bound holds for eps >= half a fixed-point unit; below that
        // every value is stored losslessly and the error is the rounding to 2^-k.
        const double bound = std::max(eps, std::ldexp(0.5, -k));
        if (prm->verify && (vo.mismatch_slice || vo.mismatch_slab || !(linf <= bound)))
            return fail(CPT_ERR_VERIFY, "reconstruction changed a face predicate or exceeded the bound");
        return CPT_OK;
    }
};

// Failure injection for tests (per host thread): the next compression's
// encoder pipeline skips the wave with this ticket and waits at most this long.
struct WaveStall {
    long long ticket = -1;
    long long timeout_ns = 0;
};
static thread_local WaveStall t_stall;

// Process-wide cache of autotuned schedules, keyed by the predictor, the
// block side and the size class of the launch.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, PipeTuning> g_tune_cache;

// Candidate schedules of the encoder pipeline for a predictor.
static std::vector<PipeTuning> tuning_candidates(int pred) {
    std::vector<PipeTuning> c;
    // {prep share %, pure-SL unit side, 3DL slice weight, slack, warps per SM, layout / wave cap}
    if (pred == CPT_PRED_LORENZO) {
        for (int kl : {1, 2, 8}) c.push_back({0, 0, kl, 0, 3, 0});
        for (int kl : {1, 2, 8}) c.push_back({0, 0, kl, 0, 0, 8});
    } else if (pred == CPT_PRED_SL) {
        // large slices balance the prediction units' throughput against the
        // wave steps (about 45 % of the warps on prediction units); small
        // ones are bound by the lag.  At most 8 working wave warps per CTA
        // keep the wave steps short.
        c.push_back({45, 8, 0, 0, 3, 0});
        for (int u : {8, 16})
            for (int share : {25, 35, 45, 55, 65}) c.push_back({share, u, 0, 0, 0, 0});
        for (int share : {35, 45, 55})
            for (int cap : {4, 8}) c.push_back({share, 8, 0, 0, 0, cap});
    } else if (pred == CPT_PRED_LEARNED) {
        for (int share : {65, 75, 85}) c.push_back({share, 0, 0, 0, 0, 0});
    } else if (pred == CPT_PRED_LEARNED_MOP) {
        for (int share : {65, 75, 85}) c.push_back({share, 0, 0, 64, 0, 0});
    } else {
        c.push_back({45, 0, 0, 64, 3, 0});
        for (int share : {25, 35, 45, 55, 65, 75}) c.push_back({share, 0, 0, 64, 0, 0});
        for (int share : {35, 45, 55, 65})
            for (int cap : {4, 6, 8}) c.push_back({share, 0, 0, 64, 0, cap});
        c.push_back({45, 0, 0, 128, 0, 0});
    }
    return c;
}

// One compression call over jobs[0..n): every phase for every field, one host
// synchronisation between phases, one pipeline launch for all fields.
struct PipeTimes {
    double ms_pipeline = 0, ms_tune = 0;
    PipeTuning used{};
    double ms_phase[8] = {0};  // host wall time of each phase, its synchronisation included
};

static cpt_status run_jobs(FieldJob* const* jobs, int n, const cpt_params* prm, cudaStream_t s, bool tune_req,
                           PipeTuning tune, PipeTimes* times) {
    const int nsm = sm_count();
    auto clk = std::chrono::steady_clock::now();
    auto mark = [&](int phase) {
        const auto now = std::chrono::steady_clock::now();
        if (times) times->ms_phase[phase] += std::chrono::duration<double, std::milli>(now - clk).count();
        clk = now;
    };
    // pinned small values of every field
    const size_t per_rb = sizeof(RangePartial) * (size_t)nsm * 4;
    const size_t per_job = ((per_rb + 15) & ~(size_t)15) + 16 * 8 + sizeof(VerifyOut) + 16;
    static thread_local Staging t_small;
    uint8_t* small = static_cast<uint8_t*>(t_small.get(per_job * (size_t)n));
    if (!small) return fail(CPT_ERR_OOM, "pinned staging allocation failed");
    for (int f = 0; f < n; ++f) {
        uint8_t* b = small + per_job * f;
        jobs[f]->part_h = reinterpret_cast<RangePartial*>(b);
        jobs[f]->small_h = reinterpret_cast<unsigned long long*>(b + ((per_rb + 15) & ~(size_t)15));
        jobs[f]->vo_h = reinterpret_cast<VerifyOut*>(b + ((per_rb + 15) & ~(size_t)15) + 16 * 8);
    }
    for (int f = 0; f < n; ++f) {
        cpt_status rc = jobs[f]->begin(nsm);
        if (rc != CPT_OK) return rc;
    }
    CPT_CUDA(cudaStreamSynchronize(s));
    mark(0);

    // call-wide device state: the log2 table, the learned predictor, the
    // pipeline's queue, ticket and status
    DevArena ar(s);
    unsigned long long* d_lg;
    CPT_CUDA(ar.alloc(&d_lg, kLog2Tab));
    launch_log2_table(d_lg, kLog2Tab, s);
    NetDev net{};
    const bool has_net = prm->pred == CPT_PRED_LEARNED || prm->pred == CPT_PRED_LEARNED_MOP;
    if (has_net) {
        if (!prm->model) return fail(CPT_ERR_ARG, "the learned predictor needs a model");
        float* d_net;
        CPT_CUDA(ar.alloc(&d_net, kNetDevFloats));
        cpt_status rc = upload_net(prm->model, d_net, &net, s);
        if (rc != CPT_OK) return rc;
    }
    for (int f = 0; f < n; ++f) {
        cpt_status rc = jobs[f]->plan(nsm, d_lg, &net, tune);
        if (rc != CPT_OK) return rc;
    }
    mark(1);
    size_t max_queue = 0, max_items = 0;
    for (int f = 0; f < n; ++f) {
        max_queue += jobs[f]->nprep_alloc;
        max_items += (size_t)jobs[f]->T * jobs[f]->nstrips;
    }
    if (max_queue >= 0x7FFFFFFFull || max_items >= 0x7FFFFFFFull)
        return fail(CPT_ERR_UNSUPPORTED, "too many pipeline items in one launch");
    unsigned *d_queue, *d_ticket;
    int* d_status;
    int4* d_order;
    SliceArgs* d_fields;
    CPT_CUDA(ar.alloc(&d_queue, max_queue + 2));
    CPT_CUDA(ar.alloc(&d_ticket, 1));
    CPT_CUDA(ar.alloc(&d_status, 1));
    CPT_CUDA(ar.alloc(&d_order, max_items));
    CPT_CUDA(ar.alloc(&d_fields, (size_t)n));
    std::vector<int4> order;
    std::vector<SliceArgs> fields((size_t)n);
    PipeArgs P{};

    cudaEvent_t e0, e1;
    CPT_CUDA(cudaEventCreate(&e0));
    CPT_CUDA(cudaEventCreate(&e1));
    struct EvG { cudaEvent_t a, b; ~EvG() { cudaEventDestroy(a); cudaEventDestroy(b); } } evg{e0, e1};

    // a pending failure injection applies to this call's launches
    const WaveStall stall = t_stall;
    t_stall = WaveStall{};
    const long long timeout_ns = stall.ticket >= 0 ? stall.timeout_ns : 2000000000ll;

    // Sets up and launches the pipeline over every field under a schedule;
    // *ms: the launch's device time (CUDA events around the kernel).
    auto launch = [&](const PipeTuning& tu, double* ms) -> cpt_status {
        unsigned qlen = 0;
        for (int f = 0; f < n; ++f) {
            cpt_status rc = jobs[f]->set_units(tu);
            if (rc != CPT_OK) return rc;
            jobs[f]->a.unit_base = qlen;
            qlen += jobs[f]->a.n_units;
        }
        // ticket order of the launch
        std::vector<OrderField> ofs((size_t)n);
        for (int f = 0; f < n; ++f) ofs[f] = {jobs[f]->T, jobs[f]->nstrips, jobs[f]->a.R, jobs[f]->a.n_units};
        merged_order(ofs, tu, order);
        for (int f = 0; f < n; ++f) {
            SliceArgs& A = jobs[f]->a;
            A.qslot = d_queue + 2;
            A.qtail = d_queue + 1;
            A.status = d_status;
            A.queue_len = qlen;
            A.timeout_ns = timeout_ns;
            fields[f] = A;
            cpt_status rc = jobs[f]->reset_pipeline();
            if (rc != CPT_OK) return rc;
        }
        CPT_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int4) * order.size(), cudaMemcpyHostToDevice, s));
        CPT_CUDA(cudaMemcpyAsync(d_fields, fields.data(), sizeof(SliceArgs) * n, cudaMemcpyHostToDevice, s));
        CPT_CUDA(cudaMemsetAsync(d_queue, 0, sizeof(unsigned) * ((size_t)qlen + 2), s));
        CPT_CUDA(cudaMemsetAsync(d_ticket, 0, sizeof(unsigned), s));
        CPT_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));
        P.one = fields[0];
        P.fields = d_fields;
        P.nfields = n;
        P.order = d_order;
        P.total_items = (unsigned)order.size();
        P.ticket = d_ticket;
        P.qhead = d_queue;
        P.queue_len = qlen;
        P.status = d_status;
        P.timeout_ns = timeout_ns;
        P.skip_item = stall.ticket >= 0 ? (unsigned)stall.ticket : ~0u;
        CPT_CUDA(cudaEventRecord(e0, s));
        CPT_CUDA(launch_encode_pipeline(P, (int)prm->pred, nsm, tu, s));
        CPT_CUDA(cudaEventRecord(e1, s));
        CPT_CUDA(cudaStreamSynchronize(s));  // the host tables outlive their copies
        float m = 0.f;
        CPT_CUDA(cudaEventElapsedTime(&m, e0, e1));
        *ms = m;
        int status = 0;
        CPT_CUDA(cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost));
        if (status != 0) return fail((cpt_status)status, "wavefront wait timed out");
        return CPT_OK;
    };

    if (tune_req) {
        size_t nv = 0;
        for (int f = 0; f < n; ++f) nv += jobs[f]->N;
        const int cls = (int)std::lround(std::log2((double)std::max<size_t>(nv, 1)));
        const int B0 = jobs[0]->B;
        const auto ck = std::make_tuple((int)prm->pred, B0, cls, n > 1 ? 1 : 0);
        bool hit = false;
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(ck);
            if (it != g_tune_cache.end()) { tune = it->second; hit = true; }
        }
        if (!hit) {
            double best = INFINITY;
            PipeTuning bt{};
            for (const PipeTuning& c : tuning_candidates((int)prm->pred)) {
                double ms = 0;
                cpt_status rc = launch(c, &ms);
                if (rc != CPT_OK) return rc;
                if (times) times->ms_tune += ms;
                if (ms < best) { best = ms; bt = c; }
            }
            tune = bt;
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune_cache[ck] = tune;
        }
    }
    double ms_pipe = 0;
    {
        cpt_status rc = launch(tune, &ms_pipe);
        if (rc != CPT_OK) return rc;
    }
    if (times) {
        times->ms_pipeline = ms_pipe;
        times->used = tune;
    }
    mark(2);
    for (int f = 0; f < n; ++f) {
        cpt_status rc = jobs[f]->compact();
        if (rc != CPT_OK) return rc;
    }
    CPT_CUDA(cudaStreamSynchronize(s));
    mark(3);
    static thread_local EventHolder t_hist_ev;  // the histograms' arrival on the host
    if (!t_hist_ev.ev && cudaEventCreateWithFlags(&t_hist_ev.ev, cudaEventDisableTiming) != cudaSuccess) {
        t_hist_ev.ev = nullptr;
        return fail(CPT_ERR_CUDA, "event creation failed");
    }
    size_t stage_total = 0;
    for (int f = 0; f < n; ++f) {
        cpt_status rc = jobs[f]->scatter_hist();
        if (rc != CPT_OK) return rc;
        stage_total += (jobs[f]->staging_bytes() + 63) & ~(size_t)63;
    }
    uint8_t* stage = static_cast<uint8_t*>(t_staging.get(stage_total));
    if (!stage) return fail(CPT_ERR_OOM, "pinned staging allocation failed");
    for (int f = 0; f < n; ++f) {
        jobs[f]->stage_h = stage;
        stage += (jobs[f]->staging_bytes() + 63) & ~(size_t)63;
        cpt_status rc = jobs[f]->copy_hist();
        if (rc != CPT_OK) return rc;
    }
    CPT_CUDA(cudaEventRecord(t_hist_ev.ev, s));
    for (int f = 0; f < n; ++f) {
        cpt_status rc = jobs[f]->verify_launch();
        if (rc != CPT_OK) return rc;
    }
    CPT_CUDA(cudaEventSynchronize(t_hist_ev.ev));
    mark(4);
    {   // the fields' code books on host threads (package-merge is the host's share of the method)
        const int nth = std::max(1, std::min<int>(n, (int)std::thread::hardware_concurrency()));
        std::vector<char> ok((size_t)n, 1);
        auto work = [&](int w) {
            for (int f = w; f < n; f += nth) ok[f] = jobs[f]->host_codebooks() ? 1 : 0;
        };
        if (nth == 1) {
            work(0);
        } else {
            std::vector<std::thread> pool;
            for (int w = 0; w < nth; ++w) pool.emplace_back(work, w);
            for (auto& th : pool) th.join();
        }
        for (int f = 0; f < n; ++f)
            if (!ok[f]) return fail(CPT_ERR_ARG, "alphabet too large for code length limit");
    }
    for (int f = 0; f < n; ++f) {
        cpt_status rc = jobs[f]->codebooks();
        if (rc != CPT_OK) return rc;
    }
    CPT_CUDA(cudaStreamSynchronize(s));
    mark(5);
    for (int f = 0; f < n; ++f) {
        cpt_status rc = jobs[f]->write_stream();
        if (rc != CPT_OK) return rc;
    }
    CPT_CUDA(cudaStreamSynchronize(s));
    mark(6);
    return CPT_OK;
}

// The optional ZSTD container around a finished stream: replaces *out (the
// stream goes back to the pool) and updates the statistics.
static cpt_status wrap_output(const cpt_params* prm, uint8_t** out, size_t* out_bytes, cpt_stats* stats,
                              size_t input_bytes) {
    if (prm->zstd_level <= 0 || !*out) return CPT_OK;
    uint8_t* z = nullptr;
    size_t zn = 0;
    const cpt_status rc = zstd_wrap(*out, *out_bytes, prm->zstd_level, &z, &zn);
    if (rc != CPT_OK) return rc;
    if (!pinned_pool().put(*out)) std::free(*out);
    *out = z;
    *out_bytes = zn;
    if (stats) {
        stats->out_bytes = zn;
        stats->ratio = (double)input_bytes / (double)zn;
    }
    return CPT_OK;
}

static cpt_status check_device() {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(CPT_ERR_CUDA, "no CUDA device available");
    }
    retain_pool_memory();
    return CPT_OK;
}

static PipeTuning tuning_of(const cpt_params* prm) {
    return PipeTuning{prm->schedule[0], prm->schedule[1], prm->schedule[2], prm->schedule[3], prm->schedule[4],
                      prm->schedule[5]};
}

static cpt_status compress_streamed(const float* uv, const cpt_dims* dims, const cpt_params* prm, uint8_t** out,
                                    size_t* out_bytes, cpt_stats* stats);

static cpt_status compress_impl(const float* uv, const cpt_dims* dims, const cpt_params* prm, uint8_t** out,
                                size_t* out_bytes, cpt_stats* stats, const cpt_debug* dbg) {
    if (!uv || !dims || !prm || !out || !out_bytes) return fail(CPT_ERR_ARG, "null argument");
    cpt_status rc = check_device();
    if (rc != CPT_OK) return rc;
    if (prm->device_budget > 0) {
        rc = check_args(*dims, prm);
        if (rc != CPT_OK) return rc;
        if (FieldJob::device_bytes(*dims, !is_device_pointer(uv)) > prm->device_budget) {
            // the field's working set exceeds the budget: slab by slab
            if (dbg || prm->repair) return fail(CPT_ERR_UNSUPPORTED, "debug outputs and repair need the in-memory call");
            *out = nullptr;
            *out_bytes = 0;
            cudaEvent_t a0, a1;
            CPT_CUDA(cudaEventCreate(&a0));
            CPT_CUDA(cudaEventCreate(&a1));
            cudaStream_t st = static_cast<cudaStream_t>(prm->cuda_stream);
            CPT_CUDA(cudaEventRecord(a0, st));
            rc = compress_streamed(uv, dims, prm, out, out_bytes, stats);
            cudaEventRecord(a1, st);
            cudaEventSynchronize(a1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a0, a1);
            cudaEventDestroy(a0);
            cudaEventDestroy(a1);
            if (stats) stats->ms_total = ms;
            if (rc != CPT_OK && rc != CPT_ERR_VERIFY) return rc;
            const cpt_status rz = wrap_output(prm, out, out_bytes, stats, (size_t)dims->H * dims->W * dims->T * 8);
            if (rz != CPT_OK) {
                cpt_free(*out);
                *out = nullptr;
                *out_bytes = 0;
                return rz;
            }
            return rc;
        }
    }
    cudaStream_t s = static_cast<cudaStream_t>(prm->cuda_stream);
    cudaEvent_t ev0, ev1;
    CPT_CUDA(cudaEventCreate(&ev0));
    CPT_CUDA(cudaEventCreate(&ev1));
    struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } evg{ev0, ev1};
    FieldJob job(s, true);
    job.uv = uv;
    job.dims = *dims;
    job.prm = prm;
    job.dbg = dbg;
    job.vfault = t_vfault;
    t_vfault = VerifyFault{};
    CPT_CUDA(cudaEventRecord(ev0, s));
    FieldJob* jp = &job;
    PipeTimes pt;
    rc = run_jobs(&jp, 1, prm, s, prm->tune != 0, tuning_of(prm), &pt);
    if (rc != CPT_OK) return rc;
    CPT_CUDA(cudaEventRecord(ev1, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    CPT_CUDA(cudaGetLastError());
    float ms_total = 0.f;
    cudaEventElapsedTime(&ms_total, ev0, ev1);
    rc = job.finish(ms_total, pt.ms_pipeline, out, out_bytes, stats);
    if (rc == CPT_ERR_VERIFY && prm->repair) {
        // reading R14: store the vertices of the changed faces (and those past
        // the bound) losslessly and encode again, at most kRepairRounds times
        constexpr int kRepairRounds = 3;
        std::vector<uint8_t> force(job.N, 0);
        cpt_status rf = job.repair_flags(force.data());
        for (int round = 1; rf == CPT_OK && rc == CPT_ERR_VERIFY && round <= kRepairRounds; ++round) {
            cpt_free(*out);
            *out = nullptr;
            *out_bytes = 0;
            FieldJob again(s, true);
            again.uv = uv;
            again.dims = *dims;
            again.prm = prm;
            again.dbg = dbg;
            again.force_h = force.data();
            FieldJob* ap = &again;
            PipeTimes pt2;
            CPT_CUDA(cudaEventRecord(ev0, s));
            rc = run_jobs(&ap, 1, prm, s, prm->tune != 0, tuning_of(prm), &pt2);
            if (rc != CPT_OK) return rc;
            CPT_CUDA(cudaEventRecord(ev1, s));
            CPT_CUDA(cudaStreamSynchronize(s));
            cudaEventElapsedTime(&ms_total, ev0, ev1);
            rc = again.finish(ms_total, pt2.ms_pipeline, out, out_bytes, stats);
            if (stats) {
                stats->repair_rounds = round;
                uint64_t nf = 0;
                for (uint8_t f : force) nf += f;
                stats->forced_vertices = nf;
            }
            if (rc == CPT_ERR_VERIFY && round < kRepairRounds) rf = again.repair_flags(force.data());
        }
        if (rf != CPT_OK) {
            cpt_free(*out);
            *out = nullptr;
            *out_bytes = 0;
            return rf;
        }
    }
    if (rc != CPT_OK && rc != CPT_ERR_VERIFY) return rc;
    const cpt_status rz = wrap_output(prm, out, out_bytes, stats, job.NV * 4);
    if (rz != CPT_OK) {
        cpt_free(*out);
        *out = nullptr;
        *out_bytes = 0;
        return rz;
    }
    return rc;
}

// ---------------------------------------------------------------------------
// Slab-by-slab compression (cpt_params.device_budget below a field's working
// set).  Alg. 3 encodes slice t from slices t-1, t and t+1 only, so the field
// is encoded in slabs of S slices [t0, t1) inside a window of slices
// [t0 - 1, t1]: the reconstruction of slice t0 - 1 (carried from the previous
// slab, with its crossed-face masks), the slab, and the original slice t1.
// The encoder pipeline runs the slab's slices only (SliceArgs::t_end; the
// prediction units of the window's first encoded slice are queued before the
// launch).  Each slab's bound codes, residual symbols and verbatim values go
// to host memory; the histograms add up on the device.  The Huffman streams
// are then built from the host codes in chunks of tiles (tile bit counts,
// one host scan, the words), and laid out exactly as in the in-memory call.
// ---------------------------------------------------------------------------
static constexpr size_t kStreamBytesPerVertexSlice = 72;  // window bytes per vertex of one window slice
static constexpr size_t kStreamChunkSyms = (size_t)1 << 24;  // symbols per entropy chunk (a multiple of the tiles)

struct StreamedField {
    // inputs
    const float* uv;
    cpt_dims dims;
    const cpt_params* prm;
    cudaStream_t s;
    int S;  // slices per slab
    // derived
    int H = 0, W = 0, T = 0, B = 16, nstride = 2;
    double dx = 1, dy = 1, dt = 1;
    size_t HW = 0, N = 0;
    bool has_net = false, has_modes = false, want_sl = false, dev_in = false;
    int k = 0, eps_int = 0;
    double eps = 0;
    float mn = 0, mx = 0, am = 0;
    int nby = 0, nbx = 0, nstrips = 0;
    cpt_stats st{};
};

// the range of u and v over the field, slab by slab through a device buffer
static cpt_status streamed_range(StreamedField& F, DevArena& ar, float* d_win) {
    const int nsm = sm_count();
    const int rblocks = nsm * 4;
    RangePartial* d_part;
    CPT_CUDA(ar.alloc(&d_part, rblocks));
    std::vector<RangePartial> part(rblocks);
    F.mn = INFINITY;
    F.mx = -INFINITY;
    F.am = 0.f;
    unsigned bad = 0;
    const int slab = F.S + 2;
    for (int t0 = 0; t0 < F.T; t0 += slab) {
        const int n = std::min(slab, F.T - t0);
        const size_t nv = 2 * F.HW * n;
        const float* src = F.uv + 2 * F.HW * t0;
        const float* d_src = src;
        if (!F.dev_in || (reinterpret_cast<uintptr_t>(src) & 15u)) {  // 16-byte aligned device copy
            CPT_CUDA(cudaMemcpyAsync(d_win, src, nv * sizeof(float), cudaMemcpyDefault, F.s));
            d_src = d_win;
        }
        launch_range(d_src, nv, d_part, rblocks, F.s);
        CPT_CUDA(cudaMemcpyAsync(part.data(), d_part, sizeof(RangePartial) * rblocks, cudaMemcpyDeviceToHost, F.s));
        CPT_CUDA(cudaStreamSynchronize(F.s));
        for (const RangePartial& p : part) {
            F.mn = std::min(F.mn, p.mn);
            F.mx = std::max(F.mx, p.mx);
            F.am = std::max(F.am, p.amax);
            bad |= p.bad;
        }
    }
    if (bad) return fail(CPT_ERR_ARG, "input holds a non-finite value");
    return CPT_OK;
}

// The Huffman words of one stream from its host symbols, in chunks: tile bit
// counts, one host scan, then each chunk's words (its two edge words OR-ed
// with the neighbouring chunks').  Fills sp.nwords and sp.chunk_off (pass
// 1) or the words (pass 2, words_h: the stream's word region in the output,
// zeroed; any alignment).
template <typename Sym>
static cpt_status streamed_huffman(StreamPlan& sp, const Sym* sym_h, const uint32_t* d_table, Sym* d_chunk,
                                   unsigned long long* d_tiles, uint32_t* d_words, std::vector<unsigned long long>& to,
                                   uint8_t* words_h, cudaStream_t s) {
    const size_t nt = (sp.nsym + kTileSyms - 1) / kTileSyms;
    const size_t per_chunk_tiles = kStreamChunkSyms / kTileSyms;
    if (!words_h) {  // pass 1: tile bit counts and their exclusive scan
        to.assign(nt + 1, 0ull);
        for (size_t c0 = 0; c0 < sp.nsym; c0 += kStreamChunkSyms) {
            const size_t n = std::min(kStreamChunkSyms, sp.nsym - c0);
            const size_t ntc = (n + kTileSyms - 1) / kTileSyms;
            CPT_CUDA(cudaMemcpyAsync(d_chunk, sym_h + c0, n * sizeof(Sym), cudaMemcpyHostToDevice, s));
            if (sizeof(Sym) == 1)
                launch_tile_bits_u8(reinterpret_cast<const uint8_t*>(d_chunk), n, d_table, d_tiles, s);
            else
                launch_tile_bits_u16(reinterpret_cast<const uint16_t*>(d_chunk), n, d_table, d_tiles, s);
            CPT_CUDA(cudaMemcpyAsync(to.data() + c0 / kTileSyms, d_tiles, ntc * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, s));
            CPT_CUDA(cudaStreamSynchronize(s));
        }
        unsigned long long acc = 0;
        for (size_t x = 0; x <= nt; ++x) {
            const unsigned long long b = x < nt ? to[x] : 0ull;
            to[x] = acc;
            acc += b;
        }
        sp.nt = nt;
        sp.nwords = (to[nt] + 31) / 32;
        const size_t per_sync = kChunkSyms / kTileSyms;
        sp.chunk_off.clear();
        for (size_t c = 0; c * kChunkSyms < sp.nsym; ++c) sp.chunk_off.push_back(to[c * per_sync]);
        return CPT_OK;
    }
    std::vector<unsigned long long> rel(per_chunk_tiles);
    std::vector<uint32_t> buf;
    for (size_t c0 = 0; c0 < sp.nsym; c0 += kStreamChunkSyms) {
        const size_t n = std::min(kStreamChunkSyms, sp.nsym - c0);
        const size_t tf = c0 / kTileSyms, ntc = (n + kTileSyms - 1) / kTileSyms;
        const size_t wbase = (size_t)(to[tf] >> 5), wend = (size_t)((to[tf + ntc] + 31) >> 5);
        if (wend <= wbase) continue;  // no bits in this chunk
        for (size_t x = 0; x < ntc; ++x) rel[x] = to[tf + x] - 32ull * wbase;
        CPT_CUDA(cudaMemcpyAsync(d_chunk, sym_h + c0, n * sizeof(Sym), cudaMemcpyHostToDevice, s));
        CPT_CUDA(cudaMemcpyAsync(d_tiles, rel.data(), ntc * sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
        CPT_CUDA(cudaMemsetAsync(d_words, 0, (wend - wbase + 1) * sizeof(uint32_t), s));
        if (sizeof(Sym) == 1)
            launch_encode_u8(reinterpret_cast<const uint8_t*>(d_chunk), n, d_table, d_tiles, d_words, s);
        else
            launch_encode_u16(reinterpret_cast<const uint16_t*>(d_chunk), n, d_table, d_tiles, d_words, s);
        buf.resize(wend - wbase);
        CPT_CUDA(cudaMemcpyAsync(buf.data(), d_words, buf.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaStreamSynchronize(s));
        for (size_t x = 0; x < buf.size(); ++x) {
            uint32_t w;
            std::memcpy(&w, words_h + 4 * (wbase + x), 4);
            w |= buf[x];
            std::memcpy(words_h + 4 * (wbase + x), &w, 4);
        }
    }
    return CPT_OK;
}

// After the slabs: code books from the summed histograms, the two Huffman
// streams from the host codes, and the stream laid out as in the in-memory
// call (FieldJob::write_stream); then the statistics and the verdict.
static cpt_status streamed_finish(StreamedField& F, const cpt_params* prm, DevArena& ar, const unsigned* d_hist,
                                  const unsigned long long* d_cnt64, const VerifyOut* d_vo,
                                  const std::vector<uint8_t>& qxi_h, const std::vector<uint16_t>& qd_h,
                                  const std::vector<int32_t>& ld_h, const std::vector<uint8_t>& modes_h,
                                  uint8_t** out, size_t* out_bytes, cpt_stats* stats) {
    cudaStream_t s = F.s;
    std::vector<unsigned> hist(33 + 2 * kRadius);
    unsigned long long cnt[8];
    VerifyOut vo;
    CPT_CUDA(cudaMemcpyAsync(hist.data(), d_hist, sizeof(unsigned) * hist.size(), cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaMemcpyAsync(cnt, d_cnt64, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaMemcpyAsync(&vo, d_vo, sizeof(VerifyOut), cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    StreamPlan sx, sd;
    sx.nsym = F.N;
    sx.alphabet = 33;
    sd.nsym = qd_h.size();
    sd.alphabet = 2 * kRadius;
    std::vector<uint32_t> tab(33 + 2 * kRadius);
    if (!build_codebook(sx, hist.data(), tab.data()) || !build_codebook(sd, hist.data() + 33, tab.data() + 33))
        return fail(CPT_ERR_ARG, "alphabet too large for code length limit");
    uint32_t *d_tab, *d_words;
    uint16_t* d_chunk;
    unsigned long long* d_tiles;
    CPT_CUDA(ar.alloc(&d_tab, tab.size()));
    CPT_CUDA(ar.alloc(&d_chunk, kStreamChunkSyms));
    CPT_CUDA(ar.alloc(&d_tiles, kStreamChunkSyms / kTileSyms + 1));
    CPT_CUDA(ar.alloc(&d_words, kStreamChunkSyms * kMaxCodeLen / 32 + 64));
    CPT_CUDA(cudaMemcpyAsync(d_tab, tab.data(), sizeof(uint32_t) * tab.size(), cudaMemcpyHostToDevice, s));
    std::vector<unsigned long long> tox, tod;
    cpt_status rc = streamed_huffman<uint8_t>(sx, qxi_h.data(), d_tab, reinterpret_cast<uint8_t*>(d_chunk), d_tiles,
                                              d_words, tox, nullptr, s);
    if (rc == CPT_OK)
        rc = streamed_huffman<uint16_t>(sd, qd_h.data(), d_tab + 33, d_chunk, d_tiles, d_words, tod, nullptr, s);
    if (rc != CPT_OK) return rc;
    // block modes as bits
    const size_t nblk = modes_h.size(), mode_bytes = (nblk + 7) / 8;
    std::vector<uint8_t> packed(mode_bytes, 0);
    cpt_stats& st = F.st;
    for (size_t x = 0; x < nblk; ++x)
        if (modes_h[x]) {
            packed[x >> 3] |= (uint8_t)(1u << (x & 7));
            ++st.sl_blocks;
        }
    // layout: header | mode bits | model | stream Q_xi | stream Q_d | L_d
    const size_t kHeaderBytes = 4 + 11 * 4 + 4 * 8 + 8 + 8;
    const size_t model_bytes = F.has_net ? 4 + 4 * (size_t)((kNetParams + 1) / 2) : 0;
    const size_t off_x = kHeaderBytes + mode_bytes + model_bytes;
    const size_t off_xw = off_x + sx.header_bytes();
    const size_t off_d = off_xw + 4 * sx.nwords;
    const size_t off_dw = off_d + sd.header_bytes();
    const size_t off_ld = off_dw + 4 * sd.nwords;
    const size_t n_ld = ld_h.size();
    const size_t total = off_ld + 4 * n_ld;
    uint8_t* obuf = static_cast<uint8_t*>(pinned_pool().get(total));
    const bool pinned = obuf != nullptr;
    if (!obuf) obuf = static_cast<uint8_t*>(std::malloc(total));
    if (!obuf) return fail(CPT_ERR_OOM, "host allocation failed");
    auto release = [&]() {
        if (!(pinned && pinned_pool().put(obuf))) std::free(obuf);
    };
    Writer w{obuf};
    w.raw("CPT1", 4);
    w.u32(kFormat);
    w.u32((uint32_t)F.H);
    w.u32((uint32_t)F.W);
    w.u32((uint32_t)F.T);
    w.u32((uint32_t)F.k);
    w.u32((uint32_t)F.eps_int);
    w.u32((uint32_t)prm->pred);
    w.u32((uint32_t)F.B);
    w.u32((uint32_t)F.nstride);
    w.u32((uint32_t)kRadius);
    w.u32(0);
    w.f64(F.dx);
    w.f64(F.dy);
    w.f64(F.dt);
    w.f64(F.eps);
    w.u64(n_ld);
    w.u64(mode_bytes);
    if (mode_bytes) w.raw(packed.data(), mode_bytes);
    if (model_bytes) {
        w.u32((uint32_t)kNetParams);
        for (int x = 0; x < kNetParams; x += 2)
            w.u32((uint32_t)prm->model[x] | (x + 1 < kNetParams ? (uint32_t)prm->model[x + 1] << 16 : 0u));
    }
    write_stream_header(w, sx);
    std::memset(obuf + off_xw, 0, 4 * sx.nwords);
    w.n = off_d;
    write_stream_header(w, sd);
    std::memset(obuf + off_dw, 0, 4 * sd.nwords);
    if (w.n != off_dw) {
        release();
        return fail(CPT_ERR_ARG, "internal: stream layout");
    }
    rc = streamed_huffman<uint8_t>(sx, qxi_h.data(), d_tab, reinterpret_cast<uint8_t*>(d_chunk), d_tiles, d_words,
                                   tox, obuf + off_xw, s);
    if (rc == CPT_OK)
        rc = streamed_huffman<uint16_t>(sd, qd_h.data(), d_tab + 33, d_chunk, d_tiles, d_words, tod, obuf + off_dw, s);
    if (rc != CPT_OK) {
        release();
        return rc;
    }
    if (n_ld) std::memcpy(obuf + off_ld, ld_h.data(), 4 * n_ld);
    // statistics, as FieldJob::finish
    {
        const unsigned long long Hl = F.H, Wl = F.W, Tl = F.T;
        const unsigned long long E = Hl * (Wl - 1) + Wl * (Hl - 1) + (Hl - 1) * (Wl - 1);
        st.faces = 2 * (Hl - 1) * (Wl - 1) * Tl + (Tl - 1) * (2 * E + 4 * (Hl - 1) * (Wl - 1));
    }
    st.crossed_faces = cnt[0];
    st.blocks = F.has_modes ? (uint64_t)F.T * F.nby * F.nbx : 0;
    st.n_ld = n_ld;
    st.n_qd = sd.nsym;
    st.out_bytes = total;
    st.raw_bytes = total;
    st.ratio = (double)(F.N * 8) / (double)total;
    st.verify_mismatch_slice = vo.mismatch_slice;
    st.verify_mismatch_slab = vo.mismatch_slab;
    double linf;
    std::memcpy(&linf, &vo.linf_bits, 8);
    st.linf = linf;
    if (prm->verify) {
        const double mse = vo.sq_err / (double)(2 * F.N);
        const double range = (double)F.mx - (double)F.mn;
        st.psnr = mse > 0 ? 20.0 * std::log10(range) - 10.0 * std::log10(mse) : INFINITY;
    }
    st.lossless_vertices = F.N - sd.nsym / 2;
    st.unpredictable = n_ld - 2 * st.lossless_vertices;
    if (stats) *stats = st;
    *out = obuf;
    *out_bytes = total;
    const double bound = std::max(F.eps, std::ldexp(0.5, -F.k));
    if (prm->verify && (vo.mismatch_slice || vo.mismatch_slab || !(linf <= bound)))
        return fail(CPT_ERR_VERIFY, "reconstruction changed a face predicate or exceeded the bound");
    return CPT_OK;
}

static cpt_status compress_streamed(const float* uv, const cpt_dims* dims, const cpt_params* prm, uint8_t** out,
                                    size_t* out_bytes, cpt_stats* stats) {
    cudaStream_t s = static_cast<cudaStream_t>(prm->cuda_stream);
    StreamedField F;
    F.uv = uv;
    F.dims = *dims;
    F.prm = prm;
    F.s = s;
    F.H = dims->H;
    F.W = dims->W;
    F.T = dims->T;
    const int H = F.H, W = F.W, T = F.T;
    F.HW = (size_t)H * W;
    F.N = F.HW * T;
    F.has_net = prm->pred == CPT_PRED_LEARNED || prm->pred == CPT_PRED_LEARNED_MOP;
    F.has_modes = prm->pred == CPT_PRED_MOP || prm->pred == CPT_PRED_LEARNED_MOP;
    F.B = prm->block > 0 ? prm->block : 16;
    F.nstride = prm->stride > 0 ? prm->stride : 2;
    F.dx = dims->dx > 0 ? dims->dx : 1.0;
    F.dy = dims->dy > 0 ? dims->dy : 1.0;
    F.dt = dims->dt > 0 ? dims->dt : 1.0;
    F.dev_in = is_device_pointer(uv);
    const int B = F.B;
    // the slab: what fits the budget after the fixed buffers
    const size_t fixed = (size_t)160 << 20;
    const size_t per_slice = kStreamBytesPerVertexSlice * F.HW;
    if (prm->device_budget <= fixed + 3 * per_slice) return fail(CPT_ERR_OOM, "device budget below one slab of one slice");
    F.S = (int)std::min<size_t>((size_t)T, (prm->device_budget - fixed) / per_slice - 2);
    const int S = F.S, Tw = S + 2;
    DevArena ar(s);
    float* d_uvw;
    CPT_CUDA(ar.alloc(&d_uvw, 2 * F.HW * Tw));
    cpt_status rc = streamed_range(F, ar, d_uvw);
    if (rc != CPT_OK) return rc;
    // scale and bound, as in the in-memory call
    int& k = F.k;
    k = 0;
    if (F.am > 0.f) { int e; std::frexp((double)F.am, &e); k = 23 - e; }
    F.eps = prm->mode == CPT_EB_REL ? prm->eb * ((double)F.mx - (double)F.mn) : prm->eb;
    const double ef = std::floor(std::ldexp(F.eps, k) - 0.5);
    F.eps_int = !(ef > 0) ? 0 : (ef > 8388608.0 ? 8388608 : (int)ef);
    cpt_stats& st = F.st;
    std::memset(&st, 0, sizeof(st));
    st.scale_log2 = k;
    st.eps_int = F.eps_int;
    st.eps = F.eps;
    F.nby = (H + B - 1) / B;
    F.nbx = (W + B - 1) / B;
    F.nstrips = (H + 31) / 32;
    F.want_sl = prm->pred != CPT_PRED_LORENZO && T > 1 && F.eps_int > 0;
    const int nsm = sm_count();
    // call-wide device state
    unsigned long long* d_lg;
    CPT_CUDA(ar.alloc(&d_lg, kLog2Tab));
    launch_log2_table(d_lg, kLog2Tab, s);
    NetDev net{};
    if (F.has_net) {
        float* d_net;
        CPT_CUDA(ar.alloc(&d_net, kNetDevFloats));
        rc = upload_net(prm->model, d_net, &net, s);
        if (rc != CPT_OK) return rc;
    }
    // the window
    const size_t HW = F.HW, ND = diag_elems(H, W, Tw);
    int32_t *d_q, *d_qhat, *d_ld;
    uint16_t *d_mask, *d_qd, *d_mask_carry;
    int2 *d_cls, *d_qdiag, *d_psl, *d_qhat_carry;
    unsigned *d_clsm, *d_hist, *d_queue, *d_ticket;
    uint8_t *d_qxi, *d_modes;
    uint32_t* d_sym;
    unsigned long long *d_cnt64, *d_off, *d_stmp;
    int* d_status;
    int4* d_order;
    VerifyOut* d_vo;
    const int Umin = F.has_modes ? (B == 32 ? 32 : 16) : 8;
    const size_t nprep = (size_t)Tw * ((H + Umin - 1) / Umin) * ((W + Umin - 1) / Umin);
    const size_t NS = HW * S;  // vertices of a slab
    CPT_CUDA(ar.alloc(&d_q, 2 * HW * Tw));
    CPT_CUDA(ar.alloc(&d_qhat, 2 * HW * Tw));
    CPT_CUDA(ar.alloc(&d_mask, HW * Tw));
    CPT_CUDA(ar.alloc(&d_mask_carry, HW));
    CPT_CUDA(ar.alloc(&d_qhat_carry, HW));
    CPT_CUDA(ar.alloc(&d_cls, ND));
    CPT_CUDA(ar.alloc(&d_clsm, ND));
    CPT_CUDA(ar.alloc(&d_qdiag, ND));
    CPT_CUDA(ar.alloc(&d_psl, F.want_sl ? HW * Tw : 1));
    CPT_CUDA(ar.alloc(&d_qxi, HW * Tw));
    CPT_CUDA(ar.alloc(&d_sym, HW * Tw));
    CPT_CUDA(ar.alloc(&d_modes, (size_t)Tw * F.nby * F.nbx));
    CPT_CUDA(ar.alloc(&d_cnt64, 8));
    CPT_CUDA(ar.alloc(&d_off, compact_tiles(NS) + 1));
    CPT_CUDA(ar.alloc(&d_stmp, scan_temp_elems(compact_tiles(NS) + 1)));
    CPT_CUDA(ar.alloc(&d_qd, 2 * NS));
    CPT_CUDA(ar.alloc(&d_ld, 2 * NS));
    CPT_CUDA(ar.alloc(&d_hist, 33 + 2 * kRadius));
    CPT_CUDA(ar.alloc(&d_queue, nprep + 2));
    CPT_CUDA(ar.alloc(&d_ticket, 1));
    CPT_CUDA(ar.alloc(&d_status, 1));
    CPT_CUDA(ar.alloc(&d_order, (size_t)Tw * F.nstrips));
    CPT_CUDA(ar.alloc(&d_vo, 1));
    CPT_CUDA(cudaMemsetAsync(d_cnt64, 0, 8 * sizeof(unsigned long long), s));
    CPT_CUDA(cudaMemsetAsync(d_hist, 0, sizeof(unsigned) * (33 + 2 * kRadius), s));
    CPT_CUDA(cudaMemsetAsync(d_vo, 0, sizeof(VerifyOut), s));
    // host copies of the codes
    std::vector<uint8_t> qxi_h(F.N), modes_h(F.has_modes ? (size_t)T * F.nby * F.nbx : 0);
    std::vector<uint16_t> qd_h;
    std::vector<int32_t> ld_h;
    const PipeTuning tune = tuning_of(prm);
    const long long timeout_ns = 2000000000ll;
    const size_t ntw = HW * 2;  // values per window slice
    for (int t0 = 0; t0 < T;) {
        const int t1 = std::min(t0 + S, T);
        const int w0 = t0 > 0 ? t0 - 1 : 0, we = std::min(t1 + 1, T);
        const int Tv = we - w0, vb = t0 - w0, ve = t1 - w0;
        // the window's input slices, 16-byte aligned on the device
        const float* src = uv + ntw * w0;
        const float* d_src = src;
        if (!F.dev_in || (reinterpret_cast<uintptr_t>(src) & 15u)) {
            CPT_CUDA(cudaMemcpyAsync(d_uvw, src, ntw * Tv * sizeof(float), cudaMemcpyDefault, s));
            d_src = d_uvw;
        }
        launch_to_fixed(d_src, ntw * Tv, k, d_q, nsm * 8, s);
        // masks: the carried slice t0 - 1, the slab's (their own slab faces
        // reach slice t1), none for the context slice
        if (vb == 1) CPT_CUDA(cudaMemcpyAsync(d_mask, d_mask_carry, HW * sizeof(uint16_t), cudaMemcpyDeviceToDevice, s));
        if (ve < Tv) CPT_CUDA(cudaMemsetAsync(d_mask + HW * ve, 0, HW * sizeof(uint16_t), s));
        launch_face_masks(d_q, H, W, Tv, d_mask, d_cnt64, s, vb, ve - vb);
        // classification of the slab (and the strip-diagonal copy of q for the context slice)
        CPT_CUDA(cudaMemsetAsync(d_cls, 0, ND * sizeof(int2), s));
        CPT_CUDA(cudaMemsetAsync(d_clsm, 0, ND * sizeof(unsigned), s));
        CPT_CUDA(cudaMemsetAsync(d_qdiag, 0, ND * sizeof(int2), s));
        launch_classify(d_q, d_mask, H, W, Tv, F.eps_int, d_cls, d_clsm, d_qdiag, s, vb, std::min(ve + 1, Tv) - vb);
        // the encoder pipeline over slices [vb, ve) of the window
        SliceArgs A;
        std::memset(&A, 0, sizeof(A));
        A.q = reinterpret_cast<const int2*>(d_q);
        A.qhat = reinterpret_cast<int2*>(d_qhat);
        A.mask = d_mask;
        A.cls = d_cls;
        A.cls_m = d_clsm;
        A.qd = d_qdiag;
        A.psl = d_psl;
        A.modes = d_modes;
        A.qxi = d_qxi;
        A.sym = d_sym;
        A.counters = d_cnt64 + 1;
        A.H = H; A.W = W; A.T = Tv;
        A.t_end = ve;
        A.eps_int = F.eps_int;
        A.pred = (int)prm->pred;
        A.B = B; A.n = F.nstride; A.nby = F.nby; A.nbx = F.nbx;
        A.nchunks = (W + 31) / 32;
        A.cfl_x = sl_cfl(F.dt, F.dx, k);
        A.cfl_y = sl_cfl(F.dt, F.dy, k);
        A.R = 0;
        if (F.want_sl && F.has_net) {
            A.R = kNetReach;
        } else if (F.want_sl) {
            const double qmax = std::ceil((double)F.am * std::ldexp(1.0, k)) +
                                (F.eps_int > 0 ? std::ldexp(1.0, (int)std::floor(std::log2((double)F.eps_int))) : 0.0);
            A.R = sl_reach(qmax, A.cfl_x, A.cfl_y, H, W);
        }
        if (F.has_net) A.net = net;
        A.log2tab = d_lg;
        int U = F.has_modes ? (B == 32 ? 32 : 16) : 8;
        if (prm->pred == CPT_PRED_SL && tune.sl_unit == 16) U = 16;
        A.U = U;
        A.nur = (H + U - 1) / U;
        A.nuc = (W + U - 1) / U;
        const int u_first = std::max(vb, 1);  // units of slices >= 1 only
        const unsigned per_slice_units = (unsigned)A.nur * (unsigned)A.nuc;
        A.n_units = F.want_sl && ve > u_first ? (unsigned)(ve - u_first) * per_slice_units : 0u;
        A.unit_base = 0;
        A.queue_len = A.n_units;
        A.qslot = d_queue + 2;
        A.qtail = d_queue + 1;
        A.status = d_status;
        A.timeout_ns = timeout_ns;
        // reconstruction words: the carried slice, then nothing present
        if (vb == 1) CPT_CUDA(cudaMemcpyAsync(d_qhat, d_qhat_carry, HW * sizeof(int2), cudaMemcpyDeviceToDevice, s));
        CPT_CUDA(cudaMemsetAsync(d_qhat + 2 * HW * vb, 0, 2 * HW * (Tv - vb) * sizeof(int32_t), s));
        if (F.want_sl) CPT_CUDA(cudaMemsetAsync(d_psl, 0, HW * Tw * sizeof(int2), s));  // no prediction word present
        CPT_CUDA(cudaMemsetAsync(d_modes, 0, (size_t)Tw * F.nby * F.nbx, s));
        CPT_CUDA(cudaMemsetAsync(d_queue, 0, sizeof(unsigned) * (nprep + 2), s));
        CPT_CUDA(cudaMemsetAsync(d_ticket, 0, sizeof(unsigned), s));
        CPT_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));
        std::vector<unsigned> pre;
        if (vb == 1 && A.n_units > 0) {
            // the slab's first slice follows a finished slice: its units are ready now
            pre.resize(per_slice_units + 2);
            pre[0] = 0;                // head
            pre[1] = per_slice_units;  // tail
            for (unsigned x = 0; x < per_slice_units; ++x) pre[2 + x] = x + 1u;  // unit id (slice 1) + 1
            CPT_CUDA(cudaMemcpyAsync(d_queue, pre.data(), sizeof(unsigned) * pre.size(), cudaMemcpyHostToDevice, s));
        }
        std::vector<int4> order, all;
        merged_order({OrderField{Tv, F.nstrips, A.R, A.n_units}}, tune, all);
        for (const int4& it : all)
            if (it.y >= vb && it.y < ve) order.push_back(it);
        CPT_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int4) * order.size(), cudaMemcpyHostToDevice, s));
        PipeArgs P;
        std::memset(&P, 0, sizeof(P));
        P.one = A;
        P.fields = nullptr;
        P.nfields = 1;
        P.order = d_order;
        P.total_items = (unsigned)order.size();
        P.ticket = d_ticket;
        P.qhead = d_queue;
        P.queue_len = A.n_units;
        P.status = d_status;
        P.timeout_ns = timeout_ns;
        P.skip_item = ~0u;
        CPT_CUDA(launch_encode_pipeline(P, (int)prm->pred, nsm, tune, s));
        int status = 0;
        CPT_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaStreamSynchronize(s));
        if (status != 0) return fail((cpt_status)status, "wavefront wait timed out");
        // the slab's codes: bound codes to the host and their histogram,
        // residual symbols and verbatim values compacted, counted, to the host
        const size_t Ns = HW * (ve - vb), o = HW * vb;
        CPT_CUDA(cudaMemcpyAsync(qxi_h.data() + HW * t0, d_qxi + o, Ns, cudaMemcpyDeviceToHost, s));
        launch_hist_u8(d_qxi + o, Ns, d_hist, s);
        const size_t nt = compact_tiles(Ns);
        CPT_CUDA(cudaMemsetAsync(d_off + nt, 0, sizeof(unsigned long long), s));
        launch_tile_count(d_qxi + o, d_sym + o, Ns, d_off, s);
        launch_exclusive_scan_u64(d_off, nt + 1, d_stmp, s);
        unsigned long long tot = 0;
        CPT_CUDA(cudaMemcpyAsync(&tot, d_off + nt, 8, cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaStreamSynchronize(s));
        const size_t nq = (size_t)(tot >> 32), nl = (size_t)(tot & 0xFFFFFFFFull);
        launch_tile_scatter(d_qxi + o, d_sym + o, d_q + 2 * o, d_off, Ns, d_qd, d_ld, s);
        launch_hist_u16(d_qd, nq, d_hist + 33, s);
        const size_t q0 = qd_h.size(), l0 = ld_h.size();
        qd_h.resize(q0 + nq);
        ld_h.resize(l0 + nl);
        if (nq) CPT_CUDA(cudaMemcpyAsync(qd_h.data() + q0, d_qd, nq * sizeof(uint16_t), cudaMemcpyDeviceToHost, s));
        if (nl) CPT_CUDA(cudaMemcpyAsync(ld_h.data() + l0, d_ld, nl * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        if (F.has_modes) {
            const size_t per = (size_t)F.nby * F.nbx;
            CPT_CUDA(cudaMemcpyAsync(modes_h.data() + per * t0, d_modes + per * vb, per * (ve - vb),
                                     cudaMemcpyDeviceToHost, s));
        }
        // verification of the slices whose slab faces are now reconstructed
        const int vend = t1 == T ? ve : ve - 1;
        if (prm->verify && vend > 0)
            launch_verify(d_qhat, d_mask, d_src, H, W, Tv, k, d_vo, s, 0, vend);
        // carry the slab's last slice
        CPT_CUDA(cudaMemcpyAsync(d_qhat_carry, d_qhat + 2 * HW * (ve - 1), HW * sizeof(int2), cudaMemcpyDeviceToDevice, s));
        CPT_CUDA(cudaMemcpyAsync(d_mask_carry, d_mask + HW * (ve - 1), HW * sizeof(uint16_t), cudaMemcpyDeviceToDevice, s));
        CPT_CUDA(cudaStreamSynchronize(s));
        t0 = t1;
    }
    return streamed_finish(F, prm, ar, d_hist, d_cnt64, d_vo, qxi_h, qd_h, ld_h, modes_h, out, out_bytes, stats);
}

// Many fields, one set of parameters: fields are taken in order into groups
// whose device memory fits the budget; each group is one run of every phase
// with one pipeline launch.
static cpt_status compress_batch_impl(const float* const* uv, const cpt_dims* dims, int nfields,
                                      const cpt_params* prm, size_t budget, uint8_t** out, size_t* out_bytes,
                                      cpt_stats* stats, cpt_batch_stats* bst) {
    if (!uv || !dims || !prm || !out || !out_bytes || nfields < 1) return fail(CPT_ERR_ARG, "null argument or no field");
    for (int f = 0; f < nfields; ++f) {
        out[f] = nullptr;
        out_bytes[f] = 0;
        if (!uv[f]) return fail(CPT_ERR_ARG, "null field");
    }
    cpt_status rc = check_device();
    if (rc != CPT_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(prm->cuda_stream);
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        CPT_CUDA(cudaMemGetInfo(&fr, &tot));
        budget = fr / 10 * 6;
    }
    cpt_batch_stats b;
    std::memset(&b, 0, sizeof(b));
    b.device_budget = budget;
    cudaEvent_t ev0, ev1;
    CPT_CUDA(cudaEventCreate(&ev0));
    CPT_CUDA(cudaEventCreate(&ev1));
    struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } evg{ev0, ev1};
    CPT_CUDA(cudaEventRecord(ev0, s));
    auto release_all = [&]() {
        for (int f = 0; f < nfields; ++f) {
            if (out[f] && !pinned_pool().put(out[f])) std::free(out[f]);
            out[f] = nullptr;
            out_bytes[f] = 0;
        }
    };
    cpt_status verdict = CPT_OK;
    int first = 0;
    while (first < nfields) {
        // the next group: at least one field, then as many as fit the budget
        int last = first;
        size_t need = 0;
        while (last < nfields) {
            const size_t m = FieldJob::device_bytes(dims[last], !is_device_pointer(uv[last]));
            if (last > first && need + m > budget) break;
            need += m;
            ++last;
        }
        std::vector<std::unique_ptr<FieldJob>> jobs;
        std::vector<FieldJob*> jp;
        for (int f = first; f < last; ++f) {
            jobs.emplace_back(new FieldJob(s, true));
            FieldJob& j = *jobs.back();
            j.uv = uv[f];
            j.dims = dims[f];
            j.prm = prm;
            jp.push_back(&j);
        }
        PipeTimes pt;
        rc = run_jobs(jp.data(), (int)jp.size(), prm, s, prm->tune != 0, tuning_of(prm), &pt);
        if (rc != CPT_OK) {
            const std::string msg = g_last_error;
            jobs.clear();
            release_all();
            return fail(rc, "field group " + std::to_string(first) + ".." + std::to_string(last - 1) + ": " + msg);
        }
        CPT_CUDA(cudaStreamSynchronize(s));
        CPT_CUDA(cudaGetLastError());
        b.ms_pipeline += pt.ms_pipeline;
        b.ms_tune += pt.ms_tune;
        for (int x = 0; x < 8; ++x) b.ms_phase[x] += pt.ms_phase[x];
        b.groups++;
        b.schedule[0] = pt.used.prep_share;
        b.schedule[1] = pt.used.sl_unit;
        b.schedule[2] = pt.used.slice_weight;
        b.schedule[3] = pt.used.slack;
        b.schedule[4] = pt.used.warps_per_sm;
        b.schedule[5] = pt.used.mixed;
        for (int f = first; f < last; ++f) {
            FieldJob& j = *jobs[f - first];
            cpt_stats st1;
            cpt_status r1 = j.finish(0.0, pt.ms_pipeline, &out[f], &out_bytes[f], &st1);
            if (r1 == CPT_ERR_VERIFY && verdict == CPT_OK) verdict = r1;
            else if (r1 != CPT_OK && r1 != CPT_ERR_VERIFY) { jobs.clear(); release_all(); return r1; }
            const cpt_status rz = wrap_output(prm, &out[f], &out_bytes[f], &st1, 8ull * j.N);
            if (rz != CPT_OK) { jobs.clear(); release_all(); return rz; }
            for (int x = 0; x < 8; ++x)
                if (x != 4) b.launches += st1.launches[x];
            b.in_bytes += 8ull * j.N;
            b.out_bytes += st1.out_bytes;
            if (stats) stats[f] = st1;
        }
        b.launches += 1;  // one pipeline launch for the group
        first = last;
    }
    CPT_CUDA(cudaEventRecord(ev1, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    b.ms_total = ms;
    if (stats)
        for (int f = 0; f < nfields; ++f) stats[f].ms_total = ms;
    if (bst) *bst = b;
    if (verdict != CPT_OK) return fail(verdict, "a reconstruction changed a face predicate or exceeded the bound");
    return CPT_OK;
}

// ---------------------------------------------------------------------------
// decompression
// ---------------------------------------------------------------------------
struct Reader {
    const uint8_t* p;
    size_t n, at = 0;
    bool bad = false;
    uint32_t u32() {
        if (n - at < 4 || at > n) { bad = true; return 0; }
        uint32_t x = (uint32_t)p[at] | ((uint32_t)p[at + 1] << 8) | ((uint32_t)p[at + 2] << 16) | ((uint32_t)p[at + 3] << 24);
        at += 4;
        return x;
    }
    uint64_t u64() { uint64_t lo = u32(); return lo | ((uint64_t)u32() << 32); }
    double f64() { uint64_t x = u64(); double d; std::memcpy(&d, &x, 8); return d; }
    const uint8_t* take(size_t k) {
        if (at > n || n - at < k) { bad = true; return nullptr; }
        const uint8_t* q = p + at;
        at += k;
        return q;
    }
};

// Host side of one Huffman stream: codebook -> decoding tables, sync points,
// words; all checked for consistency.
struct HuffHost {
    uint64_t nsym = 0, nwords = 0;
    std::vector<uint32_t> lut, first, count, base, sorted;
    std::vector<unsigned long long> lut3;  // up to three codes per 12-bit window
    std::vector<unsigned long long> chunk_off;
    const uint8_t* words = nullptr;
};

static bool parse_huff(Reader& r, uint32_t alphabet, HuffHost& h) {
    h.nsym = r.u64();
    const uint32_t nused = r.u32(), chunk = r.u32();
    if (r.bad || chunk != (uint32_t)kChunkSyms || nused > alphabet) return false;
    std::vector<uint8_t> len(alphabet, 0);
    uint32_t prev = 0;
    uint64_t kraft = 0;  // in units of 2^-24
    for (uint32_t x = 0; x < nused; ++x) {
        const uint32_t e = r.u32();
        const uint32_t sy = e >> 8, l = e & 255u;
        if (r.bad || sy >= alphabet || l == 0 || l > kMaxCodeLen || (x > 0 && sy <= prev)) return false;
        len[sy] = (uint8_t)l;
        prev = sy;
        kraft += 1ull << (kMaxCodeLen - l);
    }
    if (kraft > (1ull << kMaxCodeLen) || (h.nsym > 0 && nused == 0)) return false;
    const uint64_t nchunks = (h.nsym + kChunkSyms - 1) / kChunkSyms;
    if (nchunks > (r.n - std::min(r.n, r.at)) / 8) return false;
    h.chunk_off.resize(nchunks);
    for (uint64_t c = 0; c < nchunks; ++c) h.chunk_off[c] = r.u64();
    h.nwords = r.u64();
    if (r.bad || h.nwords > (r.n - std::min(r.n, r.at)) / 4) return false;
    h.words = r.take(4 * h.nwords);
    if (!h.words) return false;
    for (uint64_t c = 0; c < nchunks; ++c)
        if (h.chunk_off[c] > h.nwords * 32 || (c > 0 && h.chunk_off[c] < h.chunk_off[c - 1])) return false;
    // canonical decoding tables
    h.first.assign(25, 0);
    h.count.assign(25, 0);
    h.base.assign(25, 0);
    for (uint8_t l : len) if (l) h.count[l]++;
    uint32_t code = 0, idx = 0;
    for (int l = 1; l <= 24; ++l) {
        code = (code + h.count[l - 1]) << 1;
        h.first[l] = code;
        h.base[l] = idx;
        idx += h.count[l];
    }
    h.first[0] = 0;
    h.sorted.resize(std::max<uint32_t>(idx, 1));
    std::vector<uint32_t> fill(25, 0);
    for (uint32_t sy = 0; sy < alphabet; ++sy)  // by length, then symbol
        if (len[sy]) h.sorted[h.base[len[sy]] + fill[len[sy]]++] = sy;
    h.lut.assign(4096, 0);
    for (int l = 1; l <= 12; ++l)
        for (uint32_t k = 0; k < h.count[l]; ++k) {
            const uint32_t c = h.first[l] + k, sy = h.sorted[h.base[l] + k];
            const uint32_t lo = c << (12 - l), span = 1u << (12 - l);
            for (uint32_t x = 0; x < span; ++x) h.lut[lo + x] = (sy << 5) | (uint32_t)l;
        }
    // the complete codes at the start of each 12-bit window, up to three
    h.lut3.assign(4096, 0ull);
    for (uint32_t v = 0; v < 4096; ++v) {
        unsigned long long e = 0;
        uint32_t pos = 0, cnt = 0;
        while (cnt < 3 && pos < 12) {
            const uint32_t rest = (v << pos) & 4095u;  // the window's bits from pos on, left aligned
            const uint32_t le = h.lut[rest];
            const uint32_t l = le & 31u;
            if (le == 0 || pos + l > 12) break;
            e |= (unsigned long long)(le >> 5) << (7 + 16 * cnt);
            pos += l;
            ++cnt;
        }
        h.lut3[v] = e | cnt | ((unsigned long long)pos << 2);
    }
    return true;
}

// One Huffman stream's device buffers (from the arena, on the call's stream).
struct HuffBufs {
    uint32_t *words = nullptr, *tab = nullptr;
    unsigned long long *off = nullptr, *lut3 = nullptr;
    size_t ntab = 0;
};
static cpt_status huff_alloc(const HuffHost& hh, DevArena& ar, HuffBufs& b) {
    if (hh.nsym == 0) return CPT_OK;
    b.ntab = 4096 + 3 * 25 + hh.sorted.size();
    CPT_CUDA(ar.alloc(&b.words, hh.nwords + 2));
    CPT_CUDA(ar.alloc(&b.off, hh.chunk_off.size()));
    CPT_CUDA(ar.alloc(&b.lut3, 4096));
    CPT_CUDA(ar.alloc(&b.tab, b.ntab));
    return CPT_OK;
}

// Uploads one Huffman stream into its buffers and decodes it on stream s
// (the copies come from pageable host memory, staged by the driver before
// each call returns, so `tab` may go after the launch).
template <typename Sym>
static cpt_status decode_huff_stream(const HuffHost& hh, const HuffBufs& b, Sym* d_out, int* d_status,
                                     cudaStream_t s) {
    if (hh.nsym == 0) return CPT_OK;
    CPT_CUDA(cudaMemsetAsync(b.words, 0, 4 * (hh.nwords + 2), s));
    if (hh.nwords) CPT_CUDA(cudaMemcpyAsync(b.words, hh.words, 4 * hh.nwords, cudaMemcpyHostToDevice, s));
    CPT_CUDA(cudaMemcpyAsync(b.off, hh.chunk_off.data(), 8 * hh.chunk_off.size(), cudaMemcpyHostToDevice, s));
    CPT_CUDA(cudaMemcpyAsync(b.lut3, hh.lut3.data(), 8 * 4096, cudaMemcpyHostToDevice, s));
    std::vector<uint32_t> tab;
    tab.reserve(b.ntab);
    tab.insert(tab.end(), hh.lut.begin(), hh.lut.end());
    tab.insert(tab.end(), hh.first.begin(), hh.first.end());
    tab.insert(tab.end(), hh.count.begin(), hh.count.end());
    tab.insert(tab.end(), hh.base.begin(), hh.base.end());
    tab.insert(tab.end(), hh.sorted.begin(), hh.sorted.end());
    CPT_CUDA(cudaMemcpyAsync(b.tab, tab.data(), 4 * b.ntab, cudaMemcpyHostToDevice, s));
    HuffDecode h;
    h.words = b.words;
    h.nwords = hh.nwords;
    h.nsym = hh.nsym;
    h.chunk_off = b.off;
    h.lut = b.tab;
    h.first = b.tab + 4096;
    h.count = b.tab + 4096 + 25;
    h.base = b.tab + 4096 + 50;
    h.sorted = b.tab + 4096 + 75;
    h.lut3 = b.lut3;
    if constexpr (sizeof(Sym) == 1) launch_huff_decode_u8(h, reinterpret_cast<uint8_t*>(d_out), d_status, s);
    else launch_huff_decode_u16(h, reinterpret_cast<uint16_t*>(d_out), d_status, s);
    return CPT_OK;
}

static cpt_status decompress_impl(const uint8_t* in, size_t in_bytes, float* uv_out, int32_t* qhat_out,
                                  cpt_dims* dims_out, void* cuda_stream) {
    if (!in) return fail(CPT_ERR_ARG, "null stream");
    if (is_zstd_container(in, in_bytes)) {  // the optional ZSTD frame around a stream
        uint8_t* raw = nullptr;
        size_t rn = 0;
        const cpt_status rz = zstd_unwrap(in, in_bytes, &raw, &rn);
        if (rz != CPT_OK) return rz;
        if (is_zstd_container(raw, rn)) {
            std::free(raw);
            return fail(CPT_ERR_CORRUPT, "nested zstd container");
        }
        const cpt_status rc = decompress_impl(raw, rn, uv_out, qhat_out, dims_out, cuda_stream);
        std::free(raw);
        return rc;
    }
    Reader r{in, in_bytes};
    const uint8_t* magic = r.take(4);
    if (!magic || std::memcmp(magic, "CPT1", 4) != 0) return fail(CPT_ERR_CORRUPT, "not a cpt stream");
    const uint32_t ver = r.u32();
    const int H = (int)r.u32(), W = (int)r.u32(), T = (int)r.u32();
    const int k = (int)r.u32();
    const uint32_t eps_hdr = r.u32();  // eps'
    const int pred = (int)r.u32(), B = (int)r.u32();
    const int stride_hdr = (int)r.u32();  // MoP sampling stride
    const uint32_t radius = r.u32();
    r.u32();
    const double dx = r.f64(), dy = r.f64(), dt = r.f64();
    r.f64();  // eps
    const uint64_t n_ld = r.u64(), mode_bytes = r.u64();
    if (r.bad || ver != kFormat || H < 2 || W < 2 || T < 1 || pred < 0 || pred > 4 || B < 1 ||
        radius != (uint32_t)kRadius || k < -200 || k > 200 || !(dx > 0) || !(dy > 0) || !(dt > 0) ||
        eps_hdr > 8388608u || stride_hdr < 1 || ((pred == 2 || pred == 4) && (B < 4 || 32 % B != 0)) ||
        (long long)H * W > (1ll << 31) / 4)
        return fail(CPT_ERR_CORRUPT, "bad stream header");
    if (dims_out) {
        dims_out->H = H; dims_out->W = W; dims_out->T = T;
        dims_out->dx = dx; dims_out->dy = dy; dims_out->dt = dt;
    }
    if (!uv_out && !qhat_out) return CPT_OK;
    const size_t N = (size_t)H * W * T;
    const int nby = (H + B - 1) / B, nbx = (W + B - 1) / B;
    const size_t nblk = (pred == 2 || pred == 4) ? (size_t)T * nby * nbx : 0;
    if (mode_bytes != (nblk + 7) / 8) return fail(CPT_ERR_CORRUPT, "bad mode section");
    const uint8_t* modes = r.take(mode_bytes);
    std::vector<uint16_t> model;
    if (pred == 3 || pred == 4) {  // the learned predictor's parameters
        if (r.u32() != (uint32_t)kNetParams || r.bad) return fail(CPT_ERR_CORRUPT, "bad model section");
        model.resize(kNetParams);
        for (int x = 0; x < kNetParams; x += 2) {
            const uint32_t wv = r.u32();
            model[x] = (uint16_t)(wv & 0xFFFFu);
            if (x + 1 < kNetParams) model[x + 1] = (uint16_t)(wv >> 16);
        }
        if (r.bad) return fail(CPT_ERR_CORRUPT, "truncated model section");
    }
    HuffHost hx, hd;
    if (!modes || !parse_huff(r, 33, hx) || hx.nsym != N) return fail(CPT_ERR_CORRUPT, "bad bound-code stream");
    if (!parse_huff(r, 2 * kRadius, hd)) return fail(CPT_ERR_CORRUPT, "bad residual stream");
    if (n_ld > (r.n - std::min(r.n, r.at)) / 4) return fail(CPT_ERR_CORRUPT, "truncated verbatim values");
    const uint8_t* ldp = r.take(4 * n_ld);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(CPT_ERR_CUDA, "no CUDA device available");
    }
    retain_pool_memory();
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    DevArena ar(s);
    const int nsm = sm_count();
    int* d_status;
    uint8_t *d_qxi, *d_modes;
    uint16_t* d_qd;
    uint32_t* d_sym;
    int32_t* d_ld;
    int2 *d_dcs, *d_draw, *d_qhat, *d_psl, *d_rraw;
    unsigned long long *d_qoff, *d_loff, *d_tmp;
    CPT_CUDA(ar.alloc(&d_status, 1));
    CPT_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));
    CPT_CUDA(ar.alloc(&d_qxi, N));
    CPT_CUDA(ar.alloc(&d_qd, hd.nsym));
    CPT_CUDA(ar.alloc(&d_sym, N));
    CPT_CUDA(ar.alloc(&d_ld, n_ld));
    const size_t ND = diag_elems(H, W, T);  // strip-diagonal inputs of the pipeline, zero padding
    CPT_CUDA(ar.alloc(&d_dcs, ND));  // every element written by the transposing copy (padding zero)
    CPT_CUDA(ar.alloc(&d_draw, ND));
    CPT_CUDA(ar.alloc(&d_qhat, N));
    CPT_CUDA(ar.alloc(&d_psl, pred != 0 ? N : 1));
    CPT_CUDA(ar.alloc(&d_rraw, N));
    const size_t nt = compact_tiles(N);
    CPT_CUDA(ar.alloc(&d_qoff, nt + 1));
    CPT_CUDA(ar.alloc(&d_loff, nt + 1));
    CPT_CUDA(ar.alloc(&d_tmp, scan_temp_elems(nt + 1)));
    CPT_CUDA(ar.alloc(&d_modes, std::max<size_t>(mode_bytes, 1)));
    if (mode_bytes) CPT_CUDA(cudaMemcpyAsync(d_modes, modes, mode_bytes, cudaMemcpyHostToDevice, s));
    if (n_ld) CPT_CUDA(cudaMemcpyAsync(d_ld, ldp, 4 * n_ld, cudaMemcpyHostToDevice, s));
    // the two Huffman streams decode at once: Q_xi on the call's stream, Q_d
    // on a second one, joined before the residual symbols are used
    static thread_local DecodeSide t_side;
    if (!t_side.ready()) return fail(CPT_ERR_CUDA, "stream or event creation failed");
    HuffBufs bx, bd;
    cpt_status rc = huff_alloc(hx, ar, bx);
    if (rc != CPT_OK) return rc;
    rc = huff_alloc(hd, ar, bd);
    if (rc != CPT_OK) return rc;
    CPT_CUDA(cudaEventRecord(t_side.ev_fork, s));  // every buffer above exists for the second stream
    CPT_CUDA(cudaStreamWaitEvent(t_side.s2, t_side.ev_fork, 0));
    rc = decode_huff_stream<uint8_t>(hx, bx, d_qxi, d_status, s);
    if (rc == CPT_OK) rc = decode_huff_stream<uint16_t>(hd, bd, d_qd, d_status, t_side.s2);
    CPT_CUDA(cudaEventRecord(t_side.ev_join, t_side.s2));
    if (rc != CPT_OK) {
        cudaStreamWaitEvent(s, t_side.ev_join, 0);  // nothing of the call outlives s
        return rc;
    }
    // residual symbols per tile of the bound codes; their total must be the
    // length of the Q_d stream
    unsigned long long total = 0;
    int status = 0;
    CPT_CUDA(cudaMemsetAsync(d_qoff + nt, 0, sizeof(unsigned long long), s));
    launch_dec_tile_qd(d_qxi, N, d_qoff, d_status, s);
    launch_exclusive_scan_u64(d_qoff, nt + 1, d_tmp, s);
    CPT_CUDA(cudaStreamWaitEvent(s, t_side.ev_join, 0));  // the Q_d symbols (and nothing of the call outlives s)
    CPT_CUDA(cudaMemcpyAsync(&total, d_qoff + nt, 8, cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    if (status != 0 || total != hd.nsym) return fail(CPT_ERR_CORRUPT, "bound codes do not match the residuals");
    // each vertex's symbols, the verbatim values per tile, then the values;
    // (bound code, symbols) go to d_qhat and the values to d_rraw in raster
    // order, from where the transposing copy lays both out strip-diagonally
    CPT_CUDA(cudaMemsetAsync(d_loff + nt, 0, sizeof(unsigned long long), s));
    launch_dec_tile_sym(d_qxi, N, d_qd, hd.nsym, d_qoff, d_sym, d_loff, d_status, s);
    launch_exclusive_scan_u64(d_loff, nt + 1, d_tmp, s);
    launch_dec_tile_raw(d_qxi, d_sym, N, d_ld, n_ld, d_loff, d_qhat, d_rraw, d_status, s);
    launch_diag_transpose(d_qhat, d_rraw, H, W, T, d_dcs, d_draw, s);
    CPT_CUDA(cudaMemcpyAsync(&total, d_loff + nt, 8, cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    if (status != 0 || total != n_ld) return fail(CPT_ERR_CORRUPT, "verbatim values do not match the codes");
    // reconstruction: the encoder's pipeline in decoding mode.  Waves rebuild
    // qhat from the symbols in raster order, prediction units give the SL or
    // learned predictions, MoP block modes come from the stream.
    const int eps_int = (int)eps_hdr;
    const bool has_net = pred == 3 || pred == 4, has_modes = pred == 2 || pred == 4;
    const bool want_sl = pred != 0 && T > 1 && eps_int > 0;
    const int nstrips = (H + 31) / 32;
    SliceArgs A;
    std::memset(&A, 0, sizeof(A));
    unsigned long long* d_ctr;
    CPT_CUDA(ar.alloc(&d_ctr, 8));
    CPT_CUDA(cudaMemsetAsync(d_ctr, 0, 8 * sizeof(unsigned long long), s));
    CPT_CUDA(cudaMemsetAsync(d_qhat, 0, N * sizeof(int2), s));  // no reconstruction word present
    A.qhat = d_qhat;
    A.cls = d_dcs;
    A.cls_m = reinterpret_cast<const unsigned*>(d_dcs);  // (not read when decoding)
    A.qd = d_draw;
    A.psl = d_psl;
    A.mode_bits = d_modes;
    A.decode = 1;
    A.counters = d_ctr + 1;
    A.H = H; A.W = W; A.T = T;
    A.t_end = T;
    A.eps_int = eps_int;
    A.pred = pred;
    A.B = B; A.n = stride_hdr; A.nby = nby; A.nbx = nbx;
    A.nchunks = (W + 31) / 32;
    A.cfl_x = sl_cfl(dt, dx, k);
    A.cfl_y = sl_cfl(dt, dy, k);
    // Reach of the back-trace: |qhat| <= 2^23 + E for every stream (the
    // fixed-point scale keeps |q| <= 2^23, the quantiser moves a value by at
    // most E), so no displacement exceeds that times CFL.
    if (want_sl && has_net) {
        A.R = kNetReach;
    } else if (want_sl) {
        const double qmax = 8388608.0 + (eps_int > 0 ? std::ldexp(1.0, 31 - __builtin_clz((unsigned)eps_int)) : 0.0);
        A.R = sl_reach(qmax, A.cfl_x, A.cfl_y, H, W);
    }
    if (has_net) {
        float* d_net;
        CPT_CUDA(ar.alloc(&d_net, kNetDevFloats));
        cpt_status rc2 = upload_net(model.data(), d_net, &A.net, s);
        if (rc2 != CPT_OK) return rc2;
    }
    A.U = has_modes ? (B == 32 ? 32 : 16) : 8;
    A.nur = (H + A.U - 1) / A.U;
    A.nuc = (W + A.U - 1) / A.U;
    const unsigned long long nu = want_sl ? (unsigned long long)(T - 1) * A.nur * A.nuc : 0ull;
    if (nu >= 0x7FFFFFFFull) return fail(CPT_ERR_UNSUPPORTED, "too many prediction units");
    A.n_units = (unsigned)nu;
    unsigned *d_queue, *d_ticket;
    CPT_CUDA(ar.alloc(&d_queue, (size_t)A.n_units + 2));
    CPT_CUDA(ar.alloc(&d_ticket, 1));
    if (pred != 0) CPT_CUDA(cudaMemsetAsync(d_psl, 0, N * sizeof(int2), s));  // no prediction word present
    CPT_CUDA(cudaMemsetAsync(d_queue, 0, sizeof(unsigned) * ((size_t)A.n_units + 2), s));
    CPT_CUDA(cudaMemsetAsync(d_ticket, 0, sizeof(unsigned), s));
    CPT_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));
    A.qslot = d_queue + 2;
    A.qtail = d_queue + 1;
    A.status = d_status;
    A.queue_len = A.n_units;
    A.timeout_ns = 2000000000ll;
    const PipeTuning tune = kDecodeSchedule;
    std::vector<int4> order;
    merged_order({OrderField{T, nstrips, A.R, A.n_units}}, tune, order);
    int4* d_order;
    CPT_CUDA(ar.alloc(&d_order, order.size()));
    CPT_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int4) * order.size(), cudaMemcpyHostToDevice, s));
    PipeArgs P;
    std::memset(&P, 0, sizeof(P));
    P.one = A;
    P.fields = nullptr;  // one field: read from parameter space
    P.nfields = 1;
    P.order = d_order;
    P.total_items = (unsigned)order.size();
    P.ticket = d_ticket;
    P.qhead = d_queue;
    P.queue_len = A.n_units;
    P.status = d_status;
    P.timeout_ns = A.timeout_ns;
    P.skip_item = ~0u;
    CPT_CUDA(launch_encode_pipeline(P, pred, nsm, tune, s));
    CPT_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaStreamSynchronize(s));  // (the host order table outlives its copy)
    if (status == (int)CPT_ERR_TIMEOUT) return fail(CPT_ERR_TIMEOUT, "decoder wavefront wait timed out");
    if (status != 0) return fail(CPT_ERR_CORRUPT, "corrupt stream");
    // the reconstruction words lose their tag in place only when the integers
    // are asked for; the float conversion removes it on the fly
    if (qhat_out) {
        launch_untag(d_qhat, N, s);
        CPT_CUDA(cudaMemcpyAsync(qhat_out, d_qhat, N * 8, cudaMemcpyDeviceToHost, s));
    }
    if (uv_out) {
        const bool dev = is_device_pointer(uv_out) && !(reinterpret_cast<uintptr_t>(uv_out) & 7u);
        float* dst = uv_out;
        if (!dev) CPT_CUDA(ar.alloc(&dst, 2 * N));
        launch_to_float(d_qhat, N, k, dst, s, !qhat_out);
        if (!dev) CPT_CUDA(cudaMemcpyAsync(uv_out, dst, N * 8, cudaMemcpyDefault, s));
    }
    CPT_CUDA(cudaStreamSynchronize(s));
    CPT_CUDA(cudaGetLastError());
    return CPT_OK;
}

// ---------------------------------------------------------------------------
// trajectories
// ---------------------------------------------------------------------------
// Orders the crossed faces (indices in increasing face id, degree <= 2) into
// trajectories: open paths start at their lowest-id end, closed loops at their
// lowest-id face towards the lower-id neighbour; trajectories are listed by
// their first face.
static void order_trajectories(size_t n, const std::vector<unsigned>& deg, const std::vector<unsigned>& adj,
                               std::vector<uint64_t>& order, std::vector<uint64_t>& offsets) {
    std::vector<uint8_t> seen(n, 0);
    std::vector<std::pair<uint64_t, std::vector<uint64_t>>> trajs;  // (first index, faces)
    auto nbr = [&](size_t x, int slot) -> long long {
        return (deg[x] > (unsigned)slot && adj[2 * x + slot] != 0xFFFFFFFFu) ? (long long)adj[2 * x + slot] : -1;
    };
    auto walk = [&](size_t start, bool loop) {
        std::vector<uint64_t> path;
        long long prev = -1, cur = (long long)start;
        bool first = true;
        while (cur >= 0 && !seen[cur]) {
            seen[cur] = 1;
            path.push_back((uint64_t)cur);
            const long long n0 = nbr((size_t)cur, 0), n1 = nbr((size_t)cur, 1);
            long long nxt = -1;
            if (loop && first) {
                nxt = (n0 >= 0 && (n1 < 0 || n0 < n1)) ? n0 : n1;
            } else if (n0 >= 0 && n0 != prev && !seen[n0]) {
                nxt = n0;
            } else if (n1 >= 0 && n1 != prev && !seen[n1]) {
                nxt = n1;
            }
            first = false;
            prev = cur;
            cur = nxt;
        }
        trajs.emplace_back(start, std::move(path));
    };
    for (size_t a = 0; a < n; ++a)
        if (!seen[a] && deg[a] <= 1) walk(a, false);
    for (size_t a = 0; a < n; ++a)
        if (!seen[a]) walk(a, true);
    std::stable_sort(trajs.begin(), trajs.end(),
                     [](const auto& x, const auto& y) { return x.first < y.first; });
    order.clear();
    offsets.assign(1, 0);
    for (auto& tr : trajs) {
        order.insert(order.end(), tr.second.begin(), tr.second.end());
        offsets.push_back(order.size());
    }
}

static cpt_status trajectories_impl(const float* uv, const cpt_dims* dims, int32_t scale_log2, cpt_trajs** out,
                                    void* cuda_stream) {
    if (!uv || !dims || !out) return fail(CPT_ERR_ARG, "null argument");
    const int H = dims->H, W = dims->W, T = dims->T;
    if (H < 2 || W < 2 || T < 1) return fail(CPT_ERR_ARG, "need H >= 2, W >= 2, T >= 1");
    if ((long long)H * W > (1ll << 31) / 4) return fail(CPT_ERR_ARG, "slice too large");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(CPT_ERR_CUDA, "no CUDA device available");
    }
    retain_pool_memory();
    const size_t N = (size_t)H * W * T, NV = 2 * N;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    DevArena ar(s);
    const int nsm = sm_count();
    const float* d_uv = uv;
    if (!is_device_pointer(uv) || (reinterpret_cast<uintptr_t>(uv) & 15u)) {
        float* tmp;
        CPT_CUDA(ar.alloc(&tmp, NV));
        CPT_CUDA(cudaMemcpyAsync(tmp, uv, NV * sizeof(float), cudaMemcpyDefault, s));
        d_uv = tmp;
    }
    const int rblocks = nsm * 4;
    RangePartial* d_part;
    CPT_CUDA(ar.alloc(&d_part, rblocks));
    launch_range(d_uv, NV, d_part, rblocks, s);
    std::vector<RangePartial> part(rblocks);
    CPT_CUDA(cudaMemcpyAsync(part.data(), d_part, sizeof(RangePartial) * rblocks, cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    float am = 0.f;
    unsigned bad_in = 0;
    for (auto& p : part) { am = std::max(am, p.amax); bad_in |= p.bad; }
    if (bad_in) return fail(CPT_ERR_ARG, "input holds a non-finite value");
    int k = scale_log2;
    if (scale_log2 == CPT_SCALE_AUTO) {
        k = 0;
        if (am > 0.f) { int e; std::frexp((double)am, &e); k = 23 - e; }
    } else if (k < -200 || k > 200 || (am > 0.f && std::ldexp((double)am, k) >= 2147483520.0)) {
        return fail(CPT_ERR_ARG, "scale exponent out of range for the data");
    }
    int32_t* d_q;
    uint16_t* d_mask;
    unsigned long long *d_n, *d_off, *d_tmp, *d_fid;
    CPT_CUDA(ar.alloc(&d_q, NV));
    CPT_CUDA(ar.alloc(&d_mask, N));
    CPT_CUDA(ar.alloc(&d_n, 2));
    CPT_CUDA(ar.alloc(&d_off, N));
    CPT_CUDA(ar.alloc(&d_tmp, scan_temp_elems(N)));
    CPT_CUDA(cudaMemsetAsync(d_n, 0, 2 * sizeof(unsigned long long), s));
    launch_to_fixed(d_uv, NV, k, d_q, nsm * 8, s);
    launch_face_masks(d_q, H, W, T, d_mask, d_n, s);
    launch_face_count(d_mask, N, d_off, s);
    launch_exclusive_scan_u64(d_off, N, d_tmp, s);
    unsigned long long nf = 0;
    CPT_CUDA(cudaMemcpyAsync(&nf, d_n, 8, cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    if (nf >= 0xFFFFFFFFull) return fail(CPT_ERR_UNSUPPORTED, "too many crossed faces");
    unsigned *d_par, *d_deg, *d_adj;
    double* d_xyt;
    CPT_CUDA(ar.alloc(&d_fid, nf));
    CPT_CUDA(ar.alloc(&d_par, nf));
    CPT_CUDA(ar.alloc(&d_deg, nf));
    CPT_CUDA(ar.alloc(&d_adj, 2 * nf));
    CPT_CUDA(ar.alloc(&d_xyt, 3 * nf));
    launch_face_compact(d_mask, d_off, N, d_fid, s);
    launch_iota(d_par, nf, s);
    CPT_CUDA(cudaMemsetAsync(d_deg, 0, 4 * std::max<size_t>(nf, 1), s));
    CPT_CUDA(cudaMemsetAsync(d_adj, 0xFF, 8 * std::max<size_t>(nf, 1), s));
    launch_tet_link(d_mask, d_off, H, W, T, d_par, d_deg, d_adj, d_n + 1, s);
    launch_uf_flatten(d_par, nf, s);
    launch_crossing_points(d_q, d_fid, nf, H, W, d_xyt, s);
    std::vector<unsigned long long> fid(nf);
    std::vector<unsigned> deg(nf), adj(2 * nf), par(nf);
    std::vector<double> xyt(3 * nf);
    unsigned long long bad = 0;
    if (nf) {
        CPT_CUDA(cudaMemcpyAsync(fid.data(), d_fid, 8 * nf, cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaMemcpyAsync(deg.data(), d_deg, 4 * nf, cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaMemcpyAsync(adj.data(), d_adj, 8 * nf, cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaMemcpyAsync(par.data(), d_par, 4 * nf, cudaMemcpyDeviceToHost, s));
        CPT_CUDA(cudaMemcpyAsync(xyt.data(), d_xyt, 24 * nf, cudaMemcpyDeviceToHost, s));
    }
    CPT_CUDA(cudaMemcpyAsync(&bad, d_n + 1, 8, cudaMemcpyDeviceToHost, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    CPT_CUDA(cudaGetLastError());
    std::vector<uint64_t> order, offs;
    order_trajectories((size_t)nf, deg, adj, order, offs);
    // the union-find components count the trajectories independently of the walk
    uint64_t roots = 0;
    for (size_t x = 0; x < nf; ++x) roots += par[x] == (unsigned)x;
    cpt_trajs* tr = static_cast<cpt_trajs*>(std::calloc(1, sizeof(cpt_trajs)));
    if (!tr) return fail(CPT_ERR_OOM, "host allocation failed");
    tr->n_traj = offs.size() - 1;
    tr->n_points = order.size();
    tr->offsets = static_cast<uint64_t*>(std::malloc(sizeof(uint64_t) * offs.size()));
    tr->face_ids = static_cast<uint64_t*>(std::malloc(sizeof(uint64_t) * std::max<size_t>(order.size(), 1)));
    tr->xyt = static_cast<double*>(std::malloc(sizeof(double) * 3 * std::max<size_t>(order.size(), 1)));
    if (!tr->offsets || !tr->face_ids || !tr->xyt) {
        cpt_free_trajs(tr);
        return fail(CPT_ERR_OOM, "host allocation failed");
    }
    std::memcpy(tr->offsets, offs.data(), sizeof(uint64_t) * offs.size());
    for (size_t x = 0; x < order.size(); ++x) {
        tr->face_ids[x] = fid[order[x]];
        std::memcpy(tr->xyt + 3 * x, xyt.data() + 3 * order[x], 3 * sizeof(double));
    }
    tr->bad_tets = bad;
    if (roots != tr->n_traj && bad == 0) {
        cpt_free_trajs(tr);
        return fail(CPT_ERR_CUDA, "trajectory components disagree");
    }
    *out = tr;
    return CPT_OK;
}

// ---------------------------------------------------------------------------
// learned predictor (an extension; the paper has none): inference and
// training entry points
// ---------------------------------------------------------------------------
static cpt_status net_dims_ok(int n, int H, int W) {
    if (n < 1 || H < 1 || W < 1) return fail(CPT_ERR_ARG, "need n, H, W >= 1");
    if ((long long)n * H * W > (1ll << 31) / 4) return fail(CPT_ERR_ARG, "training set too large");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(CPT_ERR_CUDA, "no CUDA device");
    }
    return CPT_OK;
}

static cpt_status net_predict_impl(const uint16_t* model, const int32_t* prev, int H, int W, int32_t* out,
                                   void* stream) {
    if (!model || !prev || !out) return fail(CPT_ERR_ARG, "null argument");
    cpt_status rc = net_dims_ok(1, H, W);
    if (rc != CPT_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevArena ar(s);
    float* d_net;
    int32_t *d_prev, *d_out;
    const size_t nv = 2 * (size_t)H * W;
    CPT_CUDA(ar.alloc(&d_net, kNetDevFloats));
    CPT_CUDA(ar.alloc(&d_prev, nv));
    CPT_CUDA(ar.alloc(&d_out, nv));
    NetDev nd;
    if ((rc = upload_net(model, d_net, &nd, s)) != CPT_OK) return rc;
    CPT_CUDA(cudaMemcpyAsync(d_prev, prev, sizeof(int32_t) * nv, cudaMemcpyDefault, s));
    launch_net_predict(nd, d_prev, H, W, d_out, s);
    CPT_CUDA(cudaGetLastError());
    CPT_CUDA(cudaMemcpyAsync(out, d_out, sizeof(int32_t) * nv, cudaMemcpyDefault, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    return CPT_OK;
}

// Device state of a training run over n pairs (prev, next).
struct NetTrainer {
    float *ws = nullptr, *part = nullptr, *grad = nullptr, *P = nullptr;
    double* lpart = nullptr;
    NetTrainPtrs w{};
    int nblk = 0;
};

static cpt_status net_trainer_setup(DevArena& ar, const int32_t* prev, const int32_t* next, int n, int H, int W,
                                    NetTrainer* tr, cudaStream_t s) {
    const size_t nv = 2 * (size_t)n * H * W;
    int32_t *d_prev, *d_next;
    CPT_CUDA(ar.alloc(&d_prev, nv));
    CPT_CUDA(ar.alloc(&d_next, nv));
    CPT_CUDA(cudaMemcpyAsync(d_prev, prev, sizeof(int32_t) * nv, cudaMemcpyDefault, s));
    CPT_CUDA(cudaMemcpyAsync(d_next, next, sizeof(int32_t) * nv, cudaMemcpyDefault, s));
    tr->nblk = net_wgrad_blocks(n, H, W, sm_count());
    CPT_CUDA(ar.alloc(&tr->ws, net_train_floats(n, H, W)));
    CPT_CUDA(ar.alloc(&tr->part, (size_t)tr->nblk * kNetPartRec));
    CPT_CUDA(ar.alloc(&tr->lpart, 1216));
    CPT_CUDA(ar.alloc(&tr->grad, kNetParams));
    CPT_CUDA(ar.alloc(&tr->P, kNetParams));
    CPT_CUDA(ar.alloc(&tr->w.fwd, kNetDevFloats));
    CPT_CUDA(ar.alloc(&tr->w.bwd2, kNetW2));
    CPT_CUDA(ar.alloc(&tr->w.bwd3, kNetW3));
    CPT_CUDA(ar.alloc(&tr->w.bits, kNetParams));
    const size_t P = (size_t)n * H * W;
    CPT_CUDA(launch_net_inputs(d_prev, d_next, n, H, W, tr->ws, tr->ws + 2 * P, s));
    return CPT_OK;
}

static cpt_status net_gradients_impl(const float* params, const int32_t* prev, const int32_t* next, int n, int H,
                                     int W, float* grad_out, float* loss_out, void* stream) {
    if (!params || !prev || !next || !grad_out) return fail(CPT_ERR_ARG, "null argument");
    cpt_status rc = net_dims_ok(n, H, W);
    if (rc != CPT_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevArena ar(s);
    NetTrainer tr;
    if ((rc = net_trainer_setup(ar, prev, next, n, H, W, &tr, s)) != CPT_OK) return rc;
    float* d_loss;
    CPT_CUDA(ar.alloc(&d_loss, 1));
    CPT_CUDA(cudaMemcpyAsync(tr.P, params, sizeof(float) * kNetParams, cudaMemcpyDefault, s));
    CPT_CUDA(net_train_pass(tr.P, tr.ws, n, H, W, tr.nblk, tr.part, tr.lpart, tr.w, tr.grad, d_loss, s));
    CPT_CUDA(cudaMemcpyAsync(grad_out, tr.grad, sizeof(float) * kNetParams, cudaMemcpyDefault, s));
    float loss = 0.0f;
    CPT_CUDA(cudaMemcpyAsync(&loss, d_loss, sizeof(float), cudaMemcpyDefault, s));
    CPT_CUDA(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = loss;
    return CPT_OK;
}

// Seeded initialisation: uniform(-a, a) with a = sqrt(6 / fan_in) for the
// first two layers (fan_in = 18, 288), zero last layer (the untrained net
// predicts qhat(t-1)) and zero biases.  Uniforms from splitmix64(seed * 2^32 + j).
static uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

static void net_seeded_init(uint32_t seed, float* P) {
    std::fill(P, P + kNetParams, 0.0f);
    const double a1 = std::sqrt(6.0 / 18.0), a2 = std::sqrt(6.0 / 288.0);
    auto uni = [&](int j) { return (double)(splitmix64(((uint64_t)seed << 32) + (uint64_t)j) >> 11) * 0x1p-53; };
    for (int j = 0; j < kNetW1; ++j) P[j] = (float)((2.0 * uni(j) - 1.0) * a1);
    const int o2 = kNetW1 + kNetC;
    for (int j = 0; j < kNetW2; ++j) P[o2 + j] = (float)((2.0 * uni(o2 + j) - 1.0) * a2);
}

static cpt_status net_train_impl(const int32_t* prev, const int32_t* next, int n, int H, int W, int steps, float lr,
                                 uint32_t seed, const uint16_t* init, uint16_t* model_out, float* loss_out,
                                 void* stream) {
    if (!prev || !next || !model_out) return fail(CPT_ERR_ARG, "null argument");
    if (steps < 1 || !(lr > 0.0f) || !std::isfinite(lr)) return fail(CPT_ERR_ARG, "need steps >= 1 and lr > 0");
    cpt_status rc = net_dims_ok(n, H, W);
    if (rc != CPT_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevArena ar(s);
    NetTrainer tr;
    if ((rc = net_trainer_setup(ar, prev, next, n, H, W, &tr, s)) != CPT_OK) return rc;
    std::vector<float> P0(kNetParams);
    if (init)
        for (int j = 0; j < kNetParams; ++j) P0[j] = bf16_to_float(init[j]);
    else
        net_seeded_init(seed, P0.data());
    float *d_m, *d_v, *d_loss;
    CPT_CUDA(ar.alloc(&d_m, kNetParams));
    CPT_CUDA(ar.alloc(&d_v, kNetParams));
    CPT_CUDA(ar.alloc(&d_loss, steps));
    CPT_CUDA(cudaMemsetAsync(d_m, 0, sizeof(float) * kNetParams, s));
    CPT_CUDA(cudaMemsetAsync(d_v, 0, sizeof(float) * kNetParams, s));
    CPT_CUDA(cudaMemcpyAsync(tr.P, P0.data(), sizeof(float) * kNetParams, cudaMemcpyHostToDevice, s));
    for (int k = 1; k <= steps; ++k) {
        CPT_CUDA(net_train_pass(tr.P, tr.ws, n, H, W, tr.nblk, tr.part, tr.lpart, tr.w, tr.grad, d_loss + (k - 1), s));
        CPT_CUDA(launch_adam(tr.P, d_m, d_v, tr.grad, lr, k, s));
    }
    CPT_CUDA(launch_net_prep_weights(tr.P, tr.w, s));
    CPT_CUDA(cudaMemcpyAsync(model_out, tr.w.bits, sizeof(uint16_t) * kNetParams, cudaMemcpyDefault, s));
    if (loss_out) CPT_CUDA(cudaMemcpyAsync(loss_out, d_loss, sizeof(float) * steps, cudaMemcpyDefault, s));
    CPT_CUDA(cudaStreamSynchronize(s));  // P0 is released on return
    return CPT_OK;
}

}  // namespace cpt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

cpt_status cpt_compress_ex(const float* uv, const cpt_dims* dims, const cpt_params* params, uint8_t** out,
                           size_t* out_bytes, cpt_stats* stats, const cpt_debug* dbg) {
    return cpt::compress_impl(uv, dims, params, out, out_bytes, stats, dbg);
}

cpt_status cpt_compress(const float* uv, const cpt_dims* dims, const cpt_params* params, uint8_t** out,
                        size_t* out_bytes, cpt_stats* stats) {
    return cpt::compress_impl(uv, dims, params, out, out_bytes, stats, nullptr);
}

cpt_status cpt_compress_batch(const float* const* uv, const cpt_dims* dims, int32_t nfields, const cpt_params* params,
                              size_t device_budget, uint8_t** out, size_t* out_bytes, cpt_stats* stats,
                              cpt_batch_stats* batch_stats) {
    return cpt::compress_batch_impl(uv, dims, nfields, params, device_budget, out, out_bytes, stats, batch_stats);
}

cpt_status cpt_decompress(const uint8_t* in, size_t in_bytes, float* uv_out, int32_t* qhat_out, cpt_dims* dims_out,
                          void* cuda_stream) {
    return cpt::decompress_impl(in, in_bytes, uv_out, qhat_out, dims_out, cuda_stream);
}

cpt_status cpt_extract_trajectories(const float* uv, const cpt_dims* dims, int32_t scale_log2, cpt_trajs** out,
                                    void* cuda_stream) {
    return cpt::trajectories_impl(uv, dims, scale_log2, out, cuda_stream);
}

cpt_status cpt_inject_verify_fault(int64_t vertex, int32_t delta) {
    cpt::t_vfault.vertex = vertex < 0 ? -1 : vertex;
    cpt::t_vfault.delta = delta;
    return CPT_OK;
}

cpt_status cpt_inject_wave_stall(int64_t ticket, int64_t timeout_ns) {
    if (ticket >= 0 && (ticket > 0xFFFFFFFEll || timeout_ns < 1000000 || timeout_ns > 10000000000ll))
        return cpt::fail(CPT_ERR_ARG, "ticket must fit 32 bits and the limit lie in [1 ms, 10 s]");
    cpt::t_stall.ticket = ticket < 0 ? -1 : ticket;
    cpt::t_stall.timeout_ns = timeout_ns;
    return CPT_OK;
}

cpt_status cpt_huffman_lengths(const uint64_t* freq, uint32_t nsym, int32_t maxlen, uint8_t* len) {
    if ((!freq && nsym) || (!len && nsym) || maxlen < 1 || maxlen > 32)
        return cpt::fail(CPT_ERR_ARG, "null argument or code length limit outside [1, 32]");
    std::vector<uint64_t> f(freq, freq + nsym);
    std::vector<uint8_t> l;
    if (!cpt::huffman_lengths(f, maxlen, l)) return cpt::fail(CPT_ERR_ARG, "alphabet too large for the limit");
    std::copy(l.begin(), l.end(), len);
    return CPT_OK;
}

cpt_status cpt_pipeline_order(int32_t nfields, const int32_t* fields, const int32_t* schedule, int32_t* items,
                              uint64_t* n_items) {
    if (nfields < 1 || !fields || !n_items) return cpt::fail(CPT_ERR_ARG, "null argument or no field");
    std::vector<cpt::OrderField> fs((size_t)nfields);
    unsigned long long total = 0;
    for (int f = 0; f < nfields; ++f) {
        const int32_t* g = fields + 4 * (size_t)f;
        if (g[0] < 1 || g[1] < 1 || g[2] < 0) return cpt::fail(CPT_ERR_ARG, "need T, H >= 1 and R >= 0");
        fs[f] = {g[0], (g[1] + 31) / 32, g[2], g[3] ? 1u : 0u};
        total += (unsigned long long)fs[f].T * fs[f].nstrips;
    }
    if (total >= 0x7FFFFFFFull) return cpt::fail(CPT_ERR_ARG, "too many wave items");
    *n_items = total;
    if (!items) return CPT_OK;
    const cpt::PipeTuning tune = schedule ? cpt::PipeTuning{schedule[0], schedule[1], schedule[2], schedule[3],
                                                            schedule[4], schedule[5]}
                                          : cpt::PipeTuning{};
    std::vector<int4> order;
    cpt::merged_order(fs, tune, order);
    for (size_t x = 0; x < order.size(); ++x) {
        items[3 * x] = order[x].x;
        items[3 * x + 1] = order[x].y;
        items[3 * x + 2] = order[x].z;
    }
    return CPT_OK;
}

cpt_status cpt_net_predict(const uint16_t* model, const int32_t* prev, int32_t H, int32_t W, int32_t* pred_out,
                           void* cuda_stream) {
    return cpt::net_predict_impl(model, prev, H, W, pred_out, cuda_stream);
}

cpt_status cpt_net_gradients(const float* params, const int32_t* prev, const int32_t* next, int32_t n, int32_t H,
                             int32_t W, float* grad_out, float* loss_out, void* cuda_stream) {
    return cpt::net_gradients_impl(params, prev, next, n, H, W, grad_out, loss_out, cuda_stream);
}

cpt_status cpt_train_predictor(const int32_t* prev, const int32_t* next, int32_t n, int32_t H, int32_t W,
                               int32_t steps, float lr, uint32_t seed, const uint16_t* init, uint16_t* model_out,
                               float* loss_out, void* cuda_stream) {
    return cpt::net_train_impl(prev, next, n, H, W, steps, lr, seed, init, model_out, loss_out, cuda_stream);
}

void cpt_free(void* p) {
    if (p && !cpt::pinned_pool().put(p)) std::free(p);
}

void cpt_free_trajs(cpt_trajs* t) {
    if (!t) return;
    std::free(t->offsets);
    std::free(t->face_ids);
    std::free(t->xyt);
    std::free(t);
}

const char* cpt_error_string(cpt_status s) {
    switch (s) {
        case CPT_OK: return "ok";
        case CPT_ERR_ARG: return "invalid argument";
        case CPT_ERR_CUDA: return "CUDA error";
        case CPT_ERR_OOM: return "out of memory";
        case CPT_ERR_CORRUPT: return "corrupt stream";
        case CPT_ERR_VERIFY: return "verification failed";
        case CPT_ERR_TIMEOUT: return "kernel wait timed out";
        case CPT_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char* cpt_last_error(void) { return cpt::g_last_error.c_str(); }

uint32_t cpt_version(void) { return (1u << 8) | cpt::kFormat; }

}  // extern "C"
