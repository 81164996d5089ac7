// Optional lossless back end of the stream: the general-purpose lossless
// stage that follows the Huffman coder in the compressor's pipeline (Alg. 3,
// lossless_comp; the paper uses ZSTD).  It is applied on the host to the
// finished stream, so the stream inside is byte for byte the stream without
// it.  libzstd is loaded when first needed (dlopen of libzstd.so.1, with the
// library's public prototypes declared below); without it the option returns
// CPT_ERR_UNSUPPORTED.
//
// Container: "CPTZ", u32 version (1), u64 bytes of the stream inside, then one
// ZSTD frame holding the stream.  All integers little-endian.
#include <dlfcn.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "cpt.h"
#include "cpt_internal.h"

namespace cpt {

cpt_status fail_status(cpt_status s, const char* msg);  // cpt_host.cu

namespace {

struct ZstdLib {
    size_t (*bound)(size_t) = nullptr;
    size_t (*compress)(void*, size_t, const void*, size_t, int) = nullptr;
    size_t (*decompress)(void*, size_t, const void*, size_t) = nullptr;
    unsigned (*is_error)(size_t) = nullptr;
    int (*max_level)(void) = nullptr;
    bool ok = false;
};

const ZstdLib& zstd_lib() {
    static ZstdLib z;
    static std::once_flag once;
    std::call_once(once, [] {
        void* h = dlopen("libzstd.so.1", RTLD_NOW | RTLD_LOCAL);
        if (!h) return;
        z.bound = reinterpret_cast<size_t (*)(size_t)>(dlsym(h, "ZSTD_compressBound"));
        z.compress = reinterpret_cast<size_t (*)(void*, size_t, const void*, size_t, int)>(dlsym(h, "ZSTD_compress"));
        z.decompress = reinterpret_cast<size_t (*)(void*, size_t, const void*, size_t)>(dlsym(h, "ZSTD_decompress"));
        z.is_error = reinterpret_cast<unsigned (*)(size_t)>(dlsym(h, "ZSTD_isError"));
        z.max_level = reinterpret_cast<int (*)(void)>(dlsym(h, "ZSTD_maxCLevel"));
        z.ok = z.bound && z.compress && z.decompress && z.is_error && z.max_level;
    });
    return z;
}

constexpr size_t kZHeader = 4 + 4 + 8;
constexpr uint32_t kZVersion = 1;

void put_u32(uint8_t* p, uint32_t x) {
    for (int b = 0; b < 4; ++b) p[b] = (uint8_t)(x >> (8 * b));
}
void put_u64(uint8_t* p, uint64_t x) {
    for (int b = 0; b < 8; ++b) p[b] = (uint8_t)(x >> (8 * b));
}
uint64_t get_u64(const uint8_t* p) {
    uint64_t x = 0;
    for (int b = 7; b >= 0; --b) x = (x << 8) | p[b];
    return x;
}
uint32_t get_u32(const uint8_t* p) {
    uint32_t x = 0;
    for (int b = 3; b >= 0; --b) x = (x << 8) | p[b];
    return x;
}

}  // namespace

bool zstd_available() { return zstd_lib().ok; }

bool is_zstd_container(const uint8_t* in, size_t n) { return in && n >= 4 && std::memcmp(in, "CPTZ", 4) == 0; }

// Wraps n bytes into a malloc'd container (ownership to the caller).
cpt_status zstd_wrap(const uint8_t* in, size_t n, int level, uint8_t** out, size_t* out_n) {
    const ZstdLib& z = zstd_lib();
    if (!z.ok) return fail_status(CPT_ERR_UNSUPPORTED, "libzstd.so.1 is not available");
    if (level < 1 || level > z.max_level()) return fail_status(CPT_ERR_ARG, "zstd level out of range");
    const size_t cap = z.bound(n);
    uint8_t* buf = static_cast<uint8_t*>(std::malloc(kZHeader + cap));
    if (!buf) return fail_status(CPT_ERR_OOM, "host allocation failed");
    const size_t m = z.compress(buf + kZHeader, cap, in, n, level);
    if (z.is_error(m)) {
        std::free(buf);
        return fail_status(CPT_ERR_ARG, "zstd compression failed");
    }
    std::memcpy(buf, "CPTZ", 4);
    put_u32(buf + 4, kZVersion);
    put_u64(buf + 8, (uint64_t)n);
    *out = buf;
    *out_n = kZHeader + m;
    return CPT_OK;
}

// The stream inside a container, malloc'd (ownership to the caller).
cpt_status zstd_unwrap(const uint8_t* in, size_t n, uint8_t** out, size_t* out_n) {
    if (!is_zstd_container(in, n) || n < kZHeader) return fail_status(CPT_ERR_CORRUPT, "not a zstd container");
    if (get_u32(in + 4) != kZVersion) return fail_status(CPT_ERR_CORRUPT, "unknown zstd container version");
    const ZstdLib& z = zstd_lib();
    if (!z.ok) return fail_status(CPT_ERR_UNSUPPORTED, "libzstd.so.1 is not available");
    const uint64_t raw = get_u64(in + 8);
    if (raw > ((uint64_t)1 << 46)) return fail_status(CPT_ERR_CORRUPT, "implausible stream size");
    uint8_t* buf = static_cast<uint8_t*>(std::malloc(raw ? (size_t)raw : 1));
    if (!buf) return fail_status(CPT_ERR_OOM, "host allocation failed");
    const size_t m = z.decompress(buf, (size_t)raw, in + kZHeader, n - kZHeader);
    if (z.is_error(m) || m != raw) {
        std::free(buf);
        return fail_status(CPT_ERR_CORRUPT, "zstd frame does not decode to the stated size");
    }
    *out = buf;
    *out_n = (size_t)raw;
    return CPT_OK;
}

}  // namespace cpt

extern "C" cpt_status cpt_zstd_wrap(const uint8_t* in, size_t in_bytes, int32_t level, uint8_t** out,
                                    size_t* out_bytes) {
    if (!in || !out || !out_bytes) return cpt::fail_status(CPT_ERR_ARG, "null argument");
    *out = nullptr;
    *out_bytes = 0;
    return cpt::zstd_wrap(in, in_bytes, level, out, out_bytes);
}

extern "C" cpt_status cpt_zstd_unwrap(const uint8_t* in, size_t in_bytes, uint8_t** out, size_t* out_bytes) {
    if (!in || !out || !out_bytes) return cpt::fail_status(CPT_ERR_ARG, "null argument");
    *out = nullptr;
    *out_bytes = 0;
    return cpt::zstd_unwrap(in, in_bytes, out, out_bytes);
}
