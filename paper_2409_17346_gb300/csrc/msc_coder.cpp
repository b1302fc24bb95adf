// Lossless coding of edit records (Sec. 4.7; Sec. 5.5, where the paper compresses the edits
// of both forms with ZSTD before it compares their sizes).
//
// The coder is the system's zstd library, loaded on first use through its public C API
// (ZSTD_compress / ZSTD_decompress and their helpers), so the library builds without zstd's
// headers and still loads where zstd is absent; the calls here then report
// MSC_ERR_UNAVAILABLE.  A coded record is one zstd frame whose content size is recorded in
// the frame header, so decoding needs no side information.
#include <dlfcn.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/msc.h"
#include "msc_runtime.h"

namespace {

struct Zstd {
    size_t (*compress_bound)(size_t) = nullptr;
    size_t (*compress)(void *, size_t, const void *, size_t, int) = nullptr;
    size_t (*decompress)(void *, size_t, const void *, size_t) = nullptr;
    unsigned (*is_error)(size_t) = nullptr;
    const char *(*error_name)(size_t) = nullptr;
    unsigned long long (*frame_content_size)(const void *, size_t) = nullptr;
    int (*max_level)(void) = nullptr;
    bool ok = false;
    std::string why;
};

const Zstd &zstd()
{
    static Zstd z;
    static std::once_flag once;
    std::call_once(once, [] {
        void *h = nullptr;
        for (const char *name : {"libzstd.so.1", "libzstd.so"}) {
            h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
            if (h) break;
        }
        if (!h) {
            const char *e = dlerror();
            z.why = std::string("libzstd could not be loaded: ") + (e ? e : "unknown error");
            return;
        }
        z.compress_bound = (size_t(*)(size_t))dlsym(h, "ZSTD_compressBound");
        z.compress = (size_t(*)(void *, size_t, const void *, size_t, int))dlsym(h, "ZSTD_compress");
        z.decompress = (size_t(*)(void *, size_t, const void *, size_t))dlsym(h, "ZSTD_decompress");
        z.is_error = (unsigned (*)(size_t))dlsym(h, "ZSTD_isError");
        z.error_name = (const char *(*)(size_t))dlsym(h, "ZSTD_getErrorName");
        z.frame_content_size = (unsigned long long (*)(const void *, size_t))dlsym(h, "ZSTD_getFrameContentSize");
        z.max_level = (int (*)(void))dlsym(h, "ZSTD_maxCLevel");
        z.ok = z.compress_bound && z.compress && z.decompress && z.is_error && z.error_name && z.frame_content_size &&
               z.max_level;
        if (!z.ok) z.why = "libzstd lacks one of the functions the coder needs";
    });
    return z;
}

// zstd's frame-size sentinels (ZSTD_CONTENTSIZE_UNKNOWN / _ERROR)
constexpr unsigned long long SIZE_UNKNOWN = ~0ull, SIZE_ERROR = ~0ull - 1;

}  // namespace

extern "C" {

uint64_t msc_coded_bound(uint64_t size)
{
    const Zstd &z = zstd();
    return z.ok ? (uint64_t)z.compress_bound((size_t)size) : 0;
}

msc_status msc_code_record(const uint8_t *rec, uint64_t size, int level, uint8_t *out, uint64_t cap, uint64_t *n_out)
{
    if (!n_out || (size && !rec)) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "rec and n_out must be non-NULL");
    *n_out = 0;
    const Zstd &z = zstd();
    if (!z.ok) return msc_rt::set_error(MSC_ERR_UNAVAILABLE, z.why);
    if (level < 1 || level > z.max_level())
        return msc_rt::set_error(MSC_ERR_INVALID_ARG, "level must be 1.." + std::to_string(z.max_level()));
    const size_t bound = z.compress_bound((size_t)size);
    if (!out || cap < bound)
        return msc_rt::set_error(MSC_ERR_INVALID_ARG, "out needs msc_coded_bound(size) = " + std::to_string(bound) +
                                                          " bytes");
    const size_t r = z.compress(out, (size_t)cap, rec, (size_t)size, level);
    if (z.is_error(r)) return msc_rt::set_error(MSC_ERR_INVALID_ARG, std::string("zstd: ") + z.error_name(r));
    *n_out = r;
    return MSC_OK;
}

msc_status msc_decoded_size(const uint8_t *in, uint64_t size, uint64_t *n_out)
{
    if (!in || !n_out) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "in and n_out must be non-NULL");
    const Zstd &z = zstd();
    if (!z.ok) return msc_rt::set_error(MSC_ERR_UNAVAILABLE, z.why);
    const unsigned long long n = z.frame_content_size(in, (size_t)size);
    if (n == SIZE_UNKNOWN || n == SIZE_ERROR) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "not a coded record");
    *n_out = n;
    return MSC_OK;
}

msc_status msc_decode_record(const uint8_t *in, uint64_t size, uint8_t *out, uint64_t cap, uint64_t *n_out)
{
    if (!in || !n_out) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "in and n_out must be non-NULL");
    *n_out = 0;
    const Zstd &z = zstd();
    if (!z.ok) return msc_rt::set_error(MSC_ERR_UNAVAILABLE, z.why);
    uint64_t want = 0;
    const msc_status st = msc_decoded_size(in, size, &want);
    if (st != MSC_OK) return st;
    if ((want && !out) || cap < want)
        return msc_rt::set_error(MSC_ERR_INVALID_ARG, "out needs " + std::to_string(want) + " bytes");
    const size_t r = z.decompress(out, (size_t)cap, in, (size_t)size);
    if (z.is_error(r)) return msc_rt::set_error(MSC_ERR_INVALID_ARG, std::string("zstd: ") + z.error_name(r));
    if (r != want) return msc_rt::set_error(MSC_ERR_INVALID_ARG, "decoded size differs from the frame header");
    *n_out = r;
    return MSC_OK;
}

}  // extern "C"
