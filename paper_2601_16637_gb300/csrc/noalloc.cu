// String validation and sorting without any device allocation.
//
// Some callers cannot let a library allocate device memory on their behalf:
// a serving process whose device memory is carved up in advance by its own
// allocator, a plug-in that runs inside another framework's process and must
// not grow that process's footprint, or a latency-critical loop that may not
// touch an allocator at all.  sbd_sort_strings_noalloc gives them the string
// ingestion step (validate, sort, reject duplicates) with its work space in a
// fixed array that lives in the library itself: the caller passes the input
// and output buffers, and nothing else is allocated.
//
// The work space is one file-scope __device__ array of kNoAllocBytes: a
// ping-pong buffer for kNoAllocMaxStrings strings plus the status words.
// Every GPU that loads the library holds it until the process exits.  All
// calls share it, so calls that overlap on the GPU (on different streams, or
// from different host threads) race on it and must be serialised by the caller.
#include <mutex>

#include "common.cuh"

namespace sbd {
namespace {

constexpr int64_t kNoAllocMaxStrings = SBD_NOALLOC_MAX_STRINGS;
constexpr size_t kStatusOffset = (size_t)kNoAllocMaxStrings * sizeof(uint64_t);
constexpr size_t kNoAllocBytes = kStatusOffset + 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the work space on the current device.  Host code only holds a
// host-side stand-in under the array's name, so the address is looked up once per
// device (with that device current) and cached.  The cache assumes that the device's
// CUDA context lives as long as the library stays loaded: after a cudaDeviceReset the
// cached address would name memory of the destroyed context.
void *scratch_on_current_device()
{
    int dev = 0;
    SBD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(SBD_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        SBD_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

}  // namespace
}  // namespace sbd

using namespace sbd;

extern "C" int sbd_sort_strings_noalloc(const uint64_t *keys_dev, int64_t n, int norb, int nel, uint64_t *sorted_dev,
                                        int64_t *bad_index_host, void *stream)
{
    if (bad_index_host) *bad_index_host = -1;
    if (norb < 1 || norb > 64) {
        set_thread_error("norb must be in 1..64");
        return SBD_ERR_NORB;
    }
    if (n < 0 || nel < 0 || nel > norb || (n > 0 && (!keys_dev || !sorted_dev))) {
        set_thread_error("invalid argument to sbd_sort_strings_noalloc");
        return SBD_ERR_INVALID_ARG;
    }
    if (n > kNoAllocMaxStrings) {
        set_thread_error("sbd_sort_strings_noalloc takes at most SBD_NOALLOC_MAX_STRINGS (65536) strings; "
                             "use sbd_create for larger sets");
        return SBD_ERR_INVALID_ARG;
    }
    try {
        cudaStream_t s = (cudaStream_t)stream;
        unsigned char *base = static_cast<unsigned char *>(scratch_on_current_device());
        uint64_t *tmp = reinterpret_cast<uint64_t *>(base);
        DevStatus *st = reinterpret_cast<DevStatus *>(base + kStatusOffset);
        sort_validate_into(keys_dev, n, norb, nel, sorted_dev, tmp, st, s);
        DevStatus h{};
        SBD_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
        SBD_CUDA(cudaStreamSynchronize(s));
        if (h.first_bad != ~0ull) {
            if (bad_index_host) *bad_index_host = (int64_t)h.first_bad;
            set_thread_error("a string has the wrong electron count or a bit >= norb");
            return SBD_ERR_BAD_STRING;
        }
        if (h.first_dup != ~0ull) {
            if (bad_index_host) *bad_index_host = (int64_t)h.first_dup;
            set_thread_error("the strings contain a duplicate");
            return SBD_ERR_DUPLICATE_STRING;
        }
        return SBD_OK;
    } catch (const Error &e) {
        set_thread_error(e.msg.c_str());
        return e.code;
    } catch (...) {
        set_thread_error("unexpected internal error");
        return SBD_ERR_CUDA;
    }
}
