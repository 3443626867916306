// Allocation-free Morton ordering (declared in include/ff.h).
//
// Some callers may not allocate device memory at all: applications whose
// device memory is owned by their own pool or allocator (which must see every
// byte), and latency-bound loops that cannot afford an allocation on the way
// (cudaMalloc may synchronise the device).  For them this entry point
// computes the root cube, the 63-bit Morton keys and the stable key sort of
// up to kNoAllocMaxN particles using only the caller's input and output
// buffers plus one fixed scratch array that lives in this file.  The call
// reads its error word back to the host and waits for the stream, so it
// cannot be issued while that stream is being captured into a graph.
//
// The scratch array is a static device variable: every GPU that loads the
// library keeps it (about 3.7 MB) until the process exits.  Its name in host
// code is only a host-side stand-in, so the device address is looked up with
// cudaGetSymbolAddress, once per device, on the first call made with that
// device current; the address is kept for the life of the process, so the
// entry point must not be used on a device after cudaDeviceReset.  All calls
// share the array and it keeps the contents of the last call; calls whose GPU
// work overlaps (different streams, or several host threads on one device)
// race on it.
#include <cstddef>
#include <cstdio>
#include <mutex>

#include "ff.h"
#include "ffk.cuh"

namespace {

constexpr int64_t kNoAllocMaxN = 131072;
constexpr int kMaxDevices = 64;

// Scratch layout (bytes, each part 256-byte aligned): position records,
// second key/value buffers of the radix sort, radix histograms and scan
// space, root-cube extrema, error flags.
constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kRecOff = 0;
constexpr size_t kRecBytes = align256(sizeof(float4) * kNoAllocMaxN);
constexpr size_t kKeyOff = kRecOff + kRecBytes;
constexpr size_t kKeyBytes = align256(sizeof(uint64_t) * kNoAllocMaxN);
constexpr size_t kValOff = kKeyOff + kKeyBytes;
constexpr size_t kValBytes = align256(sizeof(uint32_t) * kNoAllocMaxN);
constexpr size_t kRadixOff = kValOff + kValBytes;
// radix scratch: the one-sweep sort's pass counts, tile status words and tickets
constexpr size_t kRadixWords = ffk::os_tmp_words(kNoAllocMaxN);
constexpr size_t kRadixBytes = align256(sizeof(uint32_t) * kRadixWords);
constexpr size_t kBoxOff = kRadixOff + kRadixBytes;
constexpr size_t kBoxBytes = align256(sizeof(ffk::BBox));
constexpr size_t kFlagOff = kBoxOff + kBoxBytes;
constexpr size_t kScratchBytes = kFlagOff + 256;

}  // namespace

static __device__ __align__(256) unsigned char ff_noalloc_scratch[kScratchBytes];

namespace {

static_assert(kNoAllocMaxN == FF_NOALLOC_MAX_N, "scratch sized for FF_NOALLOC_MAX_N");

std::mutex g_mutex;
unsigned char* g_base[kMaxDevices] = {nullptr};

// The reason is reported through ff_last_error(NULL) on the calling thread.
ff_status noalloc_fail(ff_status s, const char* msg, cudaError_t e = cudaSuccess)
{
    char buf[256];
    if (e != cudaSuccess)
        std::snprintf(buf, sizeof(buf), "ff_morton_order_noalloc: %s: %s", msg, cudaGetErrorString(e));
    else
        std::snprintf(buf, sizeof(buf), "ff_morton_order_noalloc: %s", msg);
    ffk::set_thread_error(buf);
    return s;
}

// Device address of the scratch array on the current device (set up once per
// device with that device current).
ff_status scratch_base(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(FF_ECUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(FF_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_base[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, ff_noalloc_scratch);
        if (e != cudaSuccess) return noalloc_fail(FF_ECUDA, "cudaGetSymbolAddress", e);
        g_base[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_base[dev];
    return FF_OK;
}

}  // namespace

extern "C" {

ff_status ff_morton_order_noalloc(const float* pos, int64_t n, uint64_t* keys_out,
                                  uint32_t* order_out, void* stream)
{
    if (!pos || !keys_out || !order_out) return noalloc_fail(FF_EINVAL, "pos, keys_out and order_out are required");
    if (n < 1 || n > kNoAllocMaxN) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "n = %lld is outside 1 .. %lld, the size of the fixed scratch",
                      (long long)n, (long long)kNoAllocMaxN);
        return noalloc_fail(FF_EINVAL, msg);
    }
    if (ffk::radix_tmp_words(n) > kRadixWords) return noalloc_fail(FF_EINVAL, "radix scratch too small");
    unsigned char* base = nullptr;
    ff_status st = scratch_base(&base);
    if (st != FF_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float4* rec = reinterpret_cast<float4*>(base + kRecOff);
    uint64_t* k1 = reinterpret_cast<uint64_t*>(base + kKeyOff);
    uint32_t* v1 = reinterpret_cast<uint32_t*>(base + kValOff);
    uint32_t* rtmp = reinterpret_cast<uint32_t*>(base + kRadixOff);
    ffk::BBox* bb = reinterpret_cast<ffk::BBox*>(base + kBoxOff);
    int* flags = reinterpret_cast<int*>(base + kFlagOff);
    // the flag word must start at zero; everything else is rewritten in full
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int), s);
    if (e != cudaSuccess) return noalloc_fail(FF_ECUDA, "cudaMemsetAsync", e);
    ffk::load3<float, float>(pos, n, rec, s);
    // keys and values are built directly in the caller's outputs, which the
    // eight-pass sort leaves holding the sorted data
    ffk::morton_keys<float>(rec, n, bb, keys_out, order_out, flags, ffk::Segs(), s);
    ffk::radix_sort_pairs(keys_out, order_out, k1, v1, n, rtmp, flags, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(FF_ECUDA, "kernel launch", e);
    int hflag = 0;
    e = cudaMemcpyAsync(&hflag, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return noalloc_fail(FF_ECUDA, "cudaMemcpyAsync", e);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(FF_ECUDA, "cudaStreamSynchronize", e);
    if (hflag & ffk::FLAG_NONFINITE) return noalloc_fail(FF_ENONFINITE, "a particle position is NaN or infinite");
    if (hflag & ffk::FLAG_SORT)
        return noalloc_fail(FF_EDEVICE, "a sort tile gave up waiting for an earlier tile's counts");
    return FF_OK;
}

// Self-test of the sort's bounded wait: distinct synthetic keys, values 0..n-1.
__global__ void k_selftest_keys(uint64_t* __restrict__ k, uint32_t* __restrict__ v, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    k[i] = ((uint64_t)i * 0x9E3779B97F4A7C15ull) >> 1;
    v[i] = (uint32_t)i;
}

ff_status ff_selftest_sort_wait(int64_t n, void* stream)
{
    if (n < 2 * ffk::kOsTile || n > (int64_t)1 << 24)
        return noalloc_fail(FF_EINVAL, "n must span at least two sort tiles (8192 .. 2^24)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t* k[2] = {nullptr, nullptr};
    uint32_t* v[2] = {nullptr, nullptr};
    uint32_t* tmp = nullptr;
    int* flags = nullptr;
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
        e = cudaMalloc(&k[q], sizeof(uint64_t) * n);
        if (e == cudaSuccess) e = cudaMalloc(&v[q], sizeof(uint32_t) * n);
    }
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(uint32_t) * ffk::radix_tmp_words(n));
    if (e == cudaSuccess) e = cudaMalloc(&flags, sizeof(int));
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_selftest_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(k[0], v[0], n);
        ffk::radix_sort_wait_selftest(k[0], v[0], k[1], v[1], n, tmp, flags, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const cudaError_t e_run = e;
    for (int q = 0; q < 2; ++q) {
        cudaFree(k[q]);
        cudaFree(v[q]);
    }
    cudaFree(tmp);
    cudaFree(flags);
    if (e_run != cudaSuccess) return noalloc_fail(FF_ECUDA, "sort wait self-test", e_run);
    if (!(hflag & ffk::FLAG_SORT))
        return noalloc_fail(FF_EDEVICE, "the sort's look-back wait did not run out with a tile withheld");
    return FF_OK;
}

// Synthetic sorted records: record i has key i / 4, index i and one entry.
__global__ void k_selftest_records(uint32_t* __restrict__ key, uint32_t* __restrict__ idx,
                                   uint2* __restrict__ rec, int64_t nrec,
                                   uint32_t* __restrict__ src_of, int64_t nsrc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nrec) {
        key[i] = (uint32_t)(i / 4);
        idx[i] = (uint32_t)i;
        rec[i] = make_uint2((uint32_t)i, 1u);
    }
    if (i < nsrc) src_of[i] = (uint32_t)i;
}

ff_status ff_selftest_record_wait(int64_t nrec, void* stream)
{
    const int64_t tile = ffk::record_scan_tile();
    if (nrec < 2 * tile || nrec > (int64_t)1 << 24)
        return noalloc_fail(FF_EINVAL, "nrec must span at least two scan tiles (4096 .. 2^24)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nsrc = nrec / 4 + 1;
    uint32_t *key = nullptr, *idx = nullptr, *src_of = nullptr, *recE = nullptr;
    uint32_t *rbeg = nullptr, *beg = nullptr, *end = nullptr;
    uint2 *rec = nullptr, *srec = nullptr;
    unsigned long long* words = nullptr;
    int* flags = nullptr;
    cudaError_t e = cudaMalloc(&key, sizeof(uint32_t) * nrec);
    if (e == cudaSuccess) e = cudaMalloc(&idx, sizeof(uint32_t) * nrec);
    if (e == cudaSuccess) e = cudaMalloc(&rec, sizeof(uint2) * nrec);
    if (e == cudaSuccess) e = cudaMalloc(&srec, sizeof(uint2) * nrec);
    if (e == cudaSuccess) e = cudaMalloc(&recE, sizeof(uint32_t) * (nrec + 1));
    if (e == cudaSuccess) e = cudaMalloc(&src_of, sizeof(uint32_t) * nsrc);
    if (e == cudaSuccess) e = cudaMalloc(&rbeg, sizeof(uint32_t) * nsrc);
    if (e == cudaSuccess) e = cudaMalloc(&beg, sizeof(uint32_t) * nsrc);
    if (e == cudaSuccess) e = cudaMalloc(&end, sizeof(uint32_t) * nsrc);
    if (e == cudaSuccess) e = cudaMalloc(&words, sizeof(unsigned long long) * ffk::record_scan_words(nrec));
    if (e == cudaSuccess) e = cudaMalloc(&flags, sizeof(int));
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_selftest_records<<<(unsigned)((nrec + 255) / 256), 256, 0, s>>>(key, idx, rec, nrec,
                                                                          src_of, nsrc);
        ffk::record_scan_wait_selftest(key, idx, nrec, rec, src_of, nsrc, srec, recE, words, rbeg,
                                       beg, end, flags, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const cudaError_t e_run = e;
    void* bufs[] = {key, idx, rec, srec, recE, src_of, rbeg, beg, end, words, flags};
    for (void* b : bufs) cudaFree(b);
    if (e_run != cudaSuccess) return noalloc_fail(FF_ECUDA, "record scan wait self-test", e_run);
    if (!(hflag & ffk::FLAG_SORT))
        return noalloc_fail(FF_EDEVICE, "the record scan's look-back wait did not run out with a tile withheld");
    return FF_OK;
}

}  // extern "C"
