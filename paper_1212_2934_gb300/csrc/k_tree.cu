// Octree construction on the GPU (Sec. 3.2, kernels 1-4 of the paper's
// scheme, redesigned): root cube by reduction, 63-bit Morton keys, a stable
// LSD radix sort, and a parallel build of the depth-first-preorder octree
// straight from the sorted keys, followed by one bottom-up aggregation
// launch.  The build needs no locks and the aggregation uses arrival counters
// (the last child to arrive sums its parent).  The only waits on other blocks
// are the sort's look-back polls, on tiles with earlier tickets (already
// running), each bounded, so every loop ends.
#include <climits>
#include <mutex>

#include "ffk.cuh"

namespace ffk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one value per thread over a 256-thread block.
__device__ uint32_t block_exscan(uint32_t v, uint32_t* total)
{
    __shared__ uint32_t ws[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? ws[lane] : 0u;
#pragma unroll
        for (int o = 1; o < kScanThreads / 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) ws[lane] = w;
    }
    __syncthreads();
    uint32_t pre = warp ? ws[warp - 1] : 0u;
    *total = ws[kScanThreads / 32 - 1];
    __syncthreads();
    return pre + x - v;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, int64_t n,
                              uint32_t* __restrict__ bsum)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < n) s += in[base + j];
    uint32_t tot;
    block_exscan(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums in place; bsum[nb] = total,
// out_total (if non-null) = total.
__global__ void k_scan_top(uint32_t* __restrict__ bsum, int64_t nb, uint32_t* out_total)
{
    uint32_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanTile) {
        const int64_t b0 = base + (int64_t)threadIdx.x * kScanItems;
        uint32_t v[kScanItems];
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            v[j] = (b0 + j < nb) ? bsum[b0 + j] : 0u;
            s += v[j];
        }
        uint32_t tot;
        uint32_t ex = block_exscan(s, &tot) + carry;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            if (b0 + j < nb) bsum[b0 + j] = ex;
            ex += v[j];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        bsum[nb] = carry;
        if (out_total) *out_total = carry;
    }
}

__global__ void k_scan_down(const uint32_t* __restrict__ in, int64_t n,
                            const uint32_t* __restrict__ bsum, uint32_t* __restrict__ out)
{
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = (base + j < n) ? in[base + j] : 0u;
        s += v[j];
    }
    uint32_t tot;
    uint32_t ex = block_exscan(s, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = ex;
        ex += v[j];
    }
}

// ---------------------------------------------------- one-sweep radix sort
// Digit of a sort element: 8 bits of its key at `shift` or, in a system pass
// (sysd != null), of the system that owned the element's pre-sort position
// (its value).
template <typename K>
__device__ __forceinline__ uint32_t os_digit(K key, uint32_t val, const uint32_t* __restrict__ sysd,
                                             int shift)
{
    return sysd ? (sysd[val] >> shift) & (kRadixBins - 1)
                : (uint32_t)(key >> shift) & (kRadixBins - 1);
}

// Digit counts of every pass in one read of the keys.
template <typename K>
__global__ void __launch_bounds__(kOsThreads) k_os_hist(const K* __restrict__ keys,
                                                        const uint32_t* __restrict__ vals,
                                                        const uint32_t* __restrict__ sysd,
                                                        int64_t n, int passes,
                                                        uint32_t* __restrict__ hist)
{
    __shared__ uint32_t h[kOsMaxPasses][kRadixBins];
    const int t = threadIdx.x;
    for (int p = 0; p < passes; ++p) h[p][t] = 0;
    __syncthreads();
    // keys arrive nearly sorted (the previous step's order), so the high digits
    // of a warp's 32 keys usually agree: such a digit is added once per warp
    const int lane = t & 31;
    for (int64_t i0 = (int64_t)blockIdx.x * kOsThreads; i0 < n; i0 += (int64_t)gridDim.x * kOsThreads) {
        const int64_t i = i0 + t;
        const bool valid = i < n;
        const K key = valid ? keys[i] : K(0);
        const uint32_t val = (valid && sysd) ? vals[i] : 0u;
        const bool whole = __all_sync(kFull, valid);
        for (int p = 0; p < passes; ++p) {
            const uint32_t d = os_digit<K>(key, val, sysd, p * kRadixBits);
            if (whole && __all_sync(kFull, d == __shfl_sync(kFull, d, 0))) {
                if (lane == 0) atomicAdd(&h[p][d], 32u);
            } else if (valid) {
                atomicAdd(&h[p][d], 1u);
            }
        }
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p)
        if (h[p][t]) atomicAdd(&hist[p * kRadixBins + t], h[p][t]);
}

// Tile status word of the look-back: the digit's count in the low 32 bits and
// what it covers in the high bits (0: not yet written).
constexpr unsigned long long kOsAggregate = 1ull << 32;  // this tile alone
constexpr unsigned long long kOsPrefix = 2ull << 32;     // this tile and all before it
constexpr int kOsSpinLimit = 1 << 22;                    // polls before a tile gives up
constexpr int kOsWindow = 8;                             // status words read per look-back trip

// One stable pass over the digit at `shift`.  Blocks take tiles in ticket
// order.  Each warp ranks its contiguous share of the tile in rounds of 32
// (match masks within the round, per-warp digit counters across rounds); the
// tile's count of each digit is published at once, then the tile sums the
// counts of the tiles before it (walking back until a tile that has published
// its inclusive prefix) and publishes its own prefix.  A tile waits only for
// tiles with earlier tickets, which are already running, and every wait is
// bounded.  The tile is reordered in shared memory by digit before the look-back
// and written after it, consecutive threads storing consecutive elements of
// one run.
template <typename K>
__global__ void __launch_bounds__(kOsThreads, os_min_blocks<K>()) k_os_scatter(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
    uint32_t* __restrict__ vout, int64_t n, int shift, const uint32_t* __restrict__ hist,
    unsigned long long* status, unsigned long long* __restrict__ status_next,
    uint32_t* ticket, int* flags, const uint32_t* __restrict__ sysd, int withhold)
{
    constexpr int kWarps = kOsThreads / 32;
    constexpr int kItems = os_items<K>();
    constexpr int kTile = kOsThreads * kItems;
    constexpr int kWarpItems = kTile / kWarps;
    static_assert(kWarpItems == 32 * kItems, "each warp ranks kItems rounds of 32");
    extern __shared__ __align__(16) unsigned char os_smem[];  // os_dyn_smem<K>() bytes
    K* s_key = reinterpret_cast<K*>(os_smem);
    uint32_t* s_val = reinterpret_cast<uint32_t*>(os_smem + sizeof(K) * kTile);
    __shared__ uint32_t s_wcnt[kWarps][kRadixBins];  // per-warp digit counts, then prefixes
    __shared__ uint32_t s_dstart[kRadixBins];        // where each digit starts in the tile
    __shared__ uint32_t s_gstart[kRadixBins];        // where this tile's run of it goes
    __shared__ uint32_t s_tile;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    if (t == 0) s_tile = atomicAdd(ticket, 1u);
#pragma unroll
    for (int j = 0; j < kRadixBins / 32; ++j) s_wcnt[w][lane + 32 * j] = 0;
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kTile;
    const int tile_n = (int)min((int64_t)kTile, n - base);
    // the words of this tile in the array the next pass uses
    status_next[tile * kRadixBins + t] = 0ull;

    K key[kItems];
    uint32_t val[kItems], rank[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int e = w * kWarpItems + r * 32 + lane;
        if (e < tile_n) {
            key[r] = kin[base + e];
            val[r] = vin[base + e];
        }
    }
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int e = w * kWarpItems + r * 32 + lane;
        const bool valid = e < tile_n;
        const uint32_t d = valid ? os_digit<K>(key[r], val[r], sysd, shift) : (uint32_t)kRadixBins;
        const uint32_t peers = __match_any_sync(kFull, d);
        const uint32_t before = valid ? s_wcnt[w][d] : 0u;
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (valid && (peers & lt) == 0) s_wcnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread t owns digit t: exclusive prefixes over the warps, the tile's count
    uint32_t cnt = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t c = s_wcnt[ww][t];
        s_wcnt[ww][t] = cnt;
        cnt += c;
    }
    volatile unsigned long long* st = status;
    // withhold (a self-test of the bounded wait): tile 0 never publishes and each
    // word is polled once, so the wait of tile 1 runs out
    if (!(withhold && tile == 0)) st[tile * kRadixBins + t] = (tile == 0 ? kOsPrefix : kOsAggregate) | cnt;
    const int spin_limit = withhold ? 1 : kOsSpinLimit;
    uint32_t total;
    s_dstart[t] = block_exscan(cnt, &total);
    const uint32_t bucket = block_exscan(hist[t], &total);
    // the tile in digit order in shared memory (block_exscan ends with a barrier)
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int e = w * kWarpItems + r * 32 + lane;
        if (e < tile_n) {
            const uint32_t d = os_digit<K>(key[r], val[r], sysd, shift);
            const uint32_t lp = s_dstart[d] + s_wcnt[w][d] + rank[r];
            s_key[lp] = key[r];
            s_val[lp] = val[r];
        }
    }
    // look back: the counts of the earlier tiles, kOsWindow words per round
    // trip, nearest first, up to the first inclusive prefix
    uint32_t excl = 0;
    bool done = tile == 0;
    for (int64_t j = tile - 1; !done; j -= kOsWindow) {
        unsigned long long v[kOsWindow];
#pragma unroll
        for (int q = 0; q < kOsWindow; ++q)
            v[q] = j - q >= 0 ? (unsigned long long)st[(j - q) * kRadixBins + t] : 2ull << 32;
#pragma unroll
        for (int q = 0; q < kOsWindow; ++q) {
            if (!done) {
                unsigned long long x = v[q];
                for (int it = 0; (x >> 32) == 0 && it < spin_limit; ++it) {
                    __nanosleep(32);
                    x = st[(j - q) * kRadixBins + t];
                }
                if ((x >> 32) == 0) {
                    atomicOr(flags, FLAG_SORT);
                    done = true;
                } else {
                    excl += (uint32_t)x;
                    done = (x & kOsPrefix) != 0;
                }
            }
        }
    }
    if (tile > 0) st[tile * kRadixBins + t] = kOsPrefix | (unsigned long long)(excl + cnt);
    s_gstart[t] = bucket + excl;
    __syncthreads();
    for (int j = t; j < tile_n; j += kOsThreads) {
        const K key = s_key[j];
        const uint32_t val = s_val[j];
        const uint32_t d = os_digit<K>(key, val, sysd, shift);
        const int64_t g = (int64_t)s_gstart[d] + (j - (int64_t)s_dstart[d]);
        kout[g] = key;
        vout[g] = val;
    }
}

// ------------------------------------------------------- bbox and keys
__device__ __forceinline__ long long enc(float x)
{
    int i = __float_as_int(x);
    return (long long)(i >= 0 ? i : i ^ 0x7fffffff);
}
__device__ __forceinline__ long long enc(double x)
{
    long long i = __double_as_longlong(x);
    return i >= 0 ? i : i ^ 0x7fffffffffffffffLL;
}
__device__ __forceinline__ void dec(long long e, float* x)
{
    int i = (int)e;
    *x = __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}
__device__ __forceinline__ void dec(long long e, double* x)
{
    *x = __longlong_as_double(e >= 0 ? e : e ^ 0x7fffffffffffffffLL);
}

__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rfloor(float a) { return floorf(a); }
__device__ __forceinline__ double rfloor(double a) { return floor(a); }
__device__ __forceinline__ float rscale2(float a, int e) { return ldexpf(a, e); }
__device__ __forceinline__ double rscale2(double a, int e) { return ldexp(a, e); }

__global__ void k_bbox_init(BBox* bb)
{
    for (int a = 0; a < 3; ++a) {
        bb->lo[a] = LLONG_MAX;
        bb->hi[a] = LLONG_MIN;
    }
}

// One block per system: extrema of the positions [start[s], start[s+1]).
template <typename R>
__global__ void k_bbox_seg(const vec4<R>* __restrict__ pos, const int* __restrict__ start,
                           BBox* bb, int* flags)
{
    const int sgi = blockIdx.x;
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
    long long hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    bool bad = false;
    for (int64_t i = start[sgi] + threadIdx.x; i < start[sgi + 1]; i += blockDim.x) {
        vec4<R> p = pos[i];
        R c[3] = {p.x, p.y, p.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bad |= !isfinite(c[a]);
            long long e = enc(c[a]);
            lo[a] = min(lo[a], e);
            hi[a] = max(hi[a], e);
        }
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, FLAG_NONFINITE);
    __shared__ long long sl[3][32], sh[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(kFull, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(kFull, hi[a], o));
        }
        if (lane == 0) {
            sl[a][w] = lo[a];
            sh[a][w] = hi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        long long l = LLONG_MAX, h = LLONG_MIN;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
            l = min(l, sl[a][ww]);
            h = max(h, sh[a][ww]);
        }
        bb[sgi].lo[a] = l;
        bb[sgi].hi[a] = h;
    }
}

template <typename R>
__global__ void k_bbox(const vec4<R>* __restrict__ pos, int64_t n, BBox* bb, int* flags)
{
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
    long long hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        vec4<R> p = pos[i];
        R c[3] = {p.x, p.y, p.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bad |= !isfinite(c[a]);
            long long e = enc(c[a]);
            lo[a] = min(lo[a], e);
            hi[a] = max(hi[a], e);
        }
    }
    if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, FLAG_NONFINITE);
    // warp, then block extrema: six global atomics per block
    __shared__ long long sl[3][32], sh[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(kFull, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(kFull, hi[a], o));
        }
        if (lane == 0) {
            sl[a][w] = lo[a];
            sh[a][w] = hi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int a = threadIdx.x;
        long long l = LLONG_MAX, h = LLONG_MIN;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
            l = min(l, sl[a][ww]);
            h = max(h, sh[a][ww]);
        }
        atomicMin(&bb->lo[a], l);
        atomicMax(&bb->hi[a], h);
    }
}

// Root cube: origin = minimum corner, side = largest extent (1 if all zero).
template <typename R>
__device__ __forceinline__ void root_cube(const BBox* bb, R mn[3], R* side)
{
    R mx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dec(bb->lo[a], &mn[a]);
        dec(bb->hi[a], &mx[a]);
    }
    R s = rsub(mx[0], mn[0]);
#pragma unroll
    for (int a = 1; a < 3; ++a) {
        R e = rsub(mx[a], mn[a]);
        if (e > s) s = e;
    }
    if (!(s > R(0))) s = R(1);
    *side = s;
}

template <typename R>
__device__ __forceinline__ uint32_t quantise(R x, R mn, R S)
{
    R fl = rfloor(rmul(rsub(x, mn), S));
    if (!(fl > R(0))) return 0u;
    if (fl >= R(2097151)) return 2097151u;
    return (uint32_t)fl;
}

__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

template <typename R>
__global__ void k_morton(const vec4<R>* __restrict__ pos, int64_t n, const BBox* __restrict__ bb,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                         const uint32_t* __restrict__ of_pos)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    R mn[3], side;
    root_cube<R>(of_pos ? bb + of_pos[i] : bb, mn, &side);
    const R S = rdiv(R(2097152), side);
    vec4<R> p = pos[i];
    uint32_t qx = quantise<R>(p.x, mn[0], S);
    uint32_t qy = quantise<R>(p.y, mn[1], S);
    uint32_t qz = quantise<R>(p.z, mn[2], S);
    keys[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    vals[i] = (uint32_t)i;
}

template <typename R>
__global__ void k_gather(const uint32_t* __restrict__ perm, int64_t n,
                         const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ vel,
                         const vec4<R>* __restrict__ u, const vec4<R>* __restrict__ om,
                         const uint32_t* __restrict__ id, vec4<R>* __restrict__ pos2,
                         vec4<R>* __restrict__ vel2, vec4<R>* __restrict__ u2,
                         vec4<R>* __restrict__ om2, uint32_t* __restrict__ id2)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const uint32_t p = perm[s];
    pos2[s] = pos[p];
    vel2[s] = vel[p];
    u2[s] = u[p];
    om2[s] = om[p];
    id2[s] = id[p];
}

// ------------------------------------------------------------ tree build
// Split level of sorted position j: the first level at which particles j-1
// and j fall in different cells (0 for j = 0 and j = n; 22 for equal keys).
__device__ __forceinline__ int split_level(const uint64_t* __restrict__ k, int64_t j, int64_t n,
                                           const uint32_t* __restrict__ of_pos)
{
    if (j <= 0 || j >= n) return 0;
    if (of_pos && of_pos[j] != of_pos[j - 1]) return 0;  // first particle of a system
    uint64_t x = k[j] ^ k[j - 1];
    if (!x) return kMaxLevel + 1;
    return (__clzll((long long)x) - 1) / 3 + 1;
}

// Per particle i: depth d_i of its leaf and the number of cells whose first
// particle is i (levels l_i .. d_i).  The level-L cell holding i has more
// than m particles iff some a + b = m has the a positions i, i-1, ..
// i-a+1 and the b positions i+1 .. i+b all with split level > L.
__global__ void k_levels(const uint64_t* __restrict__ k, int64_t n, int m,
                         uint32_t* __restrict__ cnt, const uint32_t* __restrict__ of_pos)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int right[kMaxLeaf + 1];
    right[0] = 99;
    for (int b = 1; b <= m; ++b) right[b] = min(right[b - 1], split_level(k, i + b, n, of_pos));
    int left = 99;
    int D = min(left, right[m]);
    for (int a = 1; a <= m; ++a) {
        left = min(left, split_level(k, i - a + 1, n, of_pos));
        D = max(D, min(left, right[m - a]));
    }
    const int d = min(D, kMaxLevel);
    const int li = split_level(k, i, n, of_pos);
    cnt[i] = d >= li ? (uint32_t)(d - li + 1) : 0u;
}

// First j in [lo, n) with k[j] >= bound, given k[lo-1] < bound.
__device__ __forceinline__ int64_t gallop_right(const uint64_t* __restrict__ k, int64_t lo,
                                                int64_t n, uint64_t bound)
{
    if (lo >= n || k[lo] >= bound) return lo;
    int64_t step = 1, hi = lo + 1;
    while (hi < n && k[hi] < bound) {
        lo = hi;
        step <<= 1;
        hi = lo + step;
    }
    if (hi > n) hi = n;
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (k[mid] < bound) lo = mid;
        else hi = mid;
    }
    return hi;
}

// First j in [first, hi] with k[j] >= bound, given k[hi] >= bound.
__device__ __forceinline__ int64_t gallop_left(const uint64_t* __restrict__ k, int64_t hi,
                                               uint64_t bound, int64_t first)
{
    int64_t lo = first - 1, step = 1;
    for (;;) {
        int64_t c = hi - step;
        if (c < first) break;
        if (k[c] < bound) {
            lo = c;
            break;
        }
        hi = c;
        step <<= 1;
    }
    while (hi - lo > 1) {
        int64_t mid = lo + ((hi - lo) >> 1);
        if (k[mid] < bound) lo = mid;
        else hi = mid;
    }
    return hi;
}

// Writes the cells whose first particle is i: level L covers the run of
// keys sharing i's level-L prefix; skip = first cell of the particle after
// the run; the deepest of them is i's leaf.  Cube of a level-L cell with
// integer coordinates q: lo = origin + q * (side 2^-L), each op rounded once.
template <typename R>
__global__ void k_emit(const uint64_t* __restrict__ k, int64_t n, const uint32_t* __restrict__ cnt,
                       const uint32_t* __restrict__ off, const BBox* __restrict__ bb, Tree<R> t,
                       int* flags, Segs sg)
{
    // The 32 particles of a warp start between 0 and 22 cells each (most one);
    // their cells are dealt out to the lanes in turn, so that a particle that
    // starts many levels does not hold up the other lanes.
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int c = i < n ? (int)cnt[i] : 0;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    const int excl = incl - c;
    const int total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    if (c > 0 && ((int64_t)off[i] + c > t.cap || (int64_t)off[n] > t.cap)) atomicOr(flags, FLAG_CAPACITY);
    if (__any_sync(kFull, c > 0 && ((int64_t)off[i] + c > t.cap || (int64_t)off[n] > t.cap))) return;
    const int li_own = c > 0 ? split_level(k, i, n, sg.of_pos) : 0;
    const uint64_t key_own = c > 0 ? k[i] : 0ull;
    const int64_t base_own = c > 0 ? (int64_t)off[i] : 0;
    for (int j0 = 0; j0 < total; j0 += 32) {
        const int j = j0 + lane;
        // owner: the last lane whose run of cells starts at or before j
        int o = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(kFull, excl, o + step);
            if (e <= j) o += step;
        }
        const int oc = __shfl_sync(kFull, c, o);
        const int oli = __shfl_sync(kFull, li_own, o);
        const int oex = __shfl_sync(kFull, excl, o);
        const uint64_t key = __shfl_sync(kFull, key_own, o);
        const int64_t base = __shfl_sync(kFull, base_own, o);
        if (j >= total) continue;
        const int64_t ip = i - lane + o;  // the owner's particle
        // the positions of its system: runs and parents never leave them
        const int sys = sg.of_pos ? (int)sg.of_pos[ip] : 0;
        const int64_t sfirst = sg.of_pos ? sg.start[sys] : 0;
        const int64_t send = sg.of_pos ? sg.start[sys + 1] : n;
        const int d = oli + oc - 1;
        const int L = d - (j - oex);  // the owner's cells, deepest first
        const int64_t idx = base + (L - oli);
        R mn[3], side;
        root_cube<R>(bb + sys, mn, &side);
        int64_t pe;
        if (L == 0) {
            pe = send;
        } else {
            const int sh = 3 * (kMaxLevel - L);
            const uint64_t bound = ((key >> sh) + 1ull) << sh;
            pe = gallop_right(k, ip + 1, send, bound);
        }
        const int skip = (int)off[pe];
        const int leaf = (L == d) ? 1 : 0;
        const int single = (leaf && pe - ip == 1) ? 1 : 0;
        t.cell[idx].node = make_int4((int)ip, (int)pe, skip, L | (leaf << 8) | (single << 9));
        int parent;
        if (L == 0) {
            parent = -1;
        } else if (L > oli) {
            parent = (int)idx - 1;
        } else {
            const int sh2 = 3 * (kMaxLevel - (L - 1));
            const uint64_t lowb = (key >> sh2) << sh2;
            const int64_t sp = gallop_left(k, ip, lowb, sfirst);
            parent = (int)off[sp] + (L - 1 - split_level(k, sp, n, sg.of_pos));
        }
        t.parent[idx] = parent;
        t.arrive[idx] = 0;
        const R sL = rscale2(side, -L);
        const uint64_t pre = (L == 0) ? 0ull : (key >> (3 * (kMaxLevel - L)));
        const R qx = (R)compact3(pre >> 2), qy = (R)compact3(pre >> 1), qz = (R)compact3(pre);
        vec4<R> lo;
        lo.x = radd(mn[0], rmul(qx, sL));
        lo.y = radd(mn[1], rmul(qy, sL));
        lo.z = radd(mn[2], rmul(qz, sL));
        lo.w = sL;
        t.lo[idx] = lo;
    }
}

// Atomic add at device scope with acquire-release ordering: the caller's
// earlier writes are visible to whoever acquires a later value of *p, and the
// caller sees the writes released by the additions before its own.
__device__ __forceinline__ int atomic_add_acq_rel(int* p, int v)
{
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
                 : "memory");
    return old;
}

__device__ __forceinline__ float4 ldcg4(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ dvec4 ldcg4(const dvec4* p)
{
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = __ldcg(q), b = __ldcg(q + 1);
    dvec4 r;
    r.x = a.x;
    r.y = a.y;
    r.z = b.x;
    r.w = b.y;
    return r;
}

// Adds the symmetric part of d (x) v and its trace to q (S_xx, S_yy, S_zz,
// S_xy, S_xz, S_yz, m).
template <typename R>
__device__ __forceinline__ void quad_add(R dx, R dy, R dz, R vx, R vy, R vz, R q[7])
{
    q[0] += dx * vx;
    q[1] += dy * vy;
    q[2] += dz * vz;
    q[3] += R(0.5) * (dx * vy + dy * vx);
    q[4] += R(0.5) * (dx * vz + dz * vx);
    q[5] += R(0.5) * (dy * vz + dz * vy);
    q[6] += dx * vx + dy * vy + dz * vz;
}

// Bottom-up aggregation (Eq. magCenter): leaves sum their particles in
// sorted order; the last child to arrive at a parent sums the parent's
// children in octant order.  centre = position sum / count.  Sums are formed
// in A and kept in ssum/smom (for A = R these are the tree's own sum and mom
// arrays); with A wider than R the moment sum and the centre are rounded to R
// once, from the A sums.
// Largest distance from the centre c to a point of the cube [lo, lo + side]
// (side = lo.w; the far corner on each axis): a particle farther than
// rcut + reach from c is at least rcut from the cube.  The traversal's opening
// test reads far2_of(rcut, reach), stored with each cell's moment sum.
template <typename R>
__device__ __forceinline__ R cube_reach(const vec4<R>& c, const vec4<R>& lo)
{
    const R cs[3] = {c.x, c.y, c.z};
    const R ls[3] = {lo.x, lo.y, lo.z};
    R r2 = R(0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const R hi = radd(ls[a], lo.w);
        const R e = fmax(fabs(rsub(cs[a], ls[a])), fabs(rsub(hi, cs[a])));
        r2 = r2 + e * e;
    }
    return sqrt(r2);
}

template <typename R, typename A>
__global__ void k_aggregate(const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ u,
                            int64_t n, const uint32_t* __restrict__ cnt,
                            const uint32_t* __restrict__ off, Tree<R> t, vec4<A>* ssum,
                            vec4<A>* smom, const int* flags_in, int* flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c0 = (int)cnt[i];
    if (c0 == 0) return;
    if (*flags_in & FLAG_CAPACITY) return;
    int c = (int)off[i] + c0 - 1;
    int4 nd = t.cell[c].node;
    vec4<R> p = pos[nd.x], q = u[nd.x];
    A sx = p.x, sy = p.y, sz = p.z, ux = q.x, uy = q.y, uz = q.z;
    for (int s = nd.x + 1; s < nd.y; ++s) {
        p = pos[s];
        q = u[s];
        sx = radd(sx, (A)p.x);
        sy = radd(sy, (A)p.y);
        sz = radd(sz, (A)p.z);
        ux = radd(ux, (A)q.x);
        uy = radd(uy, (A)q.y);
        uz = radd(uz, (A)q.z);
    }
    int guard = 0;
    for (;;) {
        const int cntc = nd.y - nd.x;
        const A rn = (A)cntc;
        vec4<A> sm, mm;
        vec4<R> cc;
        const vec4<R> lo = t.lo[c];
        cc.x = (R)rdiv(sx, rn); cc.y = (R)rdiv(sy, rn); cc.z = (R)rdiv(sz, rn);
        const R far2 = far2_of<R>(t.rcut, cube_reach<R>(cc, lo));
        cc.w = rmul(lo.w, lo.w);  // side^2 for the opening test
        sm.x = sx; sm.y = sy; sm.z = sz; sm.w = A(0);
        mm.x = ux; mm.y = uy; mm.z = uz; mm.w = (A)far2;
        if (t.q1) {
            // S and m about this centre: from the particles of a leaf, else from the
            // children by the shift M = sum_j [M_j + (c_j - c) (x) U_j]
            R q[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
            if (nd.w >> 8) {
                for (int s = nd.x; s < nd.y; ++s) {
                    const vec4<R> p = pos[s], v = u[s];
                    quad_add<R>(p.x - cc.x, p.y - cc.y, p.z - cc.z, v.x, v.y, v.z, q);
                }
            } else {
                for (int ch = c + 1, k = 0; ch < nd.z && k < 8; ch = t.cell[ch].node.z, ++k) {
                    const vec4<R> cj = ldcg4(&t.cell[ch].cen), uj = ldcg4(&t.mom[ch]);
                    const vec4<R> a = ldcg4(&t.q1[ch]), b = ldcg4(&t.q2[ch]);
                    q[0] += a.x; q[1] += a.y; q[2] += a.z; q[3] += a.w;
                    q[4] += b.x; q[5] += b.y; q[6] += b.z;
                    quad_add<R>(cj.x - cc.x, cj.y - cc.y, cj.z - cc.z, uj.x, uj.y, uj.z, q);
                }
            }
            vec4<R> a, b;
            a.x = q[0]; a.y = q[1]; a.z = q[2]; a.w = q[3];
            b.x = q[4]; b.y = q[5]; b.z = q[6]; b.w = R(0);
            t.q1[c] = a;
            t.q2[c] = b;
        }
        ssum[c] = sm;
        smom[c] = mm;
        if (sizeof(A) != sizeof(R)) {
            vec4<R> mr;
            mr.x = (R)ux; mr.y = (R)uy; mr.z = (R)uz; mr.w = far2;
            t.mom[c] = mr;
        }
        t.cell[c].cen = cc;
        const int par = t.parent[c];
        if (par < 0) break;
        // release this cell's sums to the sibling that arrives last, which
        // acquires all of them with the same operation
        const int old = atomic_add_acq_rel(&t.arrive[par], cntc);
        const int4 pn = t.cell[par].node;
        if (old + cntc != pn.y - pn.x) break;
        int ch = par + 1;
        vec4<A> a = ldcg4(&ssum[ch]), b = ldcg4(&smom[ch]);
        sx = a.x; sy = a.y; sz = a.z; ux = b.x; uy = b.y; uz = b.z;
        ch = t.cell[ch].node.z;
        int kids = 1;
        while (ch < pn.z && kids < 8) {
            a = ldcg4(&ssum[ch]);
            b = ldcg4(&smom[ch]);
            sx = radd(sx, a.x);
            sy = radd(sy, a.y);
            sz = radd(sz, a.z);
            ux = radd(ux, b.x);
            uy = radd(uy, b.y);
            uz = radd(uz, b.z);
            ch = t.cell[ch].node.z;
            ++kids;
        }
        if (ch != pn.z || ++guard > kMaxLevel + 1) {
            atomicOr(flags, FLAG_AGGREGATE);
            break;
        }
        c = par;
        nd = pn;
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ================================================================ launchers
std::atomic<int64_t> g_launches{0};

size_t scan_tmp_words(int64_t n)
{
    return (size_t)((n + kScanTile - 1) / kScanTile) + 1;
}

void scan_exclusive(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* tmp, cudaStream_t s)
{
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > 0) k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_top<<<1, kScanThreads, 0, s>>>(tmp, nb, out + n);
    if (nb > 0) k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp, out);
    counted(nb > 0 ? 3 : 1);
}

// The scatter's tile needs more dynamic shared memory than the default limit;
// the limit is raised once per device.
template <typename K>
void os_prepare()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return;
    cudaFuncSetAttribute(k_os_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)os_dyn_smem<K>());
    if (dev >= 0 && dev < 64) done[dev] = true;
}

size_t radix_tmp_words(int64_t n) { return os_tmp_words(n); }

// The passes of a one-sweep LSD sort: digits p * 8 .. p * 8 + 7 of the keys or,
// with sysd, of the system of each element's value.
template <typename K>
bool os_sort(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int64_t n, uint32_t* tmp, int passes,
             int* flags, cudaStream_t s, const uint32_t* sysd, int withhold = 0)
{
    if (n <= 1 || passes < 1) return false;
    if (passes > kOsMaxPasses) passes = kOsMaxPasses;
    if (!sysd && passes * kRadixBits > (int)(8 * sizeof(K))) passes = (int)(8 * sizeof(K)) / kRadixBits;
    const int64_t tiles = (n + kOsThreads * os_items<K>() - 1) / (kOsThreads * os_items<K>());
    uint32_t* hist = tmp;
    unsigned long long* status[2];
    status[0] = reinterpret_cast<unsigned long long*>(tmp + kOsMaxPasses * kRadixBins);
    status[1] = status[0] + kRadixBins * tiles;
    uint32_t* tickets = reinterpret_cast<uint32_t*>(status[1] + kRadixBins * tiles);
    // counts and the first pass's status words start at zero; the second
    // array is cleared tile by tile during the first pass, and so on
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kOsMaxPasses * kRadixBins, s);
    cudaMemsetAsync(status[0], 0, sizeof(unsigned long long) * kRadixBins * tiles, s);
    cudaMemsetAsync(tickets, 0, sizeof(uint32_t) * kOsMaxPasses, s);
    const int64_t hb = (n + kOsThreads - 1) / kOsThreads;
    k_os_hist<K><<<(unsigned)(hb < 1216 ? hb : 1216), kOsThreads, 0, s>>>(k0, v0, sysd, n, passes,
                                                                          hist);
    K* ka = k0;
    uint32_t* va = v0;
    K* kb = k1;
    uint32_t* vb = v1;
    os_prepare<K>();
    for (int p = 0; p < passes; ++p) {
        k_os_scatter<K><<<(unsigned)tiles, kOsThreads, os_dyn_smem<K>(), s>>>(
            ka, va, kb, vb, n, p * kRadixBits, hist + p * kRadixBins, status[p & 1],
            status[(p + 1) & 1], tickets + p, flags, sysd, withhold);
        K* tk = ka; ka = kb; kb = tk;
        uint32_t* tv = va; va = vb; vb = tv;
    }
    counted(1 + passes);
    return (passes & 1) != 0;
}

template <typename K>
bool radix_sort_pairs_passes(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int64_t n, uint32_t* tmp,
                             int passes, int* flags, cudaStream_t s)
{
    return os_sort<K>(k0, v0, k1, v1, n, tmp, passes, flags, s, nullptr);
}
template bool radix_sort_pairs_passes<uint64_t>(uint64_t*, uint32_t*, uint64_t*, uint32_t*, int64_t,
                                                uint32_t*, int, int*, cudaStream_t);
template bool radix_sort_pairs_passes<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*, int64_t,
                                                uint32_t*, int, int*, cudaStream_t);

void radix_sort_pairs(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                      uint32_t* tmp, int* flags, cudaStream_t s)
{
    // eight passes: the sorted data are back in (k0, v0)
    os_sort<uint64_t>(k0, v0, k1, v1, n, tmp, 8, flags, s, nullptr);
}

void radix_sort_wait_selftest(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                              uint32_t* tmp, int* flags, cudaStream_t s)
{
    os_sort<uint64_t>(k0, v0, k1, v1, n, tmp, 1, flags, s, nullptr, 1);
}

void radix_sort_systems(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int64_t n,
                        uint32_t* tmp, Segs sg, int* flags, cudaStream_t s)
{
    if (!sg.of_pos || sg.nseg <= 1 || n <= 1) return;
    // an even number of passes leaves the data in (k0, v0); the value of each
    // element stays its pre-sort position, so its system is of_pos[value]
    int passes = 0;
    for (int b = 0; (1 << b) < sg.nseg; b += kRadixBits) ++passes;
    if (passes & 1) ++passes;
    os_sort<uint64_t>(k0, v0, k1, v1, n, tmp, passes, flags, s, sg.of_pos);
}

template <typename R>
void morton_keys(const vec4<R>* pos, int64_t n, BBox* bb, uint64_t* keys, uint32_t* vals,
                 int* flags, Segs sg, cudaStream_t s)
{
    if (sg.of_pos) {
        k_bbox_seg<R><<<sg.nseg, 256, 0, s>>>(pos, sg.start, bb, flags);
        counted();
    } else {
        k_bbox_init<<<1, 1, 0, s>>>(bb);
        unsigned g = nblk(n, 256);
        if (g > 152u * 4u) g = 152u * 4u;
        k_bbox<R><<<g, 256, 0, s>>>(pos, n, bb, flags);
        counted(2);
    }
    k_morton<R><<<nblk(n, 256), 256, 0, s>>>(pos, n, bb, keys, vals, sg.of_pos);
    counted();
}

template <typename R>
void gather_state(const uint32_t* perm, int64_t n, const vec4<R>* pos, const vec4<R>* vel,
                  const vec4<R>* u, const vec4<R>* om, const uint32_t* id, vec4<R>* pos2,
                  vec4<R>* vel2, vec4<R>* u2, vec4<R>* om2, uint32_t* id2, cudaStream_t s)
{
    k_gather<R><<<nblk(n, 256), 256, 0, s>>>(perm, n, pos, vel, u, om, id, pos2, vel2, u2, om2,
                                              id2);
    counted();
}

template <typename R>
void build_tree(const uint64_t* skeys, int64_t n, int leaf_max, const BBox* bb, Tree<R> t,
                uint32_t* cnt, uint32_t* off, uint32_t* scan_tmp, int* flags, Segs sg,
                cudaStream_t s)
{
    k_levels<<<nblk(n, 128), 128, 0, s>>>(skeys, n, leaf_max, cnt, sg.of_pos);
    scan_exclusive(cnt, off, n, scan_tmp, s);
    k_emit<R><<<nblk(n, 128), 128, 0, s>>>(skeys, n, cnt, off, bb, t, flags, sg);
    counted(2);
}

template <typename R, typename A>
void aggregate_tree(const vec4<R>* pos, const vec4<R>* u, int64_t n, const uint32_t* cnt,
                    const uint32_t* off, Tree<R> t, vec4<A>* ssum, vec4<A>* smom, int* flags,
                    cudaStream_t s)
{
    k_aggregate<R, A><<<nblk(n, 128), 128, 0, s>>>(pos, u, n, cnt, off, t, ssum, smom, flags,
                                                   flags);
    counted();
}

#define FFK_INST(R)                                                                            \
    template void morton_keys<R>(const vec4<R>*, int64_t, BBox*, uint64_t*, uint32_t*, int*,   \
                                 Segs, cudaStream_t);                                          \
    template void gather_state<R>(const uint32_t*, int64_t, const vec4<R>*, const vec4<R>*,     \
                                  const vec4<R>*, const vec4<R>*, const uint32_t*, vec4<R>*,   \
                                  vec4<R>*, vec4<R>*, vec4<R>*, uint32_t*, cudaStream_t);      \
    template void build_tree<R>(const uint64_t*, int64_t, int, const BBox*, Tree<R>, uint32_t*, \
                                uint32_t*, uint32_t*, int*, Segs, cudaStream_t);               \
    template void aggregate_tree<R, R>(const vec4<R>*, const vec4<R>*, int64_t, const uint32_t*, \
                                       const uint32_t*, Tree<R>, vec4<R>*, vec4<R>*, int*,       \
                                       cudaStream_t);
FFK_INST(float)
FFK_INST(double)
#undef FFK_INST
template void aggregate_tree<float, double>(const float4*, const float4*, int64_t, const uint32_t*,
                                            const uint32_t*, Tree<float>, dvec4*, dvec4*, int*,
                                            cudaStream_t);

}  // namespace ffk
