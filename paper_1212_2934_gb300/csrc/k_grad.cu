// Gradient of the Barnes-Hut dipolar energy E = -1/2 sum_m u_m . h_m with
// the opening decisions frozen (Sec. 3.2 traversal, Sec. 5 energy).
//
// With phi(r; a, b) = a . T(r) b and h_m = sum over m's sources s of
// T(rho_m - x_s) w_s (cells: centre and moment sum; exact pairs: particles):
//   dE/du_k   = -1/2 [ h_k + ds sum over (m, s), k in s, of T(rho_m - x_s) u_m ]
//   dE/drho_k = -1/2 [ f_k - ds sum over (m, s), k in s, of
//                      grad phi(rho_m - x_s; w_s, u_m) / n_s ]
// h and f are the dipolar field and force of the same traversal (ds
// included).  The reverse sums are formed without atomics.  The counting walk
// writes every particle's sources (in depth-first order) to an entry pool; one
// block per task of 32 consecutive particles gathers its 32 lists into records
// (source, task, lane mask), one per source some lane takes; the records
// (about a tenth as many as the (source, target) entries) are packed in task
// order and sorted stably by source, so each source's entries, expanded lane
// by lane, come out in target order.  Each source's entries are summed in a
// fixed order (pieces of at most 1024 entries one warp each, the pieces added
// in FP64), and each leaf adds the sums of its ancestor cells for its
// particles.  The vector-Jacobian product keeps per-target entries: its walk
// also sums target-side terms lane by lane.
#include "dipole.cuh"
#include "ffk.cuh"

namespace ffk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGradThreads = 256;
// record building by hash table (k_hash_records): block size, table slots (32 KB
// of keys and masks), most sources a task may have there; a task with more is
// marked kHashOverflow and merged by k_merge_records instead
constexpr int kHashThreads = 256;
constexpr int kHashSlots = 4096;
constexpr int kHashLimit = 3072;
constexpr uint32_t kHashOverflow = 0xffffffffu;

__global__ void k_entry_counts(const int4* __restrict__ counts, int64_t n,
                               uint32_t* __restrict__ out, unsigned long long* total)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) {
        const int4 c = counts[i];
        v = (unsigned long long)(unsigned)c.x + (unsigned long long)(unsigned)c.y;
        out[i] = (uint32_t)v;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Work items: every source's entry list is cut into pieces of at most
// kGradItemEntries entries, so no warp is left alone with a top-level cell that
// most particles accept.
__global__ void k_item_counts(const uint32_t* __restrict__ beg, const uint32_t* __restrict__ end,
                              int64_t nsrc, uint32_t* __restrict__ items)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsrc) return;
    items[s] = (uint32_t)((end[s] - beg[s] + kGradItemEntries - 1) / kGradItemEntries);
}

// The source of every work item: thread s writes item_off[s] .. item_off[s + 1].
__global__ void k_item_sources(const uint32_t* __restrict__ item_off, int64_t nsrc,
                               uint32_t* __restrict__ item_src)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsrc) return;
    for (uint32_t it = item_off[s]; it < item_off[s + 1]; ++it) item_src[it] = (uint32_t)s;
}

// ------------------------------------------------------- source records
// One warp per task of 32 particles: the lanes' source lists (each rising) are
// merged; each step takes the smallest head, writes it once with the mask of
// the lanes holding it, and advances those lanes.  A lane reads its list four
// sources at a time, following the chunk links.
__global__ void __launch_bounds__(kGradThreads) k_merge_records(
    const uint32_t* __restrict__ cnt, int64_t n, EntryPool pool, const uint32_t* __restrict__ base,
    uint32_t* __restrict__ rkeys, uint32_t* __restrict__ rmask, uint32_t* __restrict__ tcount,
    int* flags)
{
    const int64_t task = ((int64_t)blockIdx.x * kGradThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t ntask = (n + 31) / 32;
    if (task >= ntask || tcount[task] != kHashOverflow) return;
    const int64_t k = task * 32 + lane;
    const uint32_t c = k < n ? cnt[k] : 0u;
    constexpr uint32_t kNone = 0xffffffffu;
    uint32_t ck = (uint32_t)k, pos = 0, head = kNone;
    uint4 buf = make_uint4(0u, 0u, 0u, 0u);
    if (c > 0u) {
        buf = *reinterpret_cast<const uint4*>(pool.keys + (size_t)ck * kPoolChunk);
        head = buf.x;
    }
    const uint32_t w0 = base[task * 32];
    const uint32_t wend = base[min(task * 32 + 32, n)];
    uint32_t w = w0;
    for (;;) {
        const uint32_t key = __reduce_min_sync(kFull, head);
        if (key == kNone) break;
        const bool mine = head == key;
        const uint32_t m = __ballot_sync(kFull, mine);
        if (lane == 0 && w < wend) {
            rkeys[w] = key;
            rmask[w] = m;
        }
        ++w;
        if (mine) {
            ++pos;
            if (pos == c) {
                head = kNone;
            } else {
                const uint32_t o = pos & (uint32_t)(kPoolChunk - 1);
                if (o == 0u) {
                    ck = pool.link[ck];
                    if (ck >= pool.cap) {  // a pool that ran out: the caller redoes the walk
                        atomicOr(flags, FLAG_TRAVERSE);
                        head = kNone;
                        continue;
                    }
                }
                if ((o & 3u) == 0u)
                    buf = *reinterpret_cast<const uint4*>(pool.keys + (size_t)ck * kPoolChunk + o);
                const uint32_t q = o & 3u;
                head = q == 0u ? buf.x : q == 1u ? buf.y : q == 2u ? buf.z : buf.w;
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
        tcount[task] = w - w0;
        if (w > wend) atomicOr(flags, FLAG_TRAVERSE);
    }
}

// Records by a hash table in shared memory, one block per task: the 32 source
// lists are read chunk by chunk (a warp reads 128 sources with one 16-byte load
// per lane) and every source is entered with its lane's bit; the table then
// holds each source of the task once with the mask of the lanes that have it,
// and is written out.  The records of a task come out in no particular order
// (each source occurs once in a task, so after the stable sort by source every
// source's records are in task order all the same).  A task with more than
// kHashLimit sources is left to the warp merge (tcount = kHashOverflow).
__device__ __forceinline__ bool seen(const uint32_t& flag)
{
    return *reinterpret_cast<const volatile uint32_t*>(&flag) != 0u;
}

__global__ void __launch_bounds__(kHashThreads) k_hash_records(
    const uint32_t* __restrict__ cnt, int64_t n, EntryPool pool, const uint32_t* __restrict__ base,
    uint32_t* __restrict__ rkeys, uint32_t* __restrict__ rmask, uint32_t* __restrict__ tcount)
{
    constexpr uint32_t kEmpty = 0xffffffffu;
    __shared__ uint32_t hk[kHashSlots];
    __shared__ uint32_t hm[kHashSlots];
    __shared__ uint32_t used, over, wout;
    const int64_t task = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int i = t; i < kHashSlots; i += kHashThreads) {
        hk[i] = kEmpty;
        hm[i] = 0u;
    }
    if (t == 0) {
        used = 0u;
        over = 0u;
        wout = 0u;
    }
    __syncthreads();
    for (int j = w; j < 32; j += kHashThreads / 32) {
        const int64_t k = task * 32 + j;
        const uint32_t c = k < n ? cnt[k] : 0u;
        const uint32_t bit = 1u << j;
        uint32_t ck = (uint32_t)k;
        for (uint32_t e0 = 0; e0 < c; e0 += (uint32_t)kPoolChunk) {
            if (e0 > 0u) {
                ck = pool.link[ck];
                if (ck >= pool.cap) {  // a pool that ran out: the caller redoes the walk
                    over = 1u;
                    break;
                }
            }
            if (seen(over)) break;
            const uint32_t e = e0 + 4u * (uint32_t)lane;
            if (e >= c) continue;
            const uint4 g = *reinterpret_cast<const uint4*>(pool.keys + (size_t)ck * kPoolChunk +
                                                            4u * (uint32_t)lane);
            const uint32_t key4[4] = {g.x, g.y, g.z, g.w};
            uint32_t fresh = 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (e + (uint32_t)q >= c) break;
                const uint32_t key = key4[q];
                uint32_t h = (key * 2654435761u) >> (32 - 12);  // 12 = log2(kHashSlots)
                for (int probe = 0; probe < kHashSlots; ++probe) {
                    const uint32_t prev = atomicCAS(&hk[h], kEmpty, key);
                    if (prev == kEmpty || prev == key) {
                        atomicOr(&hm[h], bit);
                        fresh += prev == kEmpty ? 1u : 0u;
                        break;
                    }
                    h = (h + 1u) & (uint32_t)(kHashSlots - 1);
                }
            }
            // the new sources, counted once per group of lanes that arrive here
            // together (at most 8 x 128 beyond the limit before every warp sees
            // `over`: the table never fills)
            const unsigned am = __activemask();
            const uint32_t tot = __reduce_add_sync(am, fresh);
            if (lane == __ffs(am) - 1 && tot != 0u &&
                atomicAdd(&used, tot) + tot > (uint32_t)kHashLimit)
                over = 1u;
        }
    }
    __syncthreads();
    if (over) {
        if (t == 0) tcount[task] = kHashOverflow;
        return;
    }
    const uint32_t w0 = base[task * 32];
    for (int i = t; i < kHashSlots; i += kHashThreads) {
        const uint32_t key = hk[i];
        if (key != kEmpty) {
            const uint32_t r = atomicAdd(&wout, 1u);
            rkeys[w0 + r] = key;
            rmask[w0 + r] = hm[i];
        }
    }
    __syncthreads();
    if (t == 0) tcount[task] = wout;
}

// The source at each place of the depth-first order of cells and particles.
template <typename R>
__global__ void k_source_map(Tree<R> t, int64_t ncells, uint32_t* __restrict__ src_of)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int4 nd = t.cell[c].node;
    src_of[c + nd.x] = (uint32_t)c;
    if ((nd.w >> 8) != 0)
        for (int p = nd.x; p < nd.y; ++p) src_of[c + 1 + p] = (uint32_t)(ncells + p);
}

// One block per task: its records, packed in task order.
__global__ void k_pack_records(const uint32_t* __restrict__ tcount,
                               const uint32_t* __restrict__ toff, int64_t ntask,
                               const uint32_t* __restrict__ base,
                               const uint32_t* __restrict__ rkeys,
                               const uint32_t* __restrict__ rmask, uint32_t* __restrict__ ckey,
                               uint32_t* __restrict__ cidx, uint2* __restrict__ crec)
{
    for (int64_t task = blockIdx.x; task < ntask; task += gridDim.x) {
        const uint32_t cnt = tcount[task], dst = toff[task], src = base[32 * task];
        for (uint32_t r = threadIdx.x; r < cnt; r += blockDim.x) {
            ckey[dst + r] = rkeys[src + r];
            cidx[dst + r] = dst + r;
            crec[dst + r] = make_uint2((uint32_t)task, rmask[src + r]);
        }
    }
}

// The sorted records in one pass: srec[i] = crec[sidx[i]], recE[i] = the
// entries (set mask bits) of the records before i, and per source s = src_of[key]
// its first record rbeg[s] and entry range [beg[s], end[s]) (keys outside
// 0 .. nsrc - 1 can only come from a walk that raised its flag; skipped).  Tiles
// of kRsTile records take tickets in the order they start; a tile publishes its
// own entry count, then adds up the counts of the tiles before it, back to the
// first whose running total is out (the status words: a flag in the high half,
// the count in the low half), and publishes its running total.  A wait on an
// earlier tile is bounded: when it runs out, FLAG_SORT is raised.
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;
constexpr unsigned long long kRsAggregate = 1ull << 32;  // this tile alone
constexpr unsigned long long kRsPrefix = 2ull << 32;     // this tile and all before it
constexpr int kRsSpinLimit = 1 << 22;

__global__ void __launch_bounds__(kRsThreads) k_record_scan(
    const uint32_t* __restrict__ skey, const uint32_t* __restrict__ sidx, int64_t nrec,
    const uint2* __restrict__ crec, const uint32_t* __restrict__ src_of, int64_t nsrc,
    uint2* __restrict__ srec, uint32_t* __restrict__ recE, uint32_t* __restrict__ rbeg,
    uint32_t* __restrict__ beg, uint32_t* __restrict__ end, unsigned long long* status,
    uint32_t* ticket, int* flags, int withhold)
{
    __shared__ uint32_t s_tile, s_excl;
    __shared__ uint32_t s_warp[kRsThreads / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    // warp w takes records tile * kRsTile + 256 w + [0, 256), a row of 32
    // consecutive ones per step (lane l: 32 q + l); `incl` the running
    // inclusive count of the warp's records up to this lane's in row q
    const int64_t wbase = tile * kRsTile + (int64_t)w * (32 * kRsItems);
    uint32_t cnt[kRsItems], incl[kRsItems];
    uint32_t run = 0;
    // every gather in flight at once, then the row scans
    uint32_t ix[kRsItems];
#pragma unroll
    for (int q = 0; q < kRsItems; ++q) {
        const int64_t i = wbase + 32 * q + lane;
        ix[q] = i < nrec ? sidx[i] : 0xffffffffu;
    }
#pragma unroll
    for (int q = 0; q < kRsItems; ++q) {
        cnt[q] = 0u;
        if (ix[q] != 0xffffffffu) {
            const uint2 r = crec[ix[q]];
            srec[wbase + 32 * q + lane] = r;
            cnt[q] = (uint32_t)__popc(r.y);
        }
    }
#pragma unroll
    for (int q = 0; q < kRsItems; ++q) {
        const uint32_t c = cnt[q];
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        incl[q] = run + x;
        run += __shfl_sync(kFull, x, 31);
    }
    if (lane == 0) s_warp[w] = run;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kRsThreads / 32; ++k) {
        const uint32_t v = s_warp[k];
        if (k < w) before += v;
        total += v;
    }
    if (w == 0) {
        // the first warp looks back 32 tiles a round trip: lane k reads tile
        // j0 - k; once every tile up to the nearest running total has published,
        // their counts are added (a full window of tile counts moves it back)
        volatile unsigned long long* st = status;
        // withhold (a self-test of the bounded wait): tile 0 never publishes and
        // each window is read once, so the wait of tile 1 runs out
        if (lane == 0 && !(withhold && tile == 0))
            st[tile] = (tile == 0 ? kRsPrefix : kRsAggregate) | total;
        const int spin_limit = withhold ? 1 : kRsSpinLimit;
        uint32_t excl = 0;
        int64_t j0 = tile - 1;
        for (int spins = 0; j0 >= 0;) {
            const int64_t j = j0 - lane;
            unsigned long long v = kRsPrefix;  // before the first tile: a total of 0
            if (j >= 0) v = st[j];
            const uint32_t pub = __ballot_sync(kFull, (v >> 32) != 0);
            const uint32_t pre = __ballot_sync(kFull, (v & kRsPrefix) != 0);
            const uint32_t upto = pre != 0u ? (2u << (__ffs(pre) - 1)) - 1u : kFull;
            if ((pub & upto) == upto) {
                excl += warp_sum((upto >> lane) & 1u ? (uint32_t)v : 0u);
                if (pre != 0u) break;
                j0 -= 32;
                continue;
            }
            if (++spins >= spin_limit) {
                if (lane == 0) atomicOr(flags, FLAG_SORT);
                break;
            }
            __nanosleep(32);
        }
        if (lane == 0) {
            if (tile > 0) st[tile] = kRsPrefix | (unsigned long long)(excl + total);
            s_excl = excl;
        }
    }
    __syncthreads();
    const uint32_t E0 = s_excl + before;
#pragma unroll
    for (int q = 0; q < kRsItems; ++q) {
        const int64_t i = wbase + 32 * q + lane;
        if (i < nrec) {
            const uint32_t E = E0 + incl[q] - cnt[q];
            recE[i] = E;
            const uint32_t kk = skey[i];
            if ((int64_t)kk < nsrc) {
                const uint32_t src = src_of[kk];
                if (i == 0 || skey[i - 1] != kk) {
                    rbeg[src] = (uint32_t)i;
                    beg[src] = E;
                }
                if (i == nrec - 1 || skey[i + 1] != kk) end[src] = E + cnt[q];
            }
            if (i == nrec - 1) recE[nrec] = E + cnt[q];
        }
    }
}

// Position of the set bit of m that has j set bits below it (m has more than j).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t j)
{
    uint32_t p = 0;
#pragma unroll
    for (uint32_t h = 16; h > 0; h >>= 1) {
        const uint32_t c = (uint32_t)__popc(m & ((1u << h) - 1u));
        if (j >= c) {
            j -= c;
            m >>= h;
            p += h;
        }
    }
    return p;
}

// One warp per item: the terms of its entries summed in single precision (lane
// j takes entries c0 + j for c0 = the item's first entry + 32 q, q = 0, 1, ..),
// then across the warp, written as six FP64 partials.  The entries come from
// the sorted records: those overlapping a group of 32 entries are at most 32
// consecutive ones (each holds at least one entry); lane l reads record r + l,
// the lanes whose record starts inside the group mark its offset, lane j's
// record is the last marked one at or before j, and its particle is that
// record's set lane of the right rank.
// (blocks of 4 warps: a block's warps wait less for its longest item; ten such
// blocks an SM in single precision, where the terms fit 48 registers)
constexpr int kItemThreads = 128;
template <typename R>
constexpr int item_min_blocks()
{
    return sizeof(R) == 8 ? 1 : 10;
}

template <typename R, bool VJP>
__global__ void __launch_bounds__(kItemThreads, item_min_blocks<R>()) k_item_sums_rec(
    const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ u,
    const vec4<R>* __restrict__ abar, const vec4<R>* __restrict__ bbar, R ds, Tree<R> t,
    int64_t ncells, int64_t nsrc, const uint2* __restrict__ srec, const uint32_t* __restrict__ recE,
    int64_t nrec, const uint32_t* __restrict__ rbeg, const uint32_t* __restrict__ beg,
    const uint32_t* __restrict__ end, const uint32_t* __restrict__ item_off,
    const uint32_t* __restrict__ item_src, double* __restrict__ part)
{
    const int64_t it = ((int64_t)blockIdx.x * kItemThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (it >= (int64_t)item_off[nsrc]) return;
    const int64_t s = item_src[it];  // the source owning this item
    vec4<R> x, w;
    if (s < ncells) {
        x = t.cell[s].cen;
        w = t.mom[s];
    } else {
        x = pos[s - ncells];
        w = u[s - ncells];
    }
    const uint32_t bs = beg[s];
    const uint32_t b = bs + (uint32_t)(it - item_off[s]) * (uint32_t)kGradItemEntries;
    const uint32_t e = min(end[s], b + (uint32_t)kGradItemEntries);
    const uint32_t np = (uint32_t)(nsrc - ncells);
    // the record holding entry b: the last r with recE[r] <= b, among the
    // source's first b - bs + 1 records
    uint32_t lo = rbeg[s];
    uint32_t hi = (uint32_t)min(nrec, (int64_t)lo + (int64_t)(b - bs) + 1);
    while (hi - lo > 1u) {
        const uint32_t mid = lo + (hi - lo) / 2u;
        if (recE[mid] <= b) lo = mid;
        else hi = mid;
    }
    uint32_t r = lo;
    const uint32_t le = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;  // lanes 0 .. lane
    R gx = 0, gy = 0, gz = 0, qx = 0, qy = 0, qz = 0;
    for (uint32_t c0 = b; c0 < e; c0 += 32u) {
        const uint32_t rr = r + (uint32_t)lane;
        const bool have = (int64_t)rr < nrec;
        const uint32_t E = have ? recE[rr] : 0xffffffffu;
        const uint2 rec = have ? srec[rr] : make_uint2(0u, 0u);
        const uint32_t d = E - c0;  // where record rr starts in the group
        const uint32_t mark = lane == 0 ? 1u : (have && d < 32u ? 1u << d : 0u);
        const uint32_t starts = __reduce_or_sync(kFull, mark);
        const int q = __popc(starts & le) - 1;
        const uint32_t Eq = __shfl_sync(kFull, E, q);
        const uint32_t mq = __shfl_sync(kFull, rec.y, q);
        const uint32_t tq = __shfl_sync(kFull, rec.x, q);
        const uint32_t k = c0 + (uint32_t)lane;
        if (k < e) {
            const uint32_t m = tq * 32u + nth_set_bit(mq, k - Eq);
            if (m < np) {
                const vec4<R> xm = pos[m], um = u[m];
                const R rx = xm.x - x.x, ry = xm.y - x.y, rz = xm.z - x.z;
                const R r2 = rx * rx + ry * ry + rz * rz;
                if (!VJP) {
                    // T(r) u_m (field of u_m) and grad phi(r; w_s, u_m) (force on w_s)
                    if (r2 > R(0))
                        dipole<R>(rx, ry, rz, r2, w.x, w.y, w.z, um.x, um.y, um.z, gx, gy, gz,
                                  qx, qy, qz);
                } else if (r2 > R(0)) {
                    const vec4<R> am = abar[m], bm = bbar[m];
                    const PairGeo<R> g = pair_geo<R>(rx, ry, rz, r2);
                    // dL/dw_s: T(r) abar_m + grad phi(r; bbar_m, u_m)
                    t_apply_add<R>(g, am.x, am.y, am.z, R(1), gx, gy, gz);
                    grad_phi_add<R>(g, bm.x, bm.y, bm.z, um.x, um.y, um.z, R(1), gx, gy, gz);
                    // dL/dx_s: -(grad phi(r; abar_m, w_s) + H phi(r; u_m, w_s) bbar_m)
                    grad_phi_add<R>(g, am.x, am.y, am.z, w.x, w.y, w.z, R(-1), qx, qy, qz);
                    hess_phi_add<R>(g, um.x, um.y, um.z, w.x, w.y, w.z, bm.x, bm.y, bm.z, R(-1),
                                    qx, qy, qz);
                }
            }
        }
        // the record holding entry c0 + 32: the group's last record, or the next
        const int ql = __popc(starts) - 1;
        const uint32_t El = __shfl_sync(kFull, E, ql);
        const uint32_t ml = __shfl_sync(kFull, rec.y, ql);
        r += (uint32_t)ql + (El + (uint32_t)__popc(ml) == c0 + 32u ? 1u : 0u);
    }
    gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz);
    qx = warp_sum(qx); qy = warp_sum(qy); qz = warp_sum(qz);
    if (lane == 0) {
        double* o = part + 6 * it;
        const double sc = VJP ? (double)ds : 1.0;
        o[0] = (double)gx * sc; o[1] = (double)gy * sc; o[2] = (double)gz * sc;
        o[3] = (double)qx * sc; o[4] = (double)qy * sc; o[5] = (double)qz * sc;
    }
}

// Each source's items' partials added in item order in FP64, starting from
// zero.  Lane l of a warp owns source 32 w + l and adds up a short list itself;
// a long one (a cell that a large part of the particles accept has up to
// n / 1024 items) is added by six lanes of the warp, one such source after
// another, each lane one of the six sums in item order with its loads issued
// ahead (the one-by-one sums, without one lane waiting on the loads of every
// item in turn, and with no FP64 addition repeated: FP64 is scarce on this
// part).  A cell's position terms are then divided by its particle count (its
// centre is their mean).  FP64 division is a long instruction sequence here,
// and most sources (particles, one-particle leaves) hold one particle (x / 1 is
// x): the quotients a warp does need are gathered, ten sources (30 quotients)
// to one pass of the division over the warp's lanes, and handed back.
constexpr uint32_t kReduceShort = 4;

template <typename R>
__global__ void __launch_bounds__(kGradThreads) k_item_reduce(
    Tree<R> t, int64_t ncells, int64_t nsrc, const uint32_t* __restrict__ item_off,
    const double* __restrict__ part, double* __restrict__ G, double* __restrict__ Q)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool have = s < nsrc;
    double g[3] = {0.0, 0.0, 0.0}, q[3] = {0.0, 0.0, 0.0};
    int ns = 1;
    uint32_t i0 = 0, i1 = 0;
    if (have) {
        i0 = item_off[s];
        i1 = item_off[s + 1];
        if (s < ncells) {
            const int4 nd = t.cell[s].node;
            ns = nd.y - nd.x;
        }
    }
    const bool longer = i1 - i0 > kReduceShort;
    if (!longer) {
        for (uint32_t it = i0; it < i1; ++it) {
            const double* o = part + 6 * (int64_t)it;
            g[0] += o[0]; g[1] += o[1]; g[2] += o[2];
            q[0] += o[3]; q[1] += o[4]; q[2] += o[5];
        }
    }
    for (uint32_t lm = __ballot_sync(kFull, longer); lm != 0u; lm &= lm - 1u) {
        const int l = __ffs(lm) - 1;
        const uint32_t a = __shfl_sync(kFull, i0, l), b = __shfl_sync(kFull, i1, l);
        double x = 0.0;
        if (lane < 6) {
            // lane e adds up component e, loads issued eight items ahead
            const double* o = part + 6 * (int64_t)a + lane;
            const uint32_t m = b - a;
            uint32_t j = 0;
            for (; j + 8u <= m; j += 8u) {
                double v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = o[6 * (int64_t)(j + k)];
#pragma unroll
                for (int k = 0; k < 8; ++k) x += v[k];
            }
            for (; j < m; ++j) x += o[6 * (int64_t)j];
        }
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const double y = __shfl_sync(kFull, x, e);
            if (lane == l) {
                if (e < 3) g[e] = y;
                else q[e - 3] = y;
            }
        }
    }
    double qo[3] = {q[0], q[1], q[2]};
    // lane 3 r + c (r < 10) divides component c of the pass's r-th source
    const int r = lane / 3, c = lane - 3 * r;
    const uint32_t below = (1u << lane) - 1u;
    for (uint32_t m = __ballot_sync(kFull, ns != 1); m != 0u;) {
        const int cnt = min(__popc(m), 10);
        const int from = r < cnt ? (int)nth_set_bit(m, (uint32_t)r) : lane;
        const double n0 = __shfl_sync(kFull, q[0], from);
        const double n1 = __shfl_sync(kFull, q[1], from);
        const double n2 = __shfl_sync(kFull, q[2], from);
        const int d = __shfl_sync(kFull, ns, from);
        // every lane divides (idle lanes by their own count, results unused)
        const double quo = (c == 0 ? n0 : c == 1 ? n1 : n2) / (double)d;
        const int k = __popc(m & below);  // this lane's rank in the pass
        const bool mine = ((m >> lane) & 1u) != 0u && k < cnt;
        const int at = mine ? 3 * k : 0;
        const double a0 = __shfl_sync(kFull, quo, at);
        const double a1 = __shfl_sync(kFull, quo, at + 1);
        const double a2 = __shfl_sync(kFull, quo, at + 2);
        if (mine) {
            qo[0] = a0; qo[1] = a1; qo[2] = a2;
        }
        for (int j = 0; j < cnt; ++j) m &= m - 1u;
    }
    if (!have) return;
    for (int a = 0; a < 3; ++a) {
        G[3 * s + a] = g[a];
        Q[3 * s + a] = qo[a];
    }
}

// One thread per cell; a leaf adds up its ancestors' source sums for each of
// its particles and adds the target-side terms.
template <typename R>
__global__ void k_vjp_finish(Tree<R> t, int64_t ncells, int64_t n, const double* __restrict__ G,
                             const double* __restrict__ Q, const vec4<R>* __restrict__ dxt,
                             const vec4<R>* __restrict__ dut, vec4<R>* __restrict__ dx,
                             vec4<R>* __restrict__ du)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int4 nd = t.cell[c].node;
    if ((nd.w >> 8) == 0) return;
    double dg[3] = {0.0, 0.0, 0.0}, dq[3] = {0.0, 0.0, 0.0};
    int a = (int)c;
    for (int level = 0; a >= 0 && level <= kMaxLevel; ++level) {
        for (int d = 0; d < 3; ++d) {
            dg[d] += G[3 * (int64_t)a + d];
            dq[d] += Q[3 * (int64_t)a + d];
        }
        a = t.parent[a];
    }
    for (int p = nd.x; p < nd.y; ++p) {
        const double* gs = G + 3 * (ncells + p);
        const double* qs = Q + 3 * (ncells + p);
        const vec4<R> xt = dxt[p], ut = dut[p];
        vec4<R> ox = dx[p], ou = du[p];
        ox.x = (R)((double)ox.x + (double)xt.x + dq[0] + qs[0]);
        ox.y = (R)((double)ox.y + (double)xt.y + dq[1] + qs[1]);
        ox.z = (R)((double)ox.z + (double)xt.z + dq[2] + qs[2]);
        ou.x = (R)((double)ou.x + (double)ut.x + dg[0] + gs[0]);
        ou.y = (R)((double)ou.y + (double)ut.y + dg[1] + gs[1]);
        ou.z = (R)((double)ou.z + (double)ut.z + dg[2] + gs[2]);
        dx[p] = ox;
        du[p] = ou;
    }
}

template <typename R>
__global__ void k_scatter_records(const uint32_t* __restrict__ perm, int64_t n,
                                  const vec4<R>* __restrict__ in, vec4<R>* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = in[i];
}

// per-block FP64 sums of the z components, then one block adds them in order
template <typename R>
__global__ void k_sum_z_blocks(const vec4<R>* __restrict__ v, int64_t n, double* __restrict__ tmp)
{
    __shared__ double sh[kGradThreads / 32];
    const int64_t i = (int64_t)blockIdx.x * kGradThreads + threadIdx.x;
    double x = i < n ? (double)v[i].z : 0.0;
    x = warp_sum(x);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kGradThreads / 32; ++w) s += sh[w];
        tmp[blockIdx.x] = s;
    }
}

__global__ void k_sum_final(const double* __restrict__ tmp, int64_t nb, double* out)
{
    __shared__ double sh[kGradThreads];
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nb; b += kGradThreads) s += tmp[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kGradThreads; ++k) t += sh[k];
        *out = t;
    }
}

// One thread per cell; a leaf adds up its ancestors' sums and finishes the
// gradient of each of its particles.
template <typename R>
__global__ void k_grad_finish(Tree<R> t, int64_t ncells, int64_t n, const double* __restrict__ G,
                              const double* __restrict__ Q, const vec4<R>* __restrict__ h,
                              const vec4<R>* __restrict__ f, R ds, vec4<R>* __restrict__ gp,
                              vec4<R>* __restrict__ gu)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int4 nd = t.cell[c].node;
    if ((nd.w >> 8) == 0) return;
    double dg[3] = {0.0, 0.0, 0.0}, dq[3] = {0.0, 0.0, 0.0};
    int a = (int)c;
    for (int level = 0; a >= 0 && level <= kMaxLevel; ++level) {
        for (int d = 0; d < 3; ++d) {
            dg[d] += G[3 * (int64_t)a + d];
            dq[d] += Q[3 * (int64_t)a + d];
        }
        a = t.parent[a];
    }
    const double sc = (double)ds;
    for (int p = nd.x; p < nd.y; ++p) {
        const double* gs = G + 3 * (ncells + p);
        const double* qs = Q + 3 * (ncells + p);
        const vec4<R> hp = h[p], fp = f[p];
        vec4<R> ou, op;
        ou.x = (R)(-0.5 * ((double)hp.x + sc * (dg[0] + gs[0])));
        ou.y = (R)(-0.5 * ((double)hp.y + sc * (dg[1] + gs[1])));
        ou.z = (R)(-0.5 * ((double)hp.z + sc * (dg[2] + gs[2])));
        ou.w = R(0);
        op.x = (R)(-0.5 * ((double)fp.x - sc * (dq[0] + qs[0])));
        op.y = (R)(-0.5 * ((double)fp.y - sc * (dq[1] + qs[1])));
        op.z = (R)(-0.5 * ((double)fp.z - sc * (dq[2] + qs[2])));
        op.w = R(0);
        gu[p] = ou;
        gp[p] = op;
    }
}

template <typename R>
__global__ void k_grad_from_field(const vec4<R>* __restrict__ h, const vec4<R>* __restrict__ f,
                                  int64_t n, vec4<R>* __restrict__ gp, vec4<R>* __restrict__ gu)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vec4<R> a = h[i], b = f[i];
    a.x = -a.x; a.y = -a.y; a.z = -a.z;
    b.x = -b.x; b.y = -b.y; b.z = -b.z;
    gu[i] = a;
    gp[i] = b;
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void grad_entry_counts(const int4* counts, int64_t n, uint32_t* out, unsigned long long* total64,
                       cudaStream_t s)
{
    if (n <= 0) return;
    k_entry_counts<<<blocks(n, kGradThreads), kGradThreads, 0, s>>>(counts, n, out, total64);
    counted();
}

void grad_pack_records(const uint32_t* tcount, const uint32_t* toff, int64_t ntask,
                       const uint32_t* base, const uint32_t* rkeys, const uint32_t* rmask,
                       uint32_t* ckey, uint32_t* cidx, uint2* crec, cudaStream_t s)
{
    if (ntask <= 0) return;
    const int64_t g = ntask < (1 << 20) ? ntask : (1 << 20);
    k_pack_records<<<(unsigned)g, kGradThreads, 0, s>>>(tcount, toff, ntask, base, rkeys, rmask,
                                                        ckey, cidx, crec);
    counted();
}

void grad_merge_records(const uint32_t* cnt, int64_t n, EntryPool pool, const uint32_t* base,
                        uint32_t* rkeys, uint32_t* rmask, uint32_t* tcount, int* flags,
                        cudaStream_t s)
{
    if (n <= 0) return;
    const int64_t ntask = (n + 31) / 32;
    k_hash_records<<<(unsigned)ntask, kHashThreads, 0, s>>>(cnt, n, pool, base, rkeys, rmask,
                                                           tcount);
    k_merge_records<<<blocks(ntask * 32, kGradThreads), kGradThreads, 0, s>>>(
        cnt, n, pool, base, rkeys, rmask, tcount, flags);
    counted(2);
}

template <typename R>
void grad_source_map(Tree<R> t, int64_t ncells, uint32_t* src_of, cudaStream_t s)
{
    if (ncells <= 0) return;
    k_source_map<R><<<blocks(ncells, kGradThreads), kGradThreads, 0, s>>>(t, ncells, src_of);
    counted();
}

size_t record_scan_words(int64_t nrec)
{
    return (size_t)((nrec + kRsTile - 1) / kRsTile) + 1;
}

namespace {

void record_scan(const uint32_t* skey, const uint32_t* sidx, int64_t nrec, const uint2* crec,
                 const uint32_t* src_of, int64_t nsrc, uint2* srec, uint32_t* recE,
                 unsigned long long* scan_words, uint32_t* rbeg, uint32_t* beg, uint32_t* end,
                 int* flags, int withhold, cudaStream_t s)
{
    cudaMemsetAsync(beg, 0, sizeof(uint32_t) * nsrc, s);
    cudaMemsetAsync(end, 0, sizeof(uint32_t) * nsrc, s);
    if (nrec <= 0) return;
    const int64_t ntile = (nrec + kRsTile - 1) / kRsTile;
    // the tiles' status words, then the ticket counter
    cudaMemsetAsync(scan_words, 0, sizeof(unsigned long long) * (size_t)(ntile + 1), s);
    k_record_scan<<<(unsigned)ntile, kRsThreads, 0, s>>>(
        skey, sidx, nrec, crec, src_of, nsrc, srec, recE, rbeg, beg, end, scan_words,
        reinterpret_cast<uint32_t*>(scan_words + ntile), flags, withhold);
    counted(1);
}

}  // namespace

int64_t record_scan_tile() { return kRsTile; }

void grad_record_sources(const uint32_t* skey, const uint32_t* sidx, int64_t nrec,
                         const uint2* crec, const uint32_t* src_of, int64_t nsrc, uint2* srec,
                         uint32_t* recE, unsigned long long* scan_words, uint32_t* rbeg,
                         uint32_t* beg, uint32_t* end, int* flags, cudaStream_t s)
{
    record_scan(skey, sidx, nrec, crec, src_of, nsrc, srec, recE, scan_words, rbeg, beg, end,
                flags, 0, s);
}

void record_scan_wait_selftest(const uint32_t* skey, const uint32_t* sidx, int64_t nrec,
                               const uint2* crec, const uint32_t* src_of, int64_t nsrc,
                               uint2* srec, uint32_t* recE, unsigned long long* scan_words,
                               uint32_t* rbeg, uint32_t* beg, uint32_t* end, int* flags,
                               cudaStream_t s)
{
    record_scan(skey, sidx, nrec, crec, src_of, nsrc, srec, recE, scan_words, rbeg, beg, end,
                flags, 1, s);
}

namespace {

// Both kinds of source sums: item counts, their scan, the item -> source map,
// the item sums and the per-source reduction.
template <typename R, bool VJP>
void record_source_sums(const vec4<R>* pos, const vec4<R>* u, const vec4<R>* abar,
                        const vec4<R>* bbar, R ds, Tree<R> t, int64_t ncells, int64_t n,
                        const uint2* srec, const uint32_t* recE, int64_t nrec,
                        const uint32_t* rbeg, const uint32_t* beg, const uint32_t* end,
                        uint32_t* items, uint32_t* item_off, uint32_t* scan_tmp, double* part,
                        int64_t max_items, double* G, double* Q, cudaStream_t s)
{
    const int64_t nsrc = ncells + n;
    if (nsrc <= 0) return;
    k_item_counts<<<blocks(nsrc, kGradThreads), kGradThreads, 0, s>>>(beg, end, nsrc, items);
    scan_exclusive(items, item_off, nsrc, scan_tmp, s);
    // part holds 6 partial sums per item, then the item -> source map
    uint32_t* item_src = reinterpret_cast<uint32_t*>(part + 6 * max_items);
    k_item_sources<<<blocks(nsrc, kGradThreads), kGradThreads, 0, s>>>(item_off, nsrc, item_src);
    k_item_sums_rec<R, VJP><<<blocks(max_items * 32, kItemThreads), kItemThreads, 0, s>>>(
        pos, u, abar, bbar, ds, t, ncells, nsrc, srec, recE, nrec, rbeg, beg, end, item_off,
        item_src, part);
    k_item_reduce<R><<<blocks(nsrc, kGradThreads), kGradThreads, 0, s>>>(t, ncells, nsrc, item_off,
                                                                       part, G, Q);
    counted(4);
}

}  // namespace

template <typename R>
void grad_source_sums_rec(const vec4<R>* pos, const vec4<R>* u, Tree<R> t, int64_t ncells,
                          int64_t n, const uint2* srec, const uint32_t* recE, int64_t nrec,
                          const uint32_t* rbeg, const uint32_t* beg, const uint32_t* end,
                          uint32_t* items, uint32_t* item_off, uint32_t* scan_tmp, double* part,
                          int64_t max_items, double* G, double* Q, cudaStream_t s)
{
    record_source_sums<R, false>(pos, u, nullptr, nullptr, R(1), t, ncells, n, srec, recE, nrec,
                                 rbeg, beg, end, items, item_off, scan_tmp, part, max_items, G, Q,
                                 s);
}

template <typename R>
void vjp_source_sums_rec(const vec4<R>* pos, const vec4<R>* u, const vec4<R>* abar,
                         const vec4<R>* bbar, R ds, Tree<R> t, int64_t ncells, int64_t n,
                         const uint2* srec, const uint32_t* recE, int64_t nrec,
                         const uint32_t* rbeg, const uint32_t* beg, const uint32_t* end,
                         uint32_t* items, uint32_t* item_off, uint32_t* scan_tmp, double* part,
                         int64_t max_items, double* G, double* Q, cudaStream_t s)
{
    record_source_sums<R, true>(pos, u, abar, bbar, ds, t, ncells, n, srec, recE, nrec, rbeg, beg,
                                end, items, item_off, scan_tmp, part, max_items, G, Q, s);
}

template <typename R>
void grad_finish(Tree<R> t, int64_t ncells, int64_t n, const double* G, const double* Q,
                 const vec4<R>* h, const vec4<R>* f, R ds, vec4<R>* grad_pos, vec4<R>* grad_u,
                 cudaStream_t s)
{
    if (ncells <= 0) return;
    k_grad_finish<R><<<blocks(ncells, kGradThreads), kGradThreads, 0, s>>>(
        t, ncells, n, G, Q, h, f, ds, grad_pos, grad_u);
    counted();
}

template <typename R>
void grad_from_field(const vec4<R>* h, const vec4<R>* f, int64_t n, vec4<R>* grad_pos,
                     vec4<R>* grad_u, cudaStream_t s)
{
    if (n <= 0) return;
    k_grad_from_field<R><<<blocks(n, kGradThreads), kGradThreads, 0, s>>>(h, f, n, grad_pos,
                                                                          grad_u);
    counted();
}

template <typename R>
void vjp_finish(Tree<R> t, int64_t ncells, int64_t n, const double* G, const double* Q,
                const vec4<R>* dxt, const vec4<R>* dut, vec4<R>* dx, vec4<R>* du, cudaStream_t s)
{
    if (ncells <= 0) return;
    k_vjp_finish<R><<<blocks(ncells, kGradThreads), kGradThreads, 0, s>>>(t, ncells, n, G, Q, dxt,
                                                                         dut, dx, du);
    counted();
}

template <typename R>
void scatter_records(const uint32_t* perm, int64_t n, const vec4<R>* in, vec4<R>* out,
                     cudaStream_t s)
{
    if (n <= 0) return;
    k_scatter_records<R><<<blocks(n, kGradThreads), kGradThreads, 0, s>>>(perm, n, in, out);
    counted();
}

size_t sum_tmp_words(int64_t n) { return (size_t)((n + kGradThreads - 1) / kGradThreads) + 1; }

template <typename R>
void sum_z(const vec4<R>* v, int64_t n, double* tmp, double* out, cudaStream_t s)
{
    const int64_t nb = (n + kGradThreads - 1) / kGradThreads;
    if (nb > 0) k_sum_z_blocks<R><<<(unsigned)nb, kGradThreads, 0, s>>>(v, n, tmp);
    k_sum_final<<<1, kGradThreads, 0, s>>>(tmp, nb, out);
    counted(nb > 0 ? 2 : 1);
}

#define FFK_GRAD_INST(R)                                                                          \
    template void vjp_source_sums_rec<R>(const vec4<R>*, const vec4<R>*, const vec4<R>*,          \
                                         const vec4<R>*, R, Tree<R>, int64_t, int64_t,           \
                                         const uint2*, const uint32_t*, int64_t, const uint32_t*, \
                                         const uint32_t*, const uint32_t*, uint32_t*, uint32_t*,  \
                                         uint32_t*, double*, int64_t, double*, double*,          \
                                         cudaStream_t);                                          \
    template void vjp_finish<R>(Tree<R>, int64_t, int64_t, const double*, const double*,          \
                                const vec4<R>*, const vec4<R>*, vec4<R>*, vec4<R>*, cudaStream_t);\
    template void scatter_records<R>(const uint32_t*, int64_t, const vec4<R>*, vec4<R>*,          \
                                     cudaStream_t);                                               \
    template void sum_z<R>(const vec4<R>*, int64_t, double*, double*, cudaStream_t);              \
    template void grad_from_field<R>(const vec4<R>*, const vec4<R>*, int64_t, vec4<R>*, vec4<R>*, \
                                     cudaStream_t);                                               \
    template void grad_source_map<R>(Tree<R>, int64_t, uint32_t*, cudaStream_t);                 \
    template void grad_source_sums_rec<R>(const vec4<R>*, const vec4<R>*, Tree<R>, int64_t,       \
                                          int64_t, const uint2*, const uint32_t*, int64_t,        \
                                          const uint32_t*, const uint32_t*, const uint32_t*,      \
                                          uint32_t*, uint32_t*, uint32_t*, double*, int64_t,      \
                                          double*, double*, cudaStream_t);                        \
    template void grad_finish<R>(Tree<R>, int64_t, int64_t, const double*, const double*,         \
                                 const vec4<R>*, const vec4<R>*, R, vec4<R>*, vec4<R>*,           \
                                 cudaStream_t);
FFK_GRAD_INST(float)
FFK_GRAD_INST(double)
#undef FFK_GRAD_INST

}  // namespace ffk
