// Dipolar field and force kernels: the Barnes-Hut traversal (Sec. 3.2,
// kernel 5 of the paper's scheme, redesigned) and the all-pairs sum
// (Sec. 3.1, Algorithm 1).
//
// Traversal: a warp serves 32 consecutive particles of the Morton order,
// split into groups of G lanes.  Each lane keeps its own position in the
// depth-first cell list (`nxt`); a group visits cell i = min over its lanes
// of nxt, and only the lanes whose nxt == i act on it.  A lane therefore
// makes exactly the decisions of its own per-particle traversal, in the
// same order (children in octant order), while the cell record is fetched
// once per group (a broadcast load).  Large groups share more loads; small
// groups waste fewer lane slots on cells only some lanes need.  Skip
// pointers replace a stack.  Every lane's nxt strictly increases, so the
// loop ends after at most ncells visits per group.
#include <mutex>

#include "ffk.cuh"
#include "dipole.cuh"

namespace ffk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

// Knuth's TwoSum: s + e == a + b exactly (no fused or reordered operations).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// sigma^2 - r^2 without the cancellation error of the rounded r^2.  In FP32
// each square is split exactly into its rounded value and the remainder an fma
// recovers, the rounded squares are added with TwoSum so that their rounding
// errors are kept too, and sigma^2 enters as an unevaluated pair (hi, lo): the
// result carries one final rounding relative to the difference itself.  In
// FP64 the plain difference is accurate far beyond the parity bars.
__device__ __forceinline__ float sigma2_minus_r2(const FieldParams<float>& fp, float rx, float ry,
                                                 float rz)
{
    // streamed so that few temporaries are live at once: t gathers every
    // rounding error, a the rounded sum of squares
    float a = __fmul_rn(rx, rx);
    float t = __fmaf_rn(rx, rx, -a);
    float p = __fmul_rn(ry, ry);
    t = __fadd_rn(t, __fmaf_rn(ry, ry, -p));
    float e;
    two_sum(a, p, a, e);
    t = __fadd_rn(t, e);
    p = __fmul_rn(rz, rz);
    t = __fadd_rn(t, __fmaf_rn(rz, rz, -p));
    two_sum(a, p, a, e);
    t = __fadd_rn(t, e);
    two_sum(fp.lj_sigma2, -a, a, e);
    return __fadd_rn(a, __fsub_rn(__fadd_rn(e, fp.lj_sigma2_lo), t));
}

__device__ __forceinline__ double sigma2_minus_r2(const FieldParams<double>& fp, double rx, double ry,
                                                  double rz)
{
    return fp.lj_sigma2 - (rx * rx + ry * ry + rz * rz);
}

// Printed LJ force (Sec. 2, Eq. LJ) inside the cut, and half the pair
// energy 2 eps (s/r)^12 - 4 eps (s/r)^6 shifted to zero at the cut.  Whether
// the pair is inside is decided on r^2 = (rx rx + ry ry) + rz rz with every
// operation rounded once (r2 from the field code may carry fused rounding);
// that exact value is formed only near the cut.  Near contact (r ~ sigma) the
// bracket (s/r)^12 - (s/r)^6 is a small difference of two numbers near one, so
// it is formed as s6 (s6 - 1) with s6 - 1 = (s2 - 1)(s2^2 + s2 + 1) and
// s2 - 1 = (sigma^2 - r^2) / r^2, the difference compensated below
// r^2 = 1.5 sigma^2; beyond, sigma^2 - r^2 is at least a third of r^2 and the
// plain difference of the rounded r^2 is accurate to a few ulps.
template <typename R>
__device__ __forceinline__ void lj(const FieldParams<R>& fp, R rx, R ry, R rz, R r2, R& fx, R& fy,
                                   R& fz, R& e)
{
    if (!(r2 < fp.lj_rcut2_hi)) return;
    const R r2e = radd(radd(rmul(rx, rx), rmul(ry, ry)), rmul(rz, rz));
    if (!(r2e < fp.lj_rcut2 && r2e > R(0))) return;
    const R ir2 = R(1) / r2e;
    const R dsr = r2e < R(1.5) * fp.lj_sigma2 ? sigma2_minus_r2(fp, rx, ry, rz)
                                              : rsub(fp.lj_sigma2, r2e);
    const R s2m1 = dsr * ir2;
    const R s2 = R(1) + s2m1;
    const R s6 = s2 * s2 * s2;
    const R s6m1 = s2m1 * (s2 * s2 + s2 + R(1));
    const R c = fp.lj_eps24 * (s6 * s6m1) * ir2;
    fx += c * rx;
    fy += c * ry;
    fz += c * rz;
    e += R(0.5) * (fp.lj_e2 * s6 * s6 - fp.lj_e4 * s6 - fp.lj_shift);
}

// Derivative terms of one LJ pair for a vector-Jacobian product: the pair
// enters L = sum bbar . f through c (bbar_k - bbar_j) . r with c = 24 eps
// (s^12 - s^6) / r^2, whose r-derivative is c db + 2 c'(r^2) (db . r) r,
// c' = 24 eps s^6 (4 - 7 s^6) / r^4 (the same cut and bracket as lj()).
template <typename R>
__device__ __forceinline__ void lj_vjp(const FieldParams<R>& fp, R rx, R ry, R rz, R r2, R dbx,
                                       R dby, R dbz, R& dx, R& dy, R& dz)
{
    if (!(r2 < fp.lj_rcut2_hi)) return;
    const R r2e = radd(radd(rmul(rx, rx), rmul(ry, ry)), rmul(rz, rz));
    if (!(r2e < fp.lj_rcut2 && r2e > R(0))) return;
    const R ir2 = R(1) / r2e;
    const R s2m1 = sigma2_minus_r2(fp, rx, ry, rz) * ir2;
    const R s2 = R(1) + s2m1;
    const R s6 = s2 * s2 * s2;
    const R s6m1 = s2m1 * (s2 * s2 + s2 + R(1));
    const R c = fp.lj_eps24 * (s6 * s6m1) * ir2;
    const R cp = fp.lj_eps24 * s6 * (R(4) - R(7) * s6) * ir2 * ir2;
    const R k = R(2) * cp * (dbx * rx + dby * ry + dbz * rz);
    dx += c * dbx + k * rx;
    dy += c * dby + k * ry;
    dz += c * dbz + k * rz;
}

// Dipole-position (quadrupole) term of an accepted cell (an option beyond the
// paper's pseudo-particles): with S the symmetric part of sum (rho_i - c) (x) u_i
// and m its trace (q1 = (S_xx, S_yy, S_zz, S_xy), q2 = (S_xz, S_yz, m, 0)) and
// Phi(r) = (3 r.S.r - m r^2) / r^5, the field gains -grad Phi and the force
// -H Phi u_k:
//   grad Phi = 6 S r / r^5 + r (3 m / r^5 - 15 q / r^7),           q = r.S.r
//   H Phi u  = 6 S u / r^5 - 30 (r.u) S r / r^7
//            + r (105 q (r.u) / r^9 - 30 (S r.u) / r^7 - 15 m (r.u) / r^7)
//            + u (3 m / r^5 - 15 q / r^7)
template <typename R>
__device__ __forceinline__ void quad_term(R rx, R ry, R rz, R r2, const vec4<R>& q1,
                                          const vec4<R>& q2, R ux, R uy, R uz, R& hx, R& hy,
                                          R& hz, R& fx, R& fy, R& fz)
{
    const PairGeo<R> g = pair_geo<R>(rx, ry, rz, r2);
    const R srx = q1.x * rx + q1.w * ry + q2.x * rz;
    const R sry = q1.w * rx + q1.y * ry + q2.y * rz;
    const R srz = q2.x * rx + q2.y * ry + q1.z * rz;
    const R sux = q1.x * ux + q1.w * uy + q2.x * uz;
    const R suy = q1.w * ux + q1.y * uy + q2.y * uz;
    const R suz = q2.x * ux + q2.y * uy + q1.z * uz;
    const R q = rx * srx + ry * sry + rz * srz;
    const R ru = rx * ux + ry * uy + rz * uz;
    const R sru = srx * ux + sry * uy + srz * uz;
    const R m = q2.z;
    const R c6 = R(6) * g.ir5;
    const R cmq = R(3) * m * g.ir5 - R(15) * q * g.ir7;
    hx -= c6 * srx + cmq * rx;
    hy -= c6 * sry + cmq * ry;
    hz -= c6 * srz + cmq * rz;
    const R cs = R(30) * ru * g.ir7;
    const R cr = R(105) * q * ru * g.ir9 - R(30) * sru * g.ir7 - R(15) * m * ru * g.ir7;
    fx -= c6 * sux - cs * srx + cr * rx + cmq * ux;
    fy -= c6 * suy - cs * sry + cr * ry + cmq * uy;
    fz -= c6 * suz - cs * srz + cr * rz + cmq * uz;
}

// Opening test in the tree precision, each operation rounded once:
// side^2 < theta^2 ((dx dx + dy dy) + dz dz), and with LJ on, the distance
// from the particle to the cell's cube is at least rcut.  Beyond far2 =
// far2_of(rcut, reach) from the centre (reach: the largest distance from the
// centre to a point of the cube) the exact test cannot fail; the aggregation
// stores far2 with each cell's moment sum.
// (dx, dy, dz) = x - c, each component rounded once.
template <typename R>
__device__ __forceinline__ bool accept(const FieldParams<R>& fp, R dx, R dy, R dz, const vec4<R>& x,
                                       const vec4<R>& c, const vec4<R>* __restrict__ lo_arr, int i,
                                       R far2)
{
    const R d2 = radd(radd(rmul(dx, dx), rmul(dy, dy)), rmul(dz, dz));
    // c.w holds side^2, rounded once
    if (!(c.w < rmul(fp.theta2, d2))) return false;
    if (fp.use_rcut) {
        // the cube is at least d - reach away
        if (d2 >= far2) return true;
        const vec4<R> lo = lo_arr[i];
        const R side = lo.w;
        R t[3];
        const R xs[3] = {x.x, x.y, x.z};
        const R ls[3] = {lo.x, lo.y, lo.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R hi = radd(ls[a], side);
            const R below = rsub(ls[a], xs[a]);
            const R above = rsub(xs[a], hi);
            const R m = below > R(0) ? below : R(0);
            t[a] = above > m ? above : m;
        }
        const R b2 = radd(radd(rmul(t[0], t[0]), rmul(t[1], t[1])), rmul(t[2], t[2]));
        if (b2 < fp.rcut2) return false;
    }
    return true;
}

template <typename R>
__device__ __forceinline__ bool accept(const FieldParams<R>& fp, const vec4<R>& x, const vec4<R>& c,
                                       const vec4<R>* __restrict__ lo_arr, int i, R far2)
{
    return accept<R>(fp, rsub(x.x, c.x), rsub(x.y, c.y), rsub(x.z, c.z), x, c, lo_arr, i, far2);
}

// Preferred shared-memory share of the traversal (percent of the maximum):
// 7 % selects 16 KB, room for the per-block reservation of the resident
// blocks; the rest of the unified storage serves as L1 cache.
#ifndef FFK_TRAVERSE_CARVEOUT
#define FFK_TRAVERSE_CARVEOUT 7
#endif
constexpr int kTraverseCarveout = FFK_TRAVERSE_CARVEOUT;

// Traversal block shape: warps work independently (no shared memory, no
// block barrier), so the block size only sets how registers and warps are
// traded.  Registers are allocated per SM sub-partition (16384 each, a warp
// taking 32 x its registers), so 128 x 10 allows 48 registers a thread, room
// for the whole walk without spills.  The plain FP32 walk is lean enough for
// 128 x 12 (40 registers, 48 warps) with a few spilled words, and measures
// slightly faster so; the other walks keep 10 blocks.
#ifndef FFK_BH_THREADS
#define FFK_BH_THREADS 128
#endif
#ifndef FFK_BH_MIN_BLOCKS
#define FFK_BH_MIN_BLOCKS 10
#endif
#ifndef FFK_BH_MIN_BLOCKS_LEAN
#define FFK_BH_MIN_BLOCKS_LEAN 12
#endif
constexpr int kBhThreads = FFK_BH_THREADS;
constexpr int kBhMinBlocks = FFK_BH_MIN_BLOCKS;

// FP64 walks hold twice the registers per value.
#ifndef FFK_BH_MIN_BLOCKS_FP64
#define FFK_BH_MIN_BLOCKS_FP64 6
#endif

template <typename R, bool COUNT, bool QUAD>
constexpr int bh_min_blocks()
{
    return sizeof(R) == 8 ? FFK_BH_MIN_BLOCKS_FP64
           : (!COUNT && !QUAD) ? FFK_BH_MIN_BLOCKS_LEAN
                               : FFK_BH_MIN_BLOCKS;
}
static_assert(kBhThreads % 32 == 0, "whole warps");

// The walks that also write the source lists need a few more registers than
// the counting walk: 8 blocks of 128 (64 registers) in FP32.
#ifndef FFK_BH_MIN_BLOCKS_REC
#define FFK_BH_MIN_BLOCKS_REC 8
#endif
template <typename R>
constexpr int bh_rec_min_blocks()
{
    return sizeof(R) == 8 ? FFK_BH_MIN_BLOCKS_FP64 : FFK_BH_MIN_BLOCKS_REC;
}

// Minimum of v over each aligned group of G lanes.
template <int G>
__device__ __forceinline__ unsigned group_min(unsigned v)
{
    if (G == 32) return __reduce_min_sync(kFull, v);
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v = min(v, __shfl_xor_sync(kFull, v, o, G));
    return v;
}

// One task: the 32 consecutive particles task*32 .. task*32+31 of the key order.
template <typename R, bool COUNT, int G>
__device__ __forceinline__ void bh_task(int task, const vec4<R>* __restrict__ pos,
                                        const vec4<R>* __restrict__ u, int n, const Tree<R>& t,
                                        const FieldParams<R>& fp, unsigned ncells,
                                        vec4<R>* __restrict__ h, vec4<R>* __restrict__ f,
                                        R* __restrict__ esr, int4* __restrict__ counts, int* flags,
                                        const uint32_t* __restrict__ off, const Segs& sg)
{
    const int lane = threadIdx.x & 31;
    const int k = task * 32 + lane;
    const bool active = k < n;
    vec4<R> xk, uk;
    if (active) {
        xk = pos[k];
        uk = u[k];
    } else {
        xk.x = xk.y = xk.z = xk.w = R(0);
        uk = xk;
    }
    R hx = 0, hy = 0, hz = 0, fx = 0, fy = 0, fz = 0, sx = 0, sy = 0, sz = 0, es = 0, ck = 0;
    int nacc = 0, npair = 0, nopen = 0;
    // the cells of this particle's system: [first, end)
    unsigned first = 0, end = ncells;
    if (sg.of_pos && active) {
        const int sys = (int)sg.of_pos[k];
        first = off[sg.start[sys]];
        end = off[sg.start[sys + 1]];
    }
    unsigned nxt = active && first < end ? first : 0xffffffffu;
    for (;;) {
        const unsigned i = group_min<G>(nxt);
        if (G == 32) {
            if (i >= ncells) break;
        } else if (!__any_sync(kFull, i < ncells)) {
            break;
        }
        // a finished group keeps looping with i >= ncells while other groups of
        // the warp still work; its lanes must not touch cell i then
        if (nxt == i && i < ncells) {
            const Cell<R> cl = t.cell[i];
            const int4 nd = cl.node;
            const bool inside = nd.x <= k && k < nd.y;
            const bool leaf = (nd.w >> 8) != 0;
            const bool single = (nd.w >> 9) != 0;  // a one-particle leaf
            const vec4<R> c = cl.cen;
            const vec4<R> m = t.mom[i];  // .w: the cell's far2
            const bool acc = !inside && accept<R>(fp, xk, c, t.lo, (int)i, m.w);
            if (acc || (single && !inside)) {
                // the cell's pseudo-particle; for a one-particle leaf it is the
                // particle itself (centre and moment sum of one term are exact)
                const R rx = xk.x - c.x, ry = xk.y - c.y, rz = xk.z - c.z;
                const R r2 = rx * rx + ry * ry + rz * rz;
                walk_pair(rx, ry, rz, r2, uk.x, uk.y, uk.z, m.x, m.y, m.z, hx, hy, hz, fx, fy,
                              fz, ck);
                if (acc) {
                    if (COUNT) ++nacc;
                } else {
                    if (fp.include_sr) lj<R>(fp, rx, ry, rz, r2, sx, sy, sz, es);
                    if (COUNT) ++npair;
                }
                nxt = (unsigned)nd.z;
            } else if (leaf) {
                if (!single) {
                    for (int s = nd.x; s < nd.y; ++s) {
                        if (s == k) continue;
                        const vec4<R> xj = pos[s], uj = u[s];
                        const R rx = xk.x - xj.x, ry = xk.y - xj.y, rz = xk.z - xj.z;
                        const R r2 = rx * rx + ry * ry + rz * rz;
                        if (r2 > R(0)) {
                            walk_pair(rx, ry, rz, r2, uk.x, uk.y, uk.z, uj.x, uj.y, uj.z, hx,
                                          hy, hz, fx, fy, fz, ck);
                            if (fp.include_sr) lj<R>(fp, rx, ry, rz, r2, sx, sy, sz, es);
                        }
                        if (COUNT) ++npair;
                    }
                }
                nxt = (unsigned)nd.z;
            } else {
                if (COUNT) ++nopen;
                nxt = i + 1;
            }
            if (nxt <= i) {  // skip pointers must move forward
                atomicOr(flags, FLAG_TRAVERSE);
                nxt = 0xffffffffu;
            }
            if (nxt >= end) nxt = 0xffffffffu;  // this lane's system is done
        }
    }
    if (!active) return;
    vec4<R> ho, fo;
    ho.x = fp.dip_scale * hx;
    ho.y = fp.dip_scale * hy;
    ho.z = fp.dip_scale * hz;
    ho.w = R(0);
    fo.x = fp.dip_scale * (fx + uk.x * ck) + sx;
    fo.y = fp.dip_scale * (fy + uk.y * ck) + sy;
    fo.z = fp.dip_scale * (fz + uk.z * ck) + sz;
    fo.w = R(0);
    h[k] = ho;
    f[k] = fo;
    if (esr) esr[k] = es;
    if (COUNT) counts[k] = make_int4(nacc, npair, nopen, 0);
}

// A particle's source list in the entry pool: chunk k first, then chunks taken
// from *next.  Sources are kept four at a time and stored as one 16-byte word
// (a chunk holds a multiple of four); the chunk after a full one is taken at
// once.  Nothing is written to chunks at or past cap.
struct ChunkWriter {
    const EntryPool& p;   // the kernel's parameter: read where used, not held
    uint32_t ck, f;       // current chunk, sources so far
    uint32_t s0, s1, s2;  // the current group of four so far

    __device__ __forceinline__ ChunkWriter(const EntryPool& pool, uint32_t own)
        : p(pool), ck(own), f(0), s0(0), s1(0), s2(0)
    {
    }
    __device__ __forceinline__ void put(uint32_t key)
    {
        const uint32_t q = f & 3u;
        if (q == 0u) {
            s0 = key;
        } else if (q == 1u) {
            s1 = key;
        } else if (q == 2u) {
            s2 = key;
        } else {
            const uint32_t o = f & (uint32_t)(kPoolChunk - 1);
            if (ck < p.cap)
                *reinterpret_cast<uint4*>(p.keys + (size_t)ck * kPoolChunk + (o - 3u)) =
                    make_uint4(s0, s1, s2, key);
            if (o == (uint32_t)(kPoolChunk - 1)) {
                const uint32_t nk = p.first + atomicAdd(p.next, 1u);
                if (ck < p.cap) p.link[ck] = nk;
                ck = nk;
            }
        }
        ++f;
    }
    // the last, incomplete group
    __device__ __forceinline__ void flush()
    {
        const uint32_t r = f & 3u;
        if (r == 0u || ck >= p.cap) return;
        uint32_t* q = p.keys + (size_t)ck * kPoolChunk + ((f - r) & (uint32_t)(kPoolChunk - 1));
        q[0] = s0;
        if (r > 1u) q[1] = s1;
        if (r > 2u) q[2] = s2;
    }
};

// Independent per-lane walk (group size 1): each lane follows its own path
// through the cell list; no vote or shuffle per visited cell.  With REC (and
// COUNT) each source also goes to the particle's list in the entry pool.
template <typename R, bool COUNT, bool QUAD, bool REC = false>
__device__ __forceinline__ void bh_task1(int task, const vec4<R>* __restrict__ pos,
                                         const vec4<R>* __restrict__ u, int n, const Tree<R>& t,
                                         const FieldParams<R>& fp, unsigned ncells,
                                         vec4<R>* __restrict__ h, vec4<R>* __restrict__ f,
                                         R* __restrict__ esr, int4* __restrict__ counts, int* flags,
                                         const uint32_t* __restrict__ off, const Segs& sg,
                                         const EntryPool& ep = EntryPool())
{
    static_assert(!REC || (COUNT && !QUAD), "sources are recorded by the counting walk");
    const int lane = threadIdx.x & 31;
    const int k = task * 32 + lane;
    if (k >= n) return;
    ChunkWriter cw(ep, (uint32_t)k);
    const vec4<R> xk = pos[k], uk = u[k];
    R hx = 0, hy = 0, hz = 0, fx = 0, fy = 0, fz = 0, sx = 0, sy = 0, sz = 0, es = 0, ck = 0;
    int nacc = 0, npair = 0, nopen = 0;
    // the cells of this particle's system: [i, end)
    unsigned i = 0, end = ncells;
    if (sg.of_pos) {
        const int sys = (int)sg.of_pos[k];
        i = off[sg.start[sys]];
        end = off[sg.start[sys + 1]];
    }
    while (i < end) {
        const Cell<R> cl = t.cell[i];
        // requested with the cell so that one latency covers both loads; .w is
        // the cell's far2 for the opening test
        const vec4<R> m = t.mom[i];
        const int4 nd = cl.node;
        const bool inside = nd.x <= k && k < nd.y;
        const bool leaf = (nd.w >> 8) != 0;
        const bool single = (nd.w >> 9) != 0;  // a one-particle leaf
        const vec4<R> c = cl.cen;
        // the separation serves the opening test (each component rounded once
        // either way) and the pair terms
        const R rx = rsub(xk.x, c.x), ry = rsub(xk.y, c.y), rz = rsub(xk.z, c.z);
        const R r2 = rx * rx + ry * ry + rz * rz;
        const bool out1 = single && !inside;
        // A one-particle leaf adds the same dipole term whether accepted or
        // summed as a pair; the two differ only by the LJ term, which is zero
        // unless r2 < lj_rcut2_hi, and in the counts.  Below lj_rcut2_lo the
        // particle, and so its cube, is within rcut (by a margin far above the
        // rounding of the cube's corners): the opening test fails.  The plain
        // walk therefore decides such a leaf only in between.
        const bool acc =
            (!COUNT && !QUAD && out1)
                ? (fp.include_sr && r2 < fp.lj_rcut2_hi && r2 >= fp.lj_rcut2_lo &&
                   accept<R>(fp, rx, ry, rz, xk, c, t.lo, (int)i, m.w))
                : (!inside && accept<R>(fp, rx, ry, rz, xk, c, t.lo, (int)i, m.w));
        unsigned nxt = i + 1;
        if (acc || out1) {
            // the cell's pseudo-particle; for a one-particle leaf it is the
            // particle itself (centre and moment sum of one term are exact)
            walk_pair(rx, ry, rz, r2, uk.x, uk.y, uk.z, m.x, m.y, m.z, hx, hy, hz, fx, fy, fz,
                          ck);
            if (REC) cw.put(i + (uint32_t)nd.x);
            if (QUAD && acc && r2 > R(0))
                quad_term<R>(rx, ry, rz, r2, t.q1[i], t.q2[i], uk.x, uk.y, uk.z, hx, hy, hz, fx,
                             fy, fz);
            if (acc) {
                if (COUNT) ++nacc;
            } else {
                if (fp.include_sr) lj<R>(fp, rx, ry, rz, r2, sx, sy, sz, es);
                if (COUNT) ++npair;
            }
            nxt = (unsigned)nd.z;
        } else if (leaf) {
            if (!single) {
                for (int s = nd.x; s < nd.y; ++s) {
                    if (s == k) continue;
                    if (REC) cw.put(i + 1u + (uint32_t)s);
                    const vec4<R> xj = pos[s], uj = u[s];
                    const R rx = xk.x - xj.x, ry = xk.y - xj.y, rz = xk.z - xj.z;
                    const R r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 > R(0)) {
                        walk_pair(rx, ry, rz, r2, uk.x, uk.y, uk.z, uj.x, uj.y, uj.z, hx, hy,
                                      hz, fx, fy, fz, ck);
                        if (fp.include_sr) lj<R>(fp, rx, ry, rz, r2, sx, sy, sz, es);
                    }
                    if (COUNT) ++npair;
                }
            }
            nxt = (unsigned)nd.z;
        } else {
            if (COUNT) ++nopen;
        }
        if (nxt <= i) {  // skip pointers must move forward
            atomicOr(flags, FLAG_TRAVERSE);
            break;
        }
        i = nxt;
    }
    if (REC) cw.flush();
    vec4<R> ho, fo;
    ho.x = fp.dip_scale * hx;
    ho.y = fp.dip_scale * hy;
    ho.z = fp.dip_scale * hz;
    ho.w = R(0);
    fo.x = fp.dip_scale * (fx + uk.x * ck) + sx;
    fo.y = fp.dip_scale * (fy + uk.y * ck) + sy;
    fo.z = fp.dip_scale * (fz + uk.z * ck) + sz;
    fo.w = R(0);
    h[k] = ho;
    f[k] = fo;
    if (esr) esr[k] = es;
    if (COUNT) counts[k] = make_int4(nacc, npair, nopen, 0);
}

// Target-side terms of a vector-Jacobian product of h and f (cotangents abar,
// bbar) for L = sum abar . h + bbar . f, on the walk of bh_task1 (the same
// decisions in the same order):
//   dL/du_k   += ds grad phi(r; bbar_k, w_s)
//   dL/drho_k += ds [grad phi(r; abar_k, w_s) + H phi(r; u_k, w_s) bbar_k] + LJ terms
// written to dxt, dut; the source-side terms come from the source records.
template <typename R>
struct VjpIn {
    const vec4<R>* u;
    const vec4<R>* abar;
    const vec4<R>* bbar;
    vec4<R>* dxt;
    vec4<R>* dut;
};

template <typename R>
__device__ __forceinline__ void vjp_target(const FieldParams<R>& fp, const vec4<R>& xk,
                                           const vec4<R>& uk, const vec4<R>& ak,
                                           const vec4<R>& bk, const vec4<R>& xs,
                                           const vec4<R>& ws, R& dx, R& dy, R& dz, R& ux, R& uy,
                                           R& uz)
{
    const R rx = xk.x - xs.x, ry = xk.y - xs.y, rz = xk.z - xs.z;
    const R r2 = rx * rx + ry * ry + rz * rz;
    if (!(r2 > R(0))) return;
    const PairGeo<R> g = pair_geo<R>(rx, ry, rz, r2);
    const R ds = fp.dip_scale;
    grad_phi_add<R>(g, bk.x, bk.y, bk.z, ws.x, ws.y, ws.z, ds, ux, uy, uz);
    grad_phi_add<R>(g, ak.x, ak.y, ak.z, ws.x, ws.y, ws.z, ds, dx, dy, dz);
    hess_phi_add<R>(g, uk.x, uk.y, uk.z, ws.x, ws.y, ws.z, bk.x, bk.y, bk.z, ds, dx, dy, dz);
}

// With REC the walk also writes each particle's sources to the entry pool and
// their number to counts[k].x (as the counting walk of the gradient pass does).
template <typename R, bool REC = false>
__device__ __forceinline__ void vjp_task(int task, const vec4<R>* __restrict__ pos, int n,
                                         const Tree<R>& t, const FieldParams<R>& fp,
                                         unsigned ncells, int* flags,
                                         const uint32_t* __restrict__ off, const Segs& sg,
                                         const VjpIn<R>& vj, int4* __restrict__ counts = nullptr,
                                         const EntryPool& ep = EntryPool())
{
    const int k = task * 32 + (threadIdx.x & 31);
    if (k >= n) return;
    ChunkWriter cw(ep, (uint32_t)k);
    int nent = 0;
    const vec4<R> xk = pos[k];
    const vec4<R> uk = vj.u[k], ak = vj.abar[k], bk = vj.bbar[k];
    R dx = 0, dy = 0, dz = 0, ux = 0, uy = 0, uz = 0;
    unsigned i = 0, end = ncells;
    if (sg.of_pos) {
        const int sys = (int)sg.of_pos[k];
        i = off[sg.start[sys]];
        end = off[sg.start[sys + 1]];
    }
    while (i < end) {
        const Cell<R> cl = t.cell[i];
        const int4 nd = cl.node;
        const bool inside = nd.x <= k && k < nd.y;
        const bool leaf = (nd.w >> 8) != 0;
        const bool single = (nd.w >> 9) != 0;  // a one-particle leaf
        const vec4<R> ws = t.mom[i];  // moment sum; .w: the cell's far2
        const bool out1 = single && !inside;
        const R rx = rsub(xk.x, cl.cen.x), ry = rsub(xk.y, cl.cen.y), rz = rsub(xk.z, cl.cen.z);
        const R r2 = rx * rx + ry * ry + rz * rz;
        // A one-particle leaf gives the same dipole terms whether accepted or
        // summed as a pair; only the LJ term differs, and it vanishes outside
        // [lj_rcut2_lo, lj_rcut2_hi) (see bh_task1), so it is decided only there.
        const bool acc =
            out1 ? (fp.include_sr && r2 < fp.lj_rcut2_hi && r2 >= fp.lj_rcut2_lo &&
                    accept<R>(fp, rx, ry, rz, xk, cl.cen, t.lo, (int)i, ws.w))
                 : (!inside && accept<R>(fp, rx, ry, rz, xk, cl.cen, t.lo, (int)i, ws.w));
        unsigned nxt = i + 1;
        if (acc || out1) {
            if (REC) {
                cw.put(i + (uint32_t)nd.x);
                ++nent;
            }
            vjp_target<R>(fp, xk, uk, ak, bk, cl.cen, ws, dx, dy, dz, ux, uy, uz);
            if (!acc && fp.include_sr) {
                const vec4<R> bj = vj.bbar[nd.x];
                lj_vjp<R>(fp, rx, ry, rz, r2, bk.x - bj.x, bk.y - bj.y, bk.z - bj.z, dx, dy, dz);
            }
            nxt = (unsigned)nd.z;
        } else if (leaf) {
            if (!single) {
                for (int s = nd.x; s < nd.y; ++s) {
                    if (s == k) continue;
                    if (REC) {
                        cw.put(i + 1u + (uint32_t)s);
                        ++nent;
                    }
                    const vec4<R> xj = pos[s], uj = vj.u[s], bj = vj.bbar[s];
                    vjp_target<R>(fp, xk, uk, ak, bk, xj, uj, dx, dy, dz, ux, uy, uz);
                    if (fp.include_sr) {
                        const R rx = xk.x - xj.x, ry = xk.y - xj.y, rz = xk.z - xj.z;
                        const R r2 = rx * rx + ry * ry + rz * rz;
                        if (r2 > R(0))
                            lj_vjp<R>(fp, rx, ry, rz, r2, bk.x - bj.x, bk.y - bj.y, bk.z - bj.z,
                                      dx, dy, dz);
                    }
                }
            }
            nxt = (unsigned)nd.z;
        }
        if (nxt <= i) {
            atomicOr(flags, FLAG_TRAVERSE);
            break;
        }
        i = nxt;
    }
    vec4<R> o;
    o.x = dx; o.y = dy; o.z = dz; o.w = R(0);
    vj.dxt[k] = o;
    o.x = ux; o.y = uy; o.z = uz;
    vj.dut[k] = o;
    if (REC) {
        cw.flush();
        counts[k] = make_int4(nent, 0, 0, 0);
    }
}

// The target-side walk on the traversal's schedule: warps take 32-particle
// tasks from their SM's Morton segment first (see k_bh).
template <typename R, bool REC>
__global__ void __launch_bounds__(kBhThreads, (REC ? bh_rec_min_blocks<R>() : kBhMinBlocks)) k_bh_vjp(
    const vec4<R>* __restrict__ pos, int n, Tree<R> t, FieldParams<R> fp, int* flags,
    int* __restrict__ work, int nseg, const uint32_t* __restrict__ off, Segs sg, VjpIn<R> vj,
    int4* __restrict__ counts, EntryPool ep)
{
    if (*flags & FLAG_CAPACITY) return;
    const unsigned ncells = (unsigned)*t.ncells;
    const int ntask = (n + 31) / 32;
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const int home = (int)(smid % (unsigned)nseg);
    const int lane = threadIdx.x & 31;
    for (int probe = 0; probe < nseg; ++probe) {
        const int ws = (home + probe) % nseg;
        const int t0 = (int)((int64_t)ntask * ws / nseg);
        const int t1 = (int)((int64_t)ntask * (ws + 1) / nseg);
        for (;;) {
            int got = 0;
            if (lane == 0) got = atomicAdd(&work[ws], 1);
            got = __shfl_sync(kFull, got, 0);
            const int task = t0 + got;
            if (task >= t1) break;
            vjp_task<R, REC>(task, pos, n, t, fp, ncells, flags, off, sg, vj, counts, ep);
        }
    }
}

// Persistent traversal: the key order is cut into nseg contiguous segments of
// 32-particle tasks; a warp takes tasks from the segment of the SM it runs on
// (so warps sharing an L1 cache walk neighbouring parts of the tree) and then
// from the following segments once its own is used up.  Task counters
// (work[0..nseg)) start at zero; every task is taken exactly once.
template <typename R, bool COUNT, int G, bool QUAD, int THREADS = kBhThreads,
          int MINB = bh_min_blocks<R, COUNT, QUAD>()>
__global__ void __launch_bounds__(THREADS, MINB) k_bh(const vec4<R>* __restrict__ pos,
                                            const vec4<R>* __restrict__ u, int n, Tree<R> t,
                                            FieldParams<R> fp, vec4<R>* __restrict__ h,
                                            vec4<R>* __restrict__ f, R* __restrict__ esr,
                                            int4* __restrict__ counts, int* flags,
                                            int* __restrict__ work, int nseg,
                                            const uint32_t* __restrict__ off, Segs sg)
{
    if (*flags & FLAG_CAPACITY) return;
    const unsigned ncells = (unsigned)*t.ncells;
    const int ntask = (n + 31) / 32;
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const int home = (int)(smid % (unsigned)nseg);
    const int lane = threadIdx.x & 31;
    for (int probe = 0; probe < nseg; ++probe) {
        const int ws = (home + probe) % nseg;
        const int t0 = (int)((int64_t)ntask * ws / nseg);
        const int t1 = (int)((int64_t)ntask * (ws + 1) / nseg);
        for (;;) {
            int got = 0;
            if (lane == 0) got = atomicAdd(&work[ws], 1);
            got = __shfl_sync(kFull, got, 0);
            const int task = t0 + got;
            if (task >= t1) break;
            if (G == 1)
                bh_task1<R, COUNT, QUAD>(task, pos, u, n, t, fp, ncells, h, f, esr, counts, flags,
                                         off, sg);
            else
                bh_task<R, COUNT, G>(task, pos, u, n, t, fp, ncells, h, f, esr, counts, flags, off,
                                     sg);
        }
    }
}

// The counting walk that also records every particle's sources (energy
// gradient), on the schedule of k_bh.

template <typename R>
__global__ void __launch_bounds__(kBhThreads, (bh_rec_min_blocks<R>())) k_bh_rec(
    const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ u, int n, Tree<R> t,
    FieldParams<R> fp, vec4<R>* __restrict__ h, vec4<R>* __restrict__ f, R* __restrict__ esr,
    int4* __restrict__ counts, int* flags, int* __restrict__ work, int nseg,
    const uint32_t* __restrict__ off, Segs sg, EntryPool ep)
{
    if (*flags & FLAG_CAPACITY) return;
    const unsigned ncells = (unsigned)*t.ncells;
    const int ntask = (n + 31) / 32;
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const int home = (int)(smid % (unsigned)nseg);
    const int lane = threadIdx.x & 31;
    for (int probe = 0; probe < nseg; ++probe) {
        const int ws = (home + probe) % nseg;
        const int t0 = (int)((int64_t)ntask * ws / nseg);
        const int t1 = (int)((int64_t)ntask * (ws + 1) / nseg);
        for (;;) {
            int got = 0;
            if (lane == 0) got = atomicAdd(&work[ws], 1);
            got = __shfl_sync(kFull, got, 0);
            const int task = t0 + got;
            if (task >= t1) break;
            bh_task1<R, true, false, true>(task, pos, u, n, t, fp, ncells, h, f, esr, counts,
                                           flags, off, sg, ep);
        }
    }
}

// All pairs: one thread per target; source records staged through shared
// memory one block-sized tile at a time (Sec. 3.1, Algorithm 1).
constexpr int kApThreads = 256;

template <typename R>
__global__ void __launch_bounds__(kApThreads) k_ap(const vec4<R>* __restrict__ pos,
                                                   const vec4<R>* __restrict__ u, int n,
                                                   FieldParams<R> fp, vec4<R>* __restrict__ h,
                                                   vec4<R>* __restrict__ f, R* __restrict__ esr)
{
    __shared__ vec4<R> sp[kApThreads];
    __shared__ vec4<R> su[kApThreads];
    const int k = blockIdx.x * kApThreads + threadIdx.x;
    const bool active = k < n;
    vec4<R> xk, uk;
    if (active) {
        xk = pos[k];
        uk = u[k];
    } else {
        xk.x = xk.y = xk.z = xk.w = R(0);
        uk = xk;
    }
    // two-level sums: each tile is summed on its own, then added to the total,
    // so rounding grows with sqrt(tile) + sqrt(n / tile) terms instead of sqrt(n)
    R hx = 0, hy = 0, hz = 0, fx = 0, fy = 0, fz = 0, sx = 0, sy = 0, sz = 0, es = 0;
    for (int tile = 0; tile < n; tile += kApThreads) {
        const int j = tile + threadIdx.x;
        if (j < n) {
            sp[threadIdx.x] = pos[j];
            su[threadIdx.x] = u[j];
        }
        __syncthreads();
        const int lim = min(kApThreads, n - tile);
        R thx = 0, thy = 0, thz = 0, tfx = 0, tfy = 0, tfz = 0;
        for (int jj = 0; jj < lim; ++jj) {
            if (tile + jj == k) continue;
            const vec4<R> xj = sp[jj], uj = su[jj];
            const R rx = xk.x - xj.x, ry = xk.y - xj.y, rz = xk.z - xj.z;
            const R r2 = rx * rx + ry * ry + rz * rz;
            if (r2 > R(0)) {
                dipole<R>(rx, ry, rz, r2, uk.x, uk.y, uk.z, uj.x, uj.y, uj.z, thx, thy, thz, tfx,
                          tfy, tfz);
                if (fp.include_sr) lj<R>(fp, rx, ry, rz, r2, sx, sy, sz, es);
            }
        }
        hx += thx;
        hy += thy;
        hz += thz;
        fx += tfx;
        fy += tfy;
        fz += tfz;
        __syncthreads();
    }
    if (!active) return;
    vec4<R> ho, fo;
    ho.x = fp.dip_scale * hx;
    ho.y = fp.dip_scale * hy;
    ho.z = fp.dip_scale * hz;
    ho.w = R(0);
    fo.x = fp.dip_scale * fx + sx;
    fo.y = fp.dip_scale * fy + sy;
    fo.z = fp.dip_scale * fz + sz;
    fo.w = R(0);
    h[k] = ho;
    f[k] = fo;
    if (esr) esr[k] = es;
}

// Shape of a persistent grid on the current device: one work segment per SM
// (at most kWorkSegments) and as many blocks as fit at once.  `occupancy`
// configures the caller's kernel and returns its resident blocks per SM; each
// kernel instance keeps its own per-device cache, guarded by its own mutex.
struct PersistentGrid {
    int blocks = 0;
    int nseg = 0;
};
constexpr int kMaxDevices = 64;

template <typename F>
PersistentGrid persistent_grid(PersistentGrid* cache, std::mutex& mu, F occupancy)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const bool cached = dev >= 0 && dev < kMaxDevices;
    std::lock_guard<std::mutex> lock(mu);
    if (cached && cache[dev].blocks > 0) return cache[dev];
    PersistentGrid g;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = occupancy();
    if (per_sm < 1) per_sm = 1;
    if (nsm < 1) nsm = 1;
    if (nsm > kWorkSegments) nsm = kWorkSegments;
    g.nseg = nsm;
    g.blocks = per_sm * nsm;
    if (cached) cache[dev] = g;
    return g;
}

}  // namespace

template <typename R, bool COUNT, int G, bool QUAD = false, int THREADS = kBhThreads,
          int MINB = bh_min_blocks<R, COUNT, QUAD>()>
void bh_launch_g(const vec4<R>* pos, const vec4<R>* u, int64_t n, Tree<R> t, FieldParams<R> fp,
                 vec4<R>* h, vec4<R>* f, R* esr, int4* counts, int* flags, int* work,
                 const uint32_t* off, Segs sg, cudaStream_t s)
{
    // persistent grid: as many blocks as fit on the device at once; a small
    // shared-memory carveout (the kernel uses none) leaves the rest to L1
    static std::mutex mu;
    static PersistentGrid cache[kMaxDevices];
    const auto kern = k_bh<R, COUNT, G, QUAD, THREADS, MINB>;
    const PersistentGrid g = persistent_grid(cache, mu, [kern] {
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             kTraverseCarveout);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0);
        return per_sm;
    });
    cudaMemsetAsync(work, 0, sizeof(int) * g.nseg, s);
    kern<<<g.blocks, THREADS, 0, s>>>(pos, u, (int)n, t, fp, h, f, esr, counts, flags, work,
                                      g.nseg, off, sg);
}

template <typename R, bool COUNT>
void bh_launch(const vec4<R>* pos, const vec4<R>* u, int64_t n, Tree<R> t, FieldParams<R> fp,
               vec4<R>* h, vec4<R>* f, R* esr, int4* counts, int* flags, int* work, int group,
               int sched, const uint32_t* off, Segs sg, cudaStream_t s)
{
    if constexpr (sizeof(R) == 4 && !COUNT) {
        // a tuned launch schedule of the plain FP32 walk (see kSchedules)
        if (sched >= 1 && sched <= kNumSchedules && !t.q1) {
#define FFK_SCHED(G, T, B) bh_launch_g<R, false, G, false, T, B>(pos, u, n, t, fp, h, f, esr, counts, flags, work, off, sg, s)
            switch (sched) {
                case 1: FFK_SCHED(1, 128, 12); return;
                case 2: FFK_SCHED(1, 128, 10); return;
                case 3: FFK_SCHED(1, 128, 8); return;
                case 4: FFK_SCHED(1, 256, 6); return;
                case 5: FFK_SCHED(1, 256, 4); return;
                case 6: FFK_SCHED(1, 64, 24); return;
                case 7: FFK_SCHED(1, 64, 16); return;
                case 8: FFK_SCHED(2, 128, 12); return;
                case 9: FFK_SCHED(4, 128, 12); return;
                default: FFK_SCHED(8, 128, 12); return;
            }
#undef FFK_SCHED
        }
    }
    if (sched >= 1 && sched <= kNumSchedules) group = kSchedules[sched - 1].group;
    if (t.q1) {
        // the dipole-position terms are evaluated by the one-lane walk only
        bh_launch_g<R, COUNT, 1, true>(pos, u, n, t, fp, h, f, esr, counts, flags, work, off, sg,
                                       s);
        return;
    }
#define FFK_BH_CASE(G) bh_launch_g<R, COUNT, G>(pos, u, n, t, fp, h, f, esr, counts, flags, work, off, sg, s)
    switch (group) {
        case 1: FFK_BH_CASE(1); break;
        case 2: FFK_BH_CASE(2); break;
        case 4: FFK_BH_CASE(4); break;
        case 8: FFK_BH_CASE(8); break;
        case 16: FFK_BH_CASE(16); break;
        default: FFK_BH_CASE(32); break;
    }
#undef FFK_BH_CASE
}

template <typename R>
void bh_field(const vec4<R>* pos, const vec4<R>* u, int64_t n, Tree<R> t, FieldParams<R> fp,
              vec4<R>* h, vec4<R>* f, R* esr, int4* counts, int* flags, int* work, int group,
              int sched, const uint32_t* off, Segs sg, cudaStream_t s)
{
    if (counts)
        bh_launch<R, true>(pos, u, n, t, fp, h, f, esr, counts, flags, work, group, sched, off, sg,
                           s);
    else
        bh_launch<R, false>(pos, u, n, t, fp, h, f, esr, counts, flags, work, group, sched, off,
                            sg, s);
    counted();
}

template <typename R>
void bh_field_record(const vec4<R>* pos, const vec4<R>* u, int64_t n, Tree<R> t, FieldParams<R> fp,
                     vec4<R>* h, vec4<R>* f, R* esr, int4* counts, int* flags, int* work,
                     const uint32_t* off, Segs sg, EntryPool pool, cudaStream_t s)
{
    if (n <= 0) return;
    static std::mutex mu;
    static PersistentGrid cache[kMaxDevices];
    const PersistentGrid g = persistent_grid(cache, mu, [] {
        cudaFuncSetAttribute(k_bh_rec<R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             kTraverseCarveout);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bh_rec<R>, kBhThreads, 0);
        return per_sm;
    });
    cudaMemsetAsync(work, 0, sizeof(int) * g.nseg, s);
    k_bh_rec<R><<<g.blocks, kBhThreads, 0, s>>>(pos, u, (int)n, t, fp, h, f, esr, counts, flags,
                                                work, g.nseg, off, sg, pool);
    counted();
}

template <typename R>
void ap_field(const vec4<R>* pos, const vec4<R>* u, int64_t n, FieldParams<R> fp, vec4<R>* h,
              vec4<R>* f, R* esr, cudaStream_t s)
{
    const unsigned g = (unsigned)((n + kApThreads - 1) / kApThreads);
    k_ap<R><<<g, kApThreads, 0, s>>>(pos, u, (int)n, fp, h, f, esr);
    counted();
}

template void bh_field<float>(const float4*, const float4*, int64_t, Tree<float>,
                              FieldParams<float>, float4*, float4*, float*, int4*, int*, int*,
                              int, int, const uint32_t*, Segs, cudaStream_t);
template void bh_field<double>(const dvec4*, const dvec4*, int64_t, Tree<double>,
                               FieldParams<double>, dvec4*, dvec4*, double*, int4*, int*, int*,
                               int, int, const uint32_t*, Segs, cudaStream_t);
template void bh_field_record<float>(const float4*, const float4*, int64_t, Tree<float>,
                                     FieldParams<float>, float4*, float4*, float*, int4*, int*,
                                     int*, const uint32_t*, Segs, EntryPool, cudaStream_t);
template void bh_field_record<double>(const dvec4*, const dvec4*, int64_t, Tree<double>,
                                      FieldParams<double>, dvec4*, dvec4*, double*, int4*, int*,
                                      int*, const uint32_t*, Segs, EntryPool, cudaStream_t);
template void ap_field<float>(const float4*, const float4*, int64_t, FieldParams<float>, float4*,
                              float4*, float*, cudaStream_t);
template void ap_field<double>(const dvec4*, const dvec4*, int64_t, FieldParams<double>, dvec4*,
                               dvec4*, double*, cudaStream_t);


template <typename R, bool REC>
void bh_vjp_launch(const vec4<R>* pos, int64_t n, Tree<R> t, FieldParams<R> fp, int* flags,
                   int* work, const uint32_t* off, Segs sg, VjpIn<R> vj, int4* counts,
                   EntryPool ep, cudaStream_t s)
{
    static std::mutex mu;
    static PersistentGrid cache[kMaxDevices];
    const PersistentGrid g = persistent_grid(cache, mu, [] {
        cudaFuncSetAttribute(k_bh_vjp<R, REC>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             kTraverseCarveout);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bh_vjp<R, REC>, kBhThreads, 0);
        return per_sm;
    });
    cudaMemsetAsync(work, 0, sizeof(int) * g.nseg, s);
    k_bh_vjp<R, REC><<<g.blocks, kBhThreads, 0, s>>>(pos, (int)n, t, fp, flags, work, g.nseg, off,
                                                     sg, vj, counts, ep);
    counted();
}

template <typename R>
void bh_vjp_target(const vec4<R>* pos, const vec4<R>* u, const vec4<R>* abar, const vec4<R>* bbar,
                   int64_t n, Tree<R> t, FieldParams<R> fp, int* flags, int* work,
                   const uint32_t* off, Segs sg, vec4<R>* dxt, vec4<R>* dut, cudaStream_t s,
                   int4* counts, const EntryPool* pool)
{
    if (n <= 0) return;
    VjpIn<R> vj;
    vj.u = u;
    vj.abar = abar;
    vj.bbar = bbar;
    vj.dxt = dxt;
    vj.dut = dut;
    if (pool)
        bh_vjp_launch<R, true>(pos, n, t, fp, flags, work, off, sg, vj, counts, *pool, s);
    else
        bh_vjp_launch<R, false>(pos, n, t, fp, flags, work, off, sg, vj, nullptr, EntryPool(), s);
}

template void bh_vjp_target<float>(const float4*, const float4*, const float4*, const float4*,
                                   int64_t, Tree<float>, FieldParams<float>, int*, int*,
                                   const uint32_t*, Segs, float4*, float4*, cudaStream_t, int4*,
                                   const EntryPool*);
template void bh_vjp_target<double>(const dvec4*, const dvec4*, const dvec4*, const dvec4*,
                                    int64_t, Tree<double>, FieldParams<double>, int*, int*,
                                    const uint32_t*, Segs, dvec4*, dvec4*, cudaStream_t, int4*,
                                    const EntryPool*);

}  // namespace ffk
