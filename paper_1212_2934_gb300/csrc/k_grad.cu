// Gradient of the Barnes-Hut dipolar energy E = -1/2 sum_m u_m . h_m with
// the opening decisions frozen (Sec. 3.2 traversal, Sec. 5 energy).
//
// With phi(r; a, b) = a . T(r) b and h_m = sum over m's sources s of
// T(rho_m - x_s) w_s (cells: centre and moment sum; exact pairs: particles):
//   dE/du_k   = -1/2 [ h_k + ds sum over (m, s), k in s, of T(rho_m - x_s) u_m ]
//   dE/drho_k = -1/2 [ f_k - ds sum over (m, s), k in s, of
//                      grad phi(rho_m - x_s; w_s, u_m) / n_s ]
// h and f are the dipolar field and force of the same traversal (ds
// included).  The reverse sums are formed without atomics: the traversal
// records every (source, target) entry, a stable radix sort on the source
// groups them, one warp per source sums its entries in a fixed order, and each
// leaf adds the sums of its ancestor cells for its particles.
#include "dipole.cuh"
#include "ffk.cuh"

namespace ffk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGradThreads = 256;

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

// (keys outside 0 .. nsrc - 1 can only come from a recording walk that
// raised its flag; they are skipped)
__global__ void k_segments(const uint32_t* __restrict__ keys, int64_t ne, int64_t nsrc,
                           uint32_t* beg, uint32_t* end)
{
    // four consecutive keys per thread (one 16-byte load; keys is 16-byte
    // aligned), their neighbours across the group from plain loads
    const int64_t i0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (i0 >= ne) return;
    uint32_t k[4];
    if (i0 + 4 <= ne) {
        const uint4 q = *reinterpret_cast<const uint4*>(keys + i0);
        k[0] = q.x; k[1] = q.y; k[2] = q.z; k[3] = q.w;
    } else {
        for (int j = 0; j < 4; ++j) k[j] = i0 + j < ne ? keys[i0 + j] : 0u;
    }
    uint32_t prev = i0 > 0 ? keys[i0 - 1] : 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t i = i0 + j;
        if (i >= ne) break;
        const uint32_t kk = k[j];
        const uint32_t next = i + 1 < ne ? (j < 3 ? k[j + 1] : keys[i + 1]) : 0u;
        if ((int64_t)kk < nsrc) {
            if (i == 0 || prev != kk) beg[kk] = (uint32_t)i;
            if (i == ne - 1 || next != kk) end[kk] = (uint32_t)(i + 1);
        }
        prev = kk;
    }
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

// One warp per item: the terms of its entries summed in single precision (at
// most 32 per lane, then across the warp), written as six FP64 partials.
template <typename R>
__global__ void __launch_bounds__(kGradThreads) k_item_sums(
    const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ u, Tree<R> t, int64_t ncells,
    int64_t nsrc, const uint32_t* __restrict__ vals, const uint32_t* __restrict__ beg,
    const uint32_t* __restrict__ end, const uint32_t* __restrict__ item_off,
    const uint32_t* __restrict__ item_src, double* __restrict__ part)
{
    const int64_t it = ((int64_t)blockIdx.x * kGradThreads + threadIdx.x) >> 5;
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
    const uint32_t b = beg[s] + (uint32_t)(it - item_off[s]) * (uint32_t)kGradItemEntries;
    const uint32_t e = min(end[s], b + (uint32_t)kGradItemEntries);
    const uint32_t np = (uint32_t)(nsrc - ncells);
    R gx = 0, gy = 0, gz = 0, qx = 0, qy = 0, qz = 0;
    for (uint32_t k = b + lane; k < e; k += 32) {
        const uint32_t m = vals[k];
        if (m >= np) continue;  // only after a flagged recording walk
        const vec4<R> xm = pos[m], um = u[m];
        const R rx = xm.x - x.x, ry = xm.y - x.y, rz = xm.z - x.z;
        const R r2 = rx * rx + ry * ry + rz * rz;
        // T(r) u_m (field of u_m) and grad phi(r; w_s, u_m) (force on w_s)
        if (r2 > R(0))
            dipole<R>(rx, ry, rz, r2, w.x, w.y, w.z, um.x, um.y, um.z, gx, gy, gz, qx, qy, qz);
    }
    gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz);
    qx = warp_sum(qx); qy = warp_sum(qy); qz = warp_sum(qz);
    if (lane == 0) {
        double* o = part + 6 * it;
        o[0] = gx; o[1] = gy; o[2] = gz;
        o[3] = qx; o[4] = qy; o[5] = qz;
    }
}

// One thread per source: its items' partials added in order in FP64.
template <typename R>
__global__ void k_item_reduce(Tree<R> t, int64_t ncells, int64_t nsrc,
                              const uint32_t* __restrict__ item_off,
                              const double* __restrict__ part, double* __restrict__ G,
                              double* __restrict__ Q)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsrc) return;
    double g[3] = {0.0, 0.0, 0.0}, q[3] = {0.0, 0.0, 0.0};
    for (uint32_t it = item_off[s]; it < item_off[s + 1]; ++it) {
        const double* o = part + 6 * (int64_t)it;
        g[0] += o[0]; g[1] += o[1]; g[2] += o[2];
        q[0] += o[3]; q[1] += o[4]; q[2] += o[5];
    }
    double ns = 1.0;
    if (s < ncells) {
        const int4 nd = t.cell[s].node;
        ns = (double)(nd.y - nd.x);
    }
    for (int a = 0; a < 3; ++a) {
        G[3 * s + a] = g[a];
        Q[3 * s + a] = q[a] / ns;
    }
}

// One warp per item of the general vector-Jacobian product (see
// vjp_source_sums): six single-precision sums per item, written in FP64.
template <typename R>
__global__ void __launch_bounds__(kGradThreads) k_vjp_item_sums(
    const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ u,
    const vec4<R>* __restrict__ abar, const vec4<R>* __restrict__ bbar, R ds, Tree<R> t,
    int64_t ncells, int64_t nsrc, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ beg, const uint32_t* __restrict__ end,
    const uint32_t* __restrict__ item_off, const uint32_t* __restrict__ item_src,
    double* __restrict__ part)
{
    const int64_t it = ((int64_t)blockIdx.x * kGradThreads + threadIdx.x) >> 5;
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
    const uint32_t b = beg[s] + (uint32_t)(it - item_off[s]) * (uint32_t)kGradItemEntries;
    const uint32_t e = min(end[s], b + (uint32_t)kGradItemEntries);
    const uint32_t np = (uint32_t)(nsrc - ncells);
    R gx = 0, gy = 0, gz = 0, qx = 0, qy = 0, qz = 0;
    for (uint32_t k = b + lane; k < e; k += 32) {
        const uint32_t m = vals[k];
        if (m >= np) continue;  // only after a flagged recording walk
        const vec4<R> xm = pos[m], um = u[m], am = abar[m], bm = bbar[m];
        const R rx = xm.x - x.x, ry = xm.y - x.y, rz = xm.z - x.z;
        const R r2 = rx * rx + ry * ry + rz * rz;
        if (!(r2 > R(0))) continue;
        const PairGeo<R> g = pair_geo<R>(rx, ry, rz, r2);
        // dL/dw_s: T(r) abar_m + grad phi(r; bbar_m, u_m)
        t_apply_add<R>(g, am.x, am.y, am.z, R(1), gx, gy, gz);
        grad_phi_add<R>(g, bm.x, bm.y, bm.z, um.x, um.y, um.z, R(1), gx, gy, gz);
        // dL/dx_s: -(grad phi(r; abar_m, w_s) + H phi(r; u_m, w_s) bbar_m)
        grad_phi_add<R>(g, am.x, am.y, am.z, w.x, w.y, w.z, R(-1), qx, qy, qz);
        hess_phi_add<R>(g, um.x, um.y, um.z, w.x, w.y, w.z, bm.x, bm.y, bm.z, R(-1), qx, qy, qz);
    }
    gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz);
    qx = warp_sum(qx); qy = warp_sum(qy); qz = warp_sum(qz);
    if (lane == 0) {
        double* o = part + 6 * it;
        o[0] = (double)gx * (double)ds; o[1] = (double)gy * (double)ds; o[2] = (double)gz * (double)ds;
        o[3] = (double)qx * (double)ds; o[4] = (double)qy * (double)ds; o[5] = (double)qz * (double)ds;
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

void grad_segments(const uint32_t* keys, int64_t ne, int64_t nsrc, uint32_t* beg, uint32_t* end,
                   cudaStream_t s)
{
    cudaMemsetAsync(beg, 0, sizeof(uint32_t) * nsrc, s);
    cudaMemsetAsync(end, 0, sizeof(uint32_t) * nsrc, s);
    if (ne <= 0) return;
    k_segments<<<blocks((ne + 3) / 4, kGradThreads), kGradThreads, 0, s>>>(keys, ne, nsrc, beg,
                                                                          end);
    counted();
}

template <typename R>
void grad_source_sums(const vec4<R>* pos, const vec4<R>* u, Tree<R> t, int64_t ncells, int64_t n,
                      const uint32_t* vals, const uint32_t* beg, const uint32_t* end,
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
    k_item_sums<R><<<blocks(max_items * 32, kGradThreads), kGradThreads, 0, s>>>(
        pos, u, t, ncells, nsrc, vals, beg, end, item_off, item_src, part);
    k_item_reduce<R><<<blocks(nsrc, kGradThreads), kGradThreads, 0, s>>>(t, ncells, nsrc, item_off,
                                                                       part, G, Q);
    counted(4);
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
void vjp_source_sums(const vec4<R>* pos, const vec4<R>* u, const vec4<R>* abar,
                     const vec4<R>* bbar, R ds, Tree<R> t, int64_t ncells, int64_t n,
                     const uint32_t* vals, const uint32_t* beg, const uint32_t* end,
                     uint32_t* items, uint32_t* item_off, uint32_t* scan_tmp, double* part,
                     int64_t max_items, double* G, double* Q, cudaStream_t s)
{
    const int64_t nsrc = ncells + n;
    if (nsrc <= 0) return;
    k_item_counts<<<blocks(nsrc, kGradThreads), kGradThreads, 0, s>>>(beg, end, nsrc, items);
    scan_exclusive(items, item_off, nsrc, scan_tmp, s);
    uint32_t* item_src = reinterpret_cast<uint32_t*>(part + 6 * max_items);
    k_item_sources<<<blocks(nsrc, kGradThreads), kGradThreads, 0, s>>>(item_off, nsrc, item_src);
    k_vjp_item_sums<R><<<blocks(max_items * 32, kGradThreads), kGradThreads, 0, s>>>(
        pos, u, abar, bbar, ds, t, ncells, nsrc, vals, beg, end, item_off, item_src, part);
    k_item_reduce<R><<<blocks(nsrc, kGradThreads), kGradThreads, 0, s>>>(t, ncells, nsrc, item_off,
                                                                       part, G, Q);
    counted(4);
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
    template void vjp_source_sums<R>(const vec4<R>*, const vec4<R>*, const vec4<R>*,              \
                                     const vec4<R>*, R, Tree<R>, int64_t, int64_t,               \
                                     const uint32_t*, const uint32_t*, const uint32_t*,           \
                                     uint32_t*, uint32_t*, uint32_t*, double*, int64_t, double*,  \
                                     double*, cudaStream_t);                                     \
    template void vjp_finish<R>(Tree<R>, int64_t, int64_t, const double*, const double*,          \
                                const vec4<R>*, const vec4<R>*, vec4<R>*, vec4<R>*, cudaStream_t);\
    template void scatter_records<R>(const uint32_t*, int64_t, const vec4<R>*, vec4<R>*,          \
                                     cudaStream_t);                                               \
    template void sum_z<R>(const vec4<R>*, int64_t, double*, double*, cudaStream_t);              \
    template void grad_from_field<R>(const vec4<R>*, const vec4<R>*, int64_t, vec4<R>*, vec4<R>*, \
                                     cudaStream_t);                                               \
    template void grad_source_sums<R>(const vec4<R>*, const vec4<R>*, Tree<R>, int64_t, int64_t,  \
                                      const uint32_t*, const uint32_t*, const uint32_t*,          \
                                      uint32_t*, uint32_t*, uint32_t*, double*, int64_t, double*, \
                                      double*, cudaStream_t);                                    \
    template void grad_finish<R>(Tree<R>, int64_t, int64_t, const double*, const double*,         \
                                 const vec4<R>*, const vec4<R>*, R, vec4<R>*, vec4<R>*,           \
                                 cudaStream_t);
FFK_GRAD_INST(float)
FFK_GRAD_INST(double)
#undef FFK_GRAD_INST

}  // namespace ffk
