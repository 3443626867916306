// Integration step (Sec. 4, Euler-Maruyama with the reduced Langevin
// equations of Sec. 2; kernel 6 of the paper's scheme), thermal noise from
// a counter-based generator, FP64 observables (Sec. 5), and the layout
// conversions between the caller's n x 3 arrays and the 16/32-byte records.
#include "ffk.cuh"

namespace ffk {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStepThreads = 256;

// Philox4x32 with ten rounds (Salmon, Moraes, Dror, Shaw, SC'11): each round
// multiplies words 0 and 2 by fixed odd constants and mixes the high halves
// with the other words and the round key; the key advances by the Weyl
// increments between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Box-Muller on one pair of words: u1 = (a + 1) 2^-32 in (0, 1],
// u2 = b 2^-32; z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = ... sin(2 pi u2).
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1)
{
    const float u1 = __fmaf_rn(__uint2float_rn(a), 0x1p-32f, 0x1p-32f);
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(__uint2float_rn(b) * 0x1p-31f, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& z0, double& z1)
{
    const double u1 = ((double)a + 1.0) * 0x1p-32;
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi((double)b * 0x1p-31, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

// Six normals for (seed, step, id): counter (step lo, step hi, id, block).
template <typename R>
__device__ __forceinline__ void normals6(const DynParams<R>& dp, uint32_t id, R z[6])
{
    const unsigned long long st = *dp.step;
    const uint32_t c0 = (uint32_t)st, c1 = (uint32_t)(st >> 32);
    const uint4 w0 = philox10(make_uint4(c0, c1, id, 0u), dp.key0, dp.key1);
    const uint4 w1 = philox10(make_uint4(c0, c1, id, 1u), dp.key0, dp.key1);
    box_muller(w0.x, w0.y, z[0], z[1]);
    box_muller(w0.z, w0.w, z[2], z[3]);
    box_muller(w1.x, w1.y, z[4], z[5]);
}

// LJ-type wall along one axis: distance w to the plane, sigma_w = 1/2, cut
// where the force vanishes (w = 1/2), w clamped below at 0.01.
template <typename R>
__device__ __forceinline__ R wall_force(R w, const DynParams<R>& dp, R& e)
{
    if (!(w < R(0.5))) return R(0);
    if (w < R(0.01)) w = R(0.01);
    const R s = R(0.5) / w;
    const R s2 = s * s;
    const R s6 = s2 * s2 * s2;
    e += dp.wall_e2 * s6 * s6 - dp.wall_e4 * s6 + dp.wall_e2;
    return dp.wall_eps24 * (s6 * s6 - s6) / w;
}

// Wall planes and applied field of the system owning position s.
template <typename R>
struct Local {
    R lo[3], hi[3], hx, hy, hz;
    int sys;
};

template <typename R>
__device__ __forceinline__ Local<R> local_of(const DynParams<R>& dp, int64_t s)
{
    Local<R> L;
    if (dp.sys_of_pos) {
        L.sys = (int)dp.sys_of_pos[s];
        const vec4<R> a = dp.sys_lo[L.sys], b = dp.sys_hi[L.sys], h = dp.sys_h[L.sys];
        L.lo[0] = a.x; L.lo[1] = a.y; L.lo[2] = a.z;
        L.hi[0] = b.x; L.hi[1] = b.y; L.hi[2] = b.z;
        L.hx = h.x; L.hy = h.y; L.hz = h.z;
    } else {
        L.sys = -1;
        for (int q = 0; q < 3; ++q) {
            L.lo[q] = dp.lo[q];
            L.hi[q] = dp.hi[q];
        }
        L.hx = dp.hx; L.hy = dp.hy; L.hz = dp.hz;
    }
    return L;
}

template <typename R>
__device__ __forceinline__ void walls3(const DynParams<R>& dp, const Local<R>& L, const vec4<R>& x,
                                       R& fx, R& fy, R& fz, R& e)
{
    if (!dp.walls) return;
    fx += wall_force<R>(x.x - L.lo[0], dp, e) - wall_force<R>(L.hi[0] - x.x, dp, e);
    fy += wall_force<R>(x.y - L.lo[1], dp, e) - wall_force<R>(L.hi[1] - x.y, dp, e);
    fz += wall_force<R>(x.z - L.lo[2], dp, e) - wall_force<R>(L.hi[2] - x.z, dp, e);
}

// Adds u and h_dip_z of one particle to its system's sums (warp-aggregated
// when every active lane belongs to the same system).
template <typename R>
__device__ __forceinline__ void system_acc(const DynParams<R>& dp, int sys, const vec4<R>& uu,
                                           R hdz)
{
    const unsigned am = __activemask();
    const int s0 = __shfl_sync(am, sys, __ffs(am) - 1);
    R v[4] = {uu.x, uu.y, uu.z, hdz};
    if (am == kFull && __all_sync(kFull, sys == s0)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(kFull, v[q], o);
        }
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) atomicAdd(&dp.sys_acc[4 * sys + q], (double)v[q]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(&dp.sys_acc[4 * sys + q], (double)v[q]);
    }
}

// Block sum of kObs per-thread values: warp sums in the arithmetic type R
// (32 terms), then the warp sums in FP64 in a fixed order; thread q < kObs
// writes quantity q.  Cancellation in the global sums (magnetisation,
// energies of a million particles) happens in FP64.
template <typename R>
__device__ __forceinline__ void block_sum_obs(R v[kObs], double* out)
{
    __shared__ double sh[kStepThreads / 32][kObs];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kObs; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(kFull, v[q], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < kObs; ++q) sh[w][q] = (double)v[q];
    }
    __syncthreads();
    if (threadIdx.x < kObs) {
        double s = 0.0;
        for (int ww = 0; ww < kStepThreads / 32; ++ww) s += sh[ww][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Accumulates one particle's terms: e_dip, e_zeeman, e_sr, e_wall, e_kin_t,
// w^2 (scaled by I/2 later), u (3), h_dip_z.
template <typename R>
__device__ __forceinline__ void obs_terms(R v[kObs], const Local<R>& L, const vec4<R>& uu,
                                          const vec4<R>& hd, const vec4<R>& vv, const vec4<R>& w,
                                          R es, R ew)
{
    v[0] += R(-0.5) * (uu.x * hd.x + uu.y * hd.y + uu.z * hd.z);
    v[1] += -(uu.x * L.hx + uu.y * L.hy + uu.z * L.hz);
    v[2] += es;
    v[3] += ew;
    v[4] += R(0.5) * (vv.x * vv.x + vv.y * vv.y + vv.z * vv.z);
    v[5] += w.x * w.x + w.y * w.y + w.z * w.z;
    v[6] += uu.x;
    v[7] += uu.y;
    v[8] += uu.z;
    v[9] += hd.z;
}

// x' = x + dt v; v' = v + dt (f - G_t v) + sig_t xi_t;
// w' = w + dt (u x h - G_r w) / I + sig_r xi_r; u' = normalise(u + dt w x u).
template <typename R, bool OBS>
__global__ void __launch_bounds__(kStepThreads) k_integrate(
    int64_t n, const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ vel,
    const vec4<R>* __restrict__ u, const vec4<R>* __restrict__ om, const uint32_t* __restrict__ id,
    const vec4<R>* __restrict__ hdip, const vec4<R>* __restrict__ fint, const R* __restrict__ esr,
    DynParams<R> dp, vec4<R>* __restrict__ pos2, vec4<R>* __restrict__ vel2,
    vec4<R>* __restrict__ u2, vec4<R>* __restrict__ om2, uint32_t* __restrict__ id2,
    double* __restrict__ partials)
{
    R v[kObs];
#pragma unroll
    for (int q = 0; q < kObs; ++q) v[q] = R(0);
    // the tree of this step did not fit: no field was formed, the state is kept as it is
    const bool hold = dp.flags && (*dp.flags & FLAG_CAPACITY);
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        if (hold) {
            pos2[s] = pos[s];
            vel2[s] = vel[s];
            u2[s] = u[s];
            om2[s] = om[s];
            id2[s] = id[s];
            continue;
        }
        const vec4<R> x = pos[s], vv = vel[s], uu = u[s], w = om[s], hd = hdip[s], fi = fint[s];
        const uint32_t pid = id[s];
        const Local<R> L = local_of<R>(dp, s);
        R ew = R(0);
        R fx = fi.x, fy = fi.y, fz = fi.z;
        walls3<R>(dp, L, x, fx, fy, fz, ew);
        const R hx = hd.x + L.hx, hy = hd.y + L.hy, hz = hd.z + L.hz;
        R z[6];
        normals6<R>(dp, pid, z);
        const R tx = uu.y * hz - uu.z * hy, ty = uu.z * hx - uu.x * hz, tz = uu.x * hy - uu.y * hx;
        const R cx = w.y * uu.z - w.z * uu.y, cy = w.z * uu.x - w.x * uu.z,
                cz = w.x * uu.y - w.y * uu.x;
        vec4<R> xn, vn, wn, un;
        xn.x = x.x + dp.dt * vv.x;
        xn.y = x.y + dp.dt * vv.y;
        xn.z = x.z + dp.dt * vv.z;
        xn.w = x.w;
        vn.x = vv.x + dp.dt * (fx - dp.gamma_t * vv.x) + dp.sig_t * z[0];
        vn.y = vv.y + dp.dt * (fy - dp.gamma_t * vv.y) + dp.sig_t * z[1];
        vn.z = vv.z + dp.dt * (fz - dp.gamma_t * vv.z) + dp.sig_t * z[2];
        vn.w = R(0);
        wn.x = w.x + dp.dt * (tx - dp.gamma_r * w.x) * dp.inv_inertia + dp.sig_r * z[3];
        wn.y = w.y + dp.dt * (ty - dp.gamma_r * w.y) * dp.inv_inertia + dp.sig_r * z[4];
        wn.z = w.z + dp.dt * (tz - dp.gamma_r * w.z) * dp.inv_inertia + dp.sig_r * z[5];
        wn.w = R(0);
        const R ax = uu.x + dp.dt * cx, ay = uu.y + dp.dt * cy, az = uu.z + dp.dt * cz;
        const R inv = R(1) / sqrt(ax * ax + ay * ay + az * az);
        un.x = ax * inv;
        un.y = ay * inv;
        un.z = az * inv;
        un.w = R(0);
        if (dp.printed_angles) {
            // the printed reduced angle equations: theta, phi from u, their rates in
            // w_x, w_y; angles moved by the rates, rates by the printed torques
            const R uz = uu.z < R(-1) ? R(-1) : (uu.z > R(1) ? R(1) : uu.z);
            const R th = acos(uz), ph = atan2(uu.y, uu.x);
            const R tt = uu.x * hy - uu.y * hx;
            const R tp = -(uu.y * hz - uu.z * hy) * sin(ph) + (uu.z * hx - uu.x * hz) * cos(ph);
            const R th2 = th + dp.dt * w.x, ph2 = ph + dp.dt * w.y;
            wn.x = w.x + dp.dt * (tt - dp.gamma_r * w.x) * dp.inv_inertia + dp.sig_r * z[3];
            wn.y = w.y + dp.dt * (tp - dp.gamma_r * w.y) * dp.inv_inertia + dp.sig_r * z[4];
            wn.z = R(0);
            un.x = sin(th2) * cos(ph2);
            un.y = sin(th2) * sin(ph2);
            un.z = cos(th2);
        }
        pos2[s] = xn;
        vel2[s] = vn;
        u2[s] = un;
        om2[s] = wn;
        id2[s] = pid;
        if (OBS) obs_terms<R>(v, L, uu, hd, vv, w, esr ? esr[s] : R(0), ew);
        if (dp.sys_acc) system_acc<R>(dp, L.sys, uu, hd.z);
    }
    if (OBS) block_sum_obs<R>(v, partials + (int64_t)blockIdx.x * kObs);
}

template <typename R>
__global__ void __launch_bounds__(kStepThreads) k_observables(
    int64_t n, const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ vel,
    const vec4<R>* __restrict__ u, const vec4<R>* __restrict__ om,
    const vec4<R>* __restrict__ hdip, const R* __restrict__ esr, DynParams<R> dp,
    double* __restrict__ partials)
{
    R v[kObs];
#pragma unroll
    for (int q = 0; q < kObs; ++q) v[q] = R(0);
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const vec4<R> x = pos[s];
        const Local<R> L = local_of<R>(dp, s);
        R ew = R(0);
        R fx = 0, fy = 0, fz = 0;
        walls3<R>(dp, L, x, fx, fy, fz, ew);
        obs_terms<R>(v, L, u[s], hdip[s], vel[s], om[s], esr ? esr[s] : R(0), ew);
    }
    block_sum_obs<R>(v, partials + (int64_t)blockIdx.x * kObs);
}

// Deterministic final sum: one block per quantity; thread t adds partials
// t, t + 256, ... in order, then a fixed-shape tree combines the threads.
__global__ void __launch_bounds__(kStepThreads) k_reduce_partials(
    const double* __restrict__ partials, int nblocks, double inv_n, double inertia_half,
    double* __restrict__ out)
{
    __shared__ double sh[kStepThreads];
    const int q = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kStepThreads) s += partials[(int64_t)b * kObs + q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = kStepThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double v = sh[0];
        if (q == 5) v *= inertia_half;
        if (q >= 6) v *= inv_n;
        out[q] = v;
    }
}

__global__ void k_step_advance(unsigned long long* step, const int* flags)
{
    if (flags && (*flags & FLAG_CAPACITY)) return;
    *step += 1ull;
}

template <typename R, typename I>
__global__ void k_load3(const I* __restrict__ in, int64_t n, vec4<R>* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vec4<R> v;
    v.x = (R)in[3 * i];
    v.y = (R)in[3 * i + 1];
    v.z = (R)in[3 * i + 2];
    v.w = R(0);
    out[i] = v;
}

template <typename R>
__global__ void k_zero4(vec4<R>* __restrict__ out, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vec4<R> v;
    v.x = v.y = v.z = v.w = R(0);
    out[i] = v;
}

__global__ void k_iota(uint32_t* __restrict__ out, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint32_t)i;
}

template <typename R, typename O>
__global__ void k_scatter3(const vec4<R>* __restrict__ in, const uint32_t* __restrict__ id,
                           int64_t n, O* __restrict__ out)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const vec4<R> v = in[s];
    const int64_t d = id[s];
    out[3 * d] = (O)v.x;
    out[3 * d + 1] = (O)v.y;
    out[3 * d + 2] = (O)v.z;
}

__global__ void k_scatter_counts(const int4* __restrict__ in, const uint32_t* __restrict__ id,
                                 int64_t n, int32_t* a, int32_t* p, int32_t* o)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int4 v = in[s];
    const int64_t d = id[s];
    if (a) a[d] = v.x;
    if (p) p[d] = v.y;
    if (o) o[d] = v.z;
}

// dF/dw of wall_force (zero where the force is cut or w is clamped)
template <typename R>
__device__ __forceinline__ R wall_dforce(R w, const DynParams<R>& dp)
{
    if (!(w < R(0.5))) return R(0);
    if (w < R(0.01)) return R(0);
    const R s = R(0.5) / w;
    const R s2 = s * s;
    const R s6 = s2 * s2 * s2;
    return dp.wall_eps24 * (R(7) * s6 - R(13) * s6 * s6) / (w * w);
}

// Adjoint of one step of k_integrate for each particle.  In: the step's input
// state, its dipolar field, and the adjoints of the step's outputs in
// xb, vb, ub, wb (add_uz is first added to ub.z: the mean-magnetisation term
// of the output state).  Out: the adjoints of the inputs, without the field's
// and force's own dependence on positions and moments; the cotangents abar of
// h_dip and bbar of the interaction force; per-block FP64 sums of abar (the
// cotangent of the applied field) in partials[3 * block + q].
//   u' = a / |a|, a = u + dt w x u:  aa = (ub' - u'(u'.ub')) / |a|
//        ub = aa - dt w x aa;  wb = dt u x aa
//   w' = w + dt (u x h - Gr w) / I:  wb += (1 - dt Gr / I) wb';  ub += dt/I h x wb'
//        abar = dt/I wb' x u
//   v' = v + dt (f - Gt v):         vb = (1 - dt Gt) vb' + dt xb';  bbar = dt vb'
//   x' = x + dt v:                   xb = xb' + bbar . (walls' dF/dx)
template <typename R>
__global__ void __launch_bounds__(kStepThreads) k_em_adjoint(
    int64_t n, const vec4<R>* __restrict__ pos, const vec4<R>* __restrict__ u,
    const vec4<R>* __restrict__ om, const vec4<R>* __restrict__ hdip, DynParams<R> dp, R add_uz,
    vec4<R>* __restrict__ xb, vec4<R>* __restrict__ vb, vec4<R>* __restrict__ ub,
    vec4<R>* __restrict__ wb, vec4<R>* __restrict__ abar, vec4<R>* __restrict__ bbar,
    double* __restrict__ partials)
{
    __shared__ double sh[kStepThreads / 32][3];
    R hs[3] = {R(0), R(0), R(0)};
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const vec4<R> x = pos[s], uu = u[s], w = om[s], hd = hdip[s];
        const Local<R> L = local_of<R>(dp, s);
        const R hx = hd.x + L.hx, hy = hd.y + L.hy, hz = hd.z + L.hz;
        const vec4<R> X = xb[s], V = vb[s], W = wb[s];
        vec4<R> U = ub[s];
        U.z += add_uz;
        const R dt = dp.dt;
        const R cx = w.y * uu.z - w.z * uu.y, cy = w.z * uu.x - w.x * uu.z,
                cz = w.x * uu.y - w.y * uu.x;
        const R ax = uu.x + dt * cx, ay = uu.y + dt * cy, az = uu.z + dt * cz;
        const R il = R(1) / sqrt(ax * ax + ay * ay + az * az);
        const R nx = ax * il, ny = ay * il, nz = az * il;
        const R pr = nx * U.x + ny * U.y + nz * U.z;
        const R qx = (U.x - nx * pr) * il, qy = (U.y - ny * pr) * il, qz = (U.z - nz * pr) * il;
        const R ci = dt * dp.inv_inertia;
        vec4<R> oX, oV, oU, oW, oa, ob;
        oU.x = qx - dt * (w.y * qz - w.z * qy) + ci * (hy * W.z - hz * W.y);
        oU.y = qy - dt * (w.z * qx - w.x * qz) + ci * (hz * W.x - hx * W.z);
        oU.z = qz - dt * (w.x * qy - w.y * qx) + ci * (hx * W.y - hy * W.x);
        oU.w = R(0);
        const R fr = R(1) - ci * dp.gamma_r;
        oW.x = dt * (uu.y * qz - uu.z * qy) + fr * W.x;
        oW.y = dt * (uu.z * qx - uu.x * qz) + fr * W.y;
        oW.z = dt * (uu.x * qy - uu.y * qx) + fr * W.z;
        oW.w = R(0);
        oa.x = ci * (W.y * uu.z - W.z * uu.y);
        oa.y = ci * (W.z * uu.x - W.x * uu.z);
        oa.z = ci * (W.x * uu.y - W.y * uu.x);
        oa.w = R(0);
        const R ft = R(1) - dt * dp.gamma_t;
        oV.x = ft * V.x + dt * X.x;
        oV.y = ft * V.y + dt * X.y;
        oV.z = ft * V.z + dt * X.z;
        oV.w = R(0);
        ob.x = dt * V.x;
        ob.y = dt * V.y;
        ob.z = dt * V.z;
        ob.w = R(0);
        oX = X;
        if (dp.walls) {
            oX.x += ob.x * (wall_dforce<R>(x.x - L.lo[0], dp) + wall_dforce<R>(L.hi[0] - x.x, dp));
            oX.y += ob.y * (wall_dforce<R>(x.y - L.lo[1], dp) + wall_dforce<R>(L.hi[1] - x.y, dp));
            oX.z += ob.z * (wall_dforce<R>(x.z - L.lo[2], dp) + wall_dforce<R>(L.hi[2] - x.z, dp));
        }
        xb[s] = oX;
        vb[s] = oV;
        ub[s] = oU;
        wb[s] = oW;
        abar[s] = oa;
        bbar[s] = ob;
        hs[0] += oa.x;
        hs[1] += oa.y;
        hs[2] += oa.z;
    }
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double v = (double)hs[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) sh[wi][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int k = 0; k < kStepThreads / 32; ++k) t += sh[k][threadIdx.x];
        partials[3 * (int64_t)blockIdx.x + threadIdx.x] = t;
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int integrate_blocks(int64_t n)
{
    // one particle per thread up to 2^16 blocks (16.7 M particles), grid-stride beyond
    int64_t b = (n + kStepThreads - 1) / kStepThreads;
    if (b > 65536) b = 65536;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename R>
void integrate(int64_t n, const vec4<R>* pos, const vec4<R>* vel, const vec4<R>* u,
               const vec4<R>* om, const uint32_t* id, const vec4<R>* h, const vec4<R>* f,
               const R* esr, DynParams<R> dp, vec4<R>* pos2, vec4<R>* vel2, vec4<R>* u2,
               vec4<R>* om2, uint32_t* id2, double* partials, cudaStream_t s)
{
    const int g = integrate_blocks(n);
    if (partials)
        k_integrate<R, true><<<g, kStepThreads, 0, s>>>(n, pos, vel, u, om, id, h, f, esr, dp, pos2,
                                                        vel2, u2, om2, id2, partials);
    else
        k_integrate<R, false><<<g, kStepThreads, 0, s>>>(n, pos, vel, u, om, id, h, f, esr, dp,
                                                         pos2, vel2, u2, om2, id2, partials);
    counted();
}

template <typename R>
void em_adjoint(int64_t n, const vec4<R>* pos, const vec4<R>* u, const vec4<R>* om,
                const vec4<R>* hdip, DynParams<R> dp, R add_uz, vec4<R>* xb, vec4<R>* vb,
                vec4<R>* ub, vec4<R>* wb, vec4<R>* abar, vec4<R>* bbar, double* partials,
                cudaStream_t s)
{
    k_em_adjoint<R><<<integrate_blocks(n), kStepThreads, 0, s>>>(n, pos, u, om, hdip, dp, add_uz,
                                                                 xb, vb, ub, wb, abar, bbar,
                                                                 partials);
    counted();
}

template <typename R>
void observables(int64_t n, const vec4<R>* pos, const vec4<R>* vel, const vec4<R>* u,
                 const vec4<R>* om, const vec4<R>* h, const R* esr, DynParams<R> dp,
                 double* partials, cudaStream_t s)
{
    k_observables<R><<<integrate_blocks(n), kStepThreads, 0, s>>>(n, pos, vel, u, om, h, esr, dp,
                                                                  partials);
    counted();
}

void reduce_partials(const double* partials, int nblocks, double inv_n, double inertia_half,
                     double* out, cudaStream_t s)
{
    k_reduce_partials<<<kObs, kStepThreads, 0, s>>>(partials, nblocks, inv_n, inertia_half, out);
    counted();
}

void step_advance(unsigned long long* step, const int* flags, cudaStream_t s)
{
    k_step_advance<<<1, 1, 0, s>>>(step, flags);
    counted();
}

namespace {
__global__ void k_step_set(unsigned long long* step, unsigned long long v) { *step = v; }
}  // namespace

void step_set(unsigned long long* step, unsigned long long v, cudaStream_t s)
{
    k_step_set<<<1, 1, 0, s>>>(step, v);
    counted();
}

template <typename R, typename I>
void load3(const I* in, int64_t n, vec4<R>* out, cudaStream_t s)
{
    k_load3<R, I><<<nblk(n, 256), 256, 0, s>>>(in, n, out);
    counted();
}

template <typename R>
void fill_zero4(vec4<R>* out, int64_t n, cudaStream_t s)
{
    k_zero4<R><<<nblk(n, 256), 256, 0, s>>>(out, n);
    counted();
}

void iota32(uint32_t* out, int64_t n, cudaStream_t s)
{
    k_iota<<<nblk(n, 256), 256, 0, s>>>(out, n);
    counted();
}

template <typename R, typename O>
void scatter3(const vec4<R>* in, const uint32_t* id, int64_t n, O* out, cudaStream_t s)
{
    k_scatter3<R, O><<<nblk(n, 256), 256, 0, s>>>(in, id, n, out);
    counted();
}

template <typename R>
void scatter_counts(const int4* in, const uint32_t* id, int64_t n, int32_t* a, int32_t* p,
                    int32_t* o, cudaStream_t s)
{
    k_scatter_counts<<<nblk(n, 256), 256, 0, s>>>(in, id, n, a, p, o);
    counted();
}

#define FFK_INST(R)                                                                             \
    template void integrate<R>(int64_t, const vec4<R>*, const vec4<R>*, const vec4<R>*,          \
                               const vec4<R>*, const uint32_t*, const vec4<R>*, const vec4<R>*,  \
                               const R*, DynParams<R>, vec4<R>*, vec4<R>*, vec4<R>*, vec4<R>*,   \
                               uint32_t*, double*, cudaStream_t);                               \
    template void em_adjoint<R>(int64_t, const vec4<R>*, const vec4<R>*, const vec4<R>*,          \
                                const vec4<R>*, DynParams<R>, R, vec4<R>*, vec4<R>*, vec4<R>*,    \
                                vec4<R>*, vec4<R>*, vec4<R>*, double*, cudaStream_t);            \
    template void observables<R>(int64_t, const vec4<R>*, const vec4<R>*, const vec4<R>*,        \
                                 const vec4<R>*, const vec4<R>*, const R*, DynParams<R>,         \
                                 double*, cudaStream_t);                                        \
    template void load3<R, float>(const float*, int64_t, vec4<R>*, cudaStream_t);               \
    template void load3<R, double>(const double*, int64_t, vec4<R>*, cudaStream_t);             \
    template void fill_zero4<R>(vec4<R>*, int64_t, cudaStream_t);                               \
    template void scatter3<R, float>(const vec4<R>*, const uint32_t*, int64_t, float*,           \
                                     cudaStream_t);                                             \
    template void scatter3<R, double>(const vec4<R>*, const uint32_t*, int64_t, double*,         \
                                      cudaStream_t);                                            \
    template void scatter_counts<R>(const int4*, const uint32_t*, int64_t, int32_t*, int32_t*,   \
                                    int32_t*, cudaStream_t);
FFK_INST(float)
FFK_INST(double)
#undef FFK_INST

}  // namespace ffk
