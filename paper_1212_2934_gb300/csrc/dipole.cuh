// The reduced dipole pair kernel shared by the field traversal and the
// gradient pass (Sec. 2, reduced Eqs. h_dip and f_dip).
#pragma once

#include "ffk.cuh"

namespace ffk {

__device__ __forceinline__ float dip_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double dip_rsqrt(double x) { return rsqrt(x); }

// Reduced dipolar field of u_j and force on u_k at separation r = rho_k - rho_j
// (Sec. 2, reduced Eqs. h_dip and f_dip), accumulated:
//   h += [3 r (u_j.r) - u_j r^2] / r^5
//   f += 3 [r (u_j.u_k) + u_k (u_j.r) + u_j (u_k.r)] / r^5 - 15 r (u_k.r)(u_j.r) / r^7
template <typename R>
__device__ __forceinline__ void dipole(R rx, R ry, R rz, R r2, R ukx, R uky, R ukz, R ujx, R ujy,
                                       R ujz, R& hx, R& hy, R& hz, R& fx, R& fy, R& fz)
{
    const R ir = dip_rsqrt(r2);
    const R ir2 = ir * ir;
    const R ir3 = ir2 * ir;
    const R ir5 = ir3 * ir2;
    const R ir7 = ir5 * ir2;
    const R bj = ujx * rx + ujy * ry + ujz * rz;
    const R bk = ukx * rx + uky * ry + ukz * rz;
    const R a = ujx * ukx + ujy * uky + ujz * ukz;
    const R s3 = R(3) * ir5;
    const R cuk = s3 * bj, cuj = s3 * bk;  // cuk = 3 (u_j.r) / r^5 serves h and f
    hx += rx * cuk - ujx * ir3;
    hy += ry * cuk - ujy * ir3;
    hz += rz * cuk - ujz * ir3;
    const R cr = s3 * a - R(15) * bk * bj * ir7;
    fx += rx * cr + ukx * cuk + ujx * cuj;
    fy += ry * cr + uky * cuk + ujy * cuj;
    fz += rz * cr + ukz * cuk + ujz * cuj;
}

// The same terms with u_k's part of the force kept as one scalar: adds
//   h += r cuk - u_j / r^3,   f += r cr + u_j cuj,   c += cuk,
// cuk = 3 (u_j.r) / r^5, cuj = 3 (u_k.r) / r^5, cr = 3 (u_j.u_k) / r^5 - 15 (u_k.r)(u_j.r) / r^7,
// so that the force on u_k is f + u_k c once every source has been added (u_k
// is the same for all of them).  A pair at r2 = 0 adds nothing.
template <typename R>
__device__ __forceinline__ void dipole_acc(R rx, R ry, R rz, R r2, R ukx, R uky, R ukz, R ujx,
                                           R ujy, R ujz, R& hx, R& hy, R& hz, R& fx, R& fy,
                                           R& fz, R& c)
{
    const R ir = r2 > R(0) ? dip_rsqrt(r2) : R(0);
    const R ir2 = ir * ir;
    const R ir3 = ir2 * ir;
    const R ir5 = ir3 * ir2;
    const R ir7 = ir5 * ir2;
    const R bj = ujx * rx + ujy * ry + ujz * rz;
    const R bk = ukx * rx + uky * ry + ukz * rz;
    const R a = ujx * ukx + ujy * uky + ujz * ukz;
    const R s3 = R(3) * ir5;
    const R cuk = s3 * bj, cuj = s3 * bk;
    hx += rx * cuk;
    hy += ry * cuk;
    hz += rz * cuk;
    hx -= ujx * ir3;
    hy -= ujy * ir3;
    hz -= ujz * ir3;
    const R cr = s3 * a - R(15) * bk * bj * ir7;
    fx += rx * cr;
    fy += ry * cr;
    fz += rz * cr;
    fx += ujx * cuj;
    fy += ujy * cuj;
    fz += ujz * cuj;
    c += cuk;
}

// The traversal's pair terms: FP64 takes the form above with u_k factored out
// (fewer FP64 operations, the scarce ones on this part); FP32 keeps dipole(),
// whose extra operations measured no slower than the accumulator they save.
// A pair at r2 = 0 adds nothing in either.
__device__ __forceinline__ void walk_pair(float rx, float ry, float rz, float r2, float ukx,
                                          float uky, float ukz, float ujx, float ujy, float ujz,
                                          float& hx, float& hy, float& hz, float& fx, float& fy,
                                          float& fz, float&)
{
    if (r2 > 0.0f) dipole<float>(rx, ry, rz, r2, ukx, uky, ukz, ujx, ujy, ujz, hx, hy, hz, fx, fy, fz);
}

__device__ __forceinline__ void walk_pair(double rx, double ry, double rz, double r2, double ukx,
                                          double uky, double ukz, double ujx, double ujy,
                                          double ujz, double& hx, double& hy, double& hz,
                                          double& fx, double& fy, double& fz, double& c)
{
    dipole_acc<double>(rx, ry, rz, r2, ukx, uky, ukz, ujx, ujy, ujz, hx, hy, hz, fx, fy, fz, c);
}

// Inverse powers of r shared by the derivative terms below.
template <typename R>
struct PairGeo {
    R rx, ry, rz, ir3, ir5, ir7, ir9;
};

template <typename R>
__device__ __forceinline__ PairGeo<R> pair_geo(R rx, R ry, R rz, R r2)
{
    PairGeo<R> g;
    g.rx = rx;
    g.ry = ry;
    g.rz = rz;
    const R ir = dip_rsqrt(r2);
    const R ir2 = ir * ir;
    g.ir3 = ir2 * ir;
    g.ir5 = g.ir3 * ir2;
    g.ir7 = g.ir5 * ir2;
    g.ir9 = g.ir7 * ir2;
    return g;
}

// grad phi(r; p, q) with phi = p . T(r) q (the printed force with u_k = p,
// u_j = q): 3[p (q.r) + q (p.r) + r (p.q)]/r^5 - 15 r (p.r)(q.r)/r^7, added.
template <typename R>
__device__ __forceinline__ void grad_phi_add(const PairGeo<R>& g, R px, R py, R pz, R qx, R qy,
                                             R qz, R s, R& ox, R& oy, R& oz)
{
    const R pr = px * g.rx + py * g.ry + pz * g.rz;
    const R qr = qx * g.rx + qy * g.ry + qz * g.rz;
    const R pq = px * qx + py * qy + pz * qz;
    const R a = R(3) * g.ir5 * s;
    const R c = (R(3) * pq * g.ir5 - R(15) * pr * qr * g.ir7) * s;
    ox += a * (px * qr + qx * pr) + c * g.rx;
    oy += a * (py * qr + qy * pr) + c * g.ry;
    oz += a * (pz * qr + qz * pr) + c * g.rz;
}

// T(r) p = [3 r (p.r) - p r^2]/r^5, scaled by s and added.
template <typename R>
__device__ __forceinline__ void t_apply_add(const PairGeo<R>& g, R px, R py, R pz, R s, R& ox,
                                            R& oy, R& oz)
{
    const R pr = px * g.rx + py * g.ry + pz * g.rz;
    const R a = R(3) * pr * g.ir5 * s, b = g.ir3 * s;
    ox += a * g.rx - b * px;
    oy += a * g.ry - b * py;
    oz += a * g.rz - b * pz;
}

// H phi(r; p, q) v, the derivative of grad phi(r; p, q) along v:
//   3[(p.v) q + (q.v) p + (p.q) v]/r^5
//   - 15 [r((p.v)(q.r) + (q.v)(p.r) + (r.v)(p.q)) + v (p.r)(q.r) + (r.v)(p (q.r) + q (p.r))]/r^7
//   + 105 r (r.v)(p.r)(q.r)/r^9,   scaled by s and added.
template <typename R>
__device__ __forceinline__ void hess_phi_add(const PairGeo<R>& g, R px, R py, R pz, R qx, R qy,
                                             R qz, R vx, R vy, R vz, R s, R& ox, R& oy, R& oz)
{
    const R pr = px * g.rx + py * g.ry + pz * g.rz;
    const R qr = qx * g.rx + qy * g.ry + qz * g.rz;
    const R rv = g.rx * vx + g.ry * vy + g.rz * vz;
    const R pv = px * vx + py * vy + pz * vz;
    const R qv = qx * vx + qy * vy + qz * vz;
    const R pq = px * qx + py * qy + pz * qz;
    const R a5 = R(3) * g.ir5 * s;
    const R a7 = R(15) * g.ir7 * s;
    const R cr = -a7 * (pv * qr + qv * pr + rv * pq) + R(105) * rv * pr * qr * g.ir9 * s;
    const R cv = a5 * pq - a7 * pr * qr;
    const R cp = a5 * qv - a7 * rv * qr;
    const R cq = a5 * pv - a7 * rv * pr;
    ox += cr * g.rx + cv * vx + cp * px + cq * qx;
    oy += cr * g.ry + cv * vy + cp * py + cq * qy;
    oz += cr * g.rz + cv * vz + cp * pz + cq * qz;
}

}  // namespace ffk
