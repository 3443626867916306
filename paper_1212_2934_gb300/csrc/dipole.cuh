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
    const R t = R(3) * bj * ir5;
    hx += rx * t - ujx * ir3;
    hy += ry * t - ujy * ir3;
    hz += rz * t - ujz * ir3;
    const R s3 = R(3) * ir5;
    const R cr = s3 * a - R(15) * bk * bj * ir7;
    const R cuk = s3 * bj, cuj = s3 * bk;
    fx += rx * cr + ukx * cuk + ujx * cuj;
    fy += ry * cr + uky * cuk + ujy * cuj;
    fz += rz * cr + ukz * cuk + ujz * cuj;
}

}  // namespace ffk
