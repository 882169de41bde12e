// View-dependent colour (Sec. 3.1): real spherical harmonics of degree <= 3
// of the unit direction d from the camera centre to the surfel centre,
// c = max(0, sum_b k_b Y_b(d) + 1/2) per channel, basis index b = l^2 + l + m.
// The harmonics are the real ones without the Condon-Shortley sign, as
// Cartesian polynomials on the unit sphere (normalisation sqrt((2l+1)/(4 pi)
// (l-m)!/(l+m)!), times sqrt(2) for m != 0):
//   l = 0: c0
//   l = 1: c1 y, c1 z, c1 x
//   l = 2: c2a xy, c2a yz, c20 (3z^2 - 1), c2a xz, c22 (x^2 - y^2)
//   l = 3: c3a y(3x^2 - y^2), c3b xyz, c3c y(5z^2 - 1), c30 z(5z^2 - 3),
//          c3c x(5z^2 - 1), c32 z(x^2 - y^2), c3a x(x^2 - 3y^2)
#pragma once

#include "fss_internal.cuh"

namespace fss {

namespace sh {
constexpr float c0 = 0.28209479177387814f;   // (1/2) sqrt(1/pi)
constexpr float c1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float c2a = 1.0925484305920792f;   // (1/2) sqrt(15/pi)
constexpr float c20 = 0.31539156525252005f;  // (1/4) sqrt(5/pi)
constexpr float c22 = 0.5462742152960396f;   // (1/4) sqrt(15/pi)
constexpr float c3a = 0.5900435899266435f;   // (1/4) sqrt(35/(2 pi))
constexpr float c3b = 2.890611442640554f;    // (1/2) sqrt(105/pi)
constexpr float c3c = 0.4570457994644658f;   // (1/4) sqrt(21/(2 pi))
constexpr float c30 = 0.3731763325901154f;   // (1/4) sqrt(7/pi)
constexpr float c32 = 1.445305721320277f;    // (1/4) sqrt(105/pi)
}  // namespace sh

// basis Y[0 .. (deg+1)^2) at the unit direction (x, y, z)
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
    using namespace sh;
    Y[0] = c0;
    if (deg < 1) return;
    Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = c2a * x * y; Y[5] = c2a * y * z; Y[6] = c20 * (3.0f * zz - 1.0f); Y[7] = c2a * x * z;
    Y[8] = c22 * (xx - yy);
    if (deg < 3) return;
    Y[9] = c3a * y * (3.0f * xx - yy); Y[10] = c3b * x * y * z; Y[11] = c3c * y * (5.0f * zz - 1.0f);
    Y[12] = c30 * z * (5.0f * zz - 3.0f); Y[13] = c3c * x * (5.0f * zz - 1.0f); Y[14] = c32 * z * (xx - yy);
    Y[15] = c3a * x * (xx - 3.0f * yy);
}

// gradient of sum_b k[b] Y_b with respect to (x, y, z), for the k[b] of one
// channel (k strided by `ks`): the partial derivatives of the polynomials
__device__ __forceinline__ void sh_grad_dot(int deg, float x, float y, float z, const float* k, int ks, float& gx,
                                            float& gy, float& gz) {
    using namespace sh;
    gx = gy = gz = 0.0f;
    if (deg < 1) return;
    gy += c1 * k[1 * ks]; gz += c1 * k[2 * ks]; gx += c1 * k[3 * ks];
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float k4 = k[4 * ks], k5 = k[5 * ks], k6 = k[6 * ks], k7 = k[7 * ks], k8 = k[8 * ks];
    gx += c2a * (y * k4 + z * k7) + 2.0f * c22 * x * k8;
    gy += c2a * (x * k4 + z * k5) - 2.0f * c22 * y * k8;
    gz += c2a * (y * k5 + x * k7) + 6.0f * c20 * z * k6;
    if (deg < 3) return;
    const float k9 = k[9 * ks], k10 = k[10 * ks], k11 = k[11 * ks], k12 = k[12 * ks], k13 = k[13 * ks],
                k14 = k[14 * ks], k15 = k[15 * ks];
    gx += c3a * 6.0f * x * y * k9 + c3b * y * z * k10 + c3c * (5.0f * zz - 1.0f) * k13 + c32 * 2.0f * x * z * k14 +
          c3a * 3.0f * (xx - yy) * k15;
    gy += c3a * 3.0f * (xx - yy) * k9 + c3b * x * z * k10 + c3c * (5.0f * zz - 1.0f) * k11 -
          c32 * 2.0f * y * z * k14 - c3a * 6.0f * x * y * k15;
    gz += c3b * x * y * k10 + c3c * 10.0f * y * z * k11 + c30 * (15.0f * zz - 3.0f) * k12 +
          c3c * 10.0f * x * z * k13 + c32 * (xx - yy) * k14;
}

// camera centre -R^T t of a view
__device__ __forceinline__ void cam_centre(const CamDev& cam, float& cx, float& cy, float& cz) {
    cx = -(cam.R[0] * cam.t[0] + cam.R[3] * cam.t[1] + cam.R[6] * cam.t[2]);
    cy = -(cam.R[1] * cam.t[0] + cam.R[4] * cam.t[1] + cam.R[7] * cam.t[2]);
    cz = -(cam.R[2] * cam.t[0] + cam.R[5] * cam.t[1] + cam.R[8] * cam.t[2]);
}

}  // namespace fss
