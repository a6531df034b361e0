// gc_sh.cuh - real spherical harmonics of degree <= 3 as Cartesian polynomials of
// a unit direction (x, y, z), Condon-Shortley phase, index k = l^2 + l + m.
// The paper colours each Gaussian by SH coefficients "in the viewing
// direction" (Sec. 3.1); this is the standard real basis.
//
// Normalisation constants (closed forms):
//   K0  = 1/(2 sqrt(pi))           K1  = sqrt(3/(4 pi))
//   K2a = (1/2) sqrt(15/pi)        K2b = (1/4) sqrt(5/pi)      K2c = (1/4) sqrt(15/pi)
//   K3a = (1/4) sqrt(35/(2 pi))    K3b = (1/2) sqrt(105/pi)    K3c = (1/4) sqrt(21/(2 pi))
//   K3d = (1/4) sqrt(7/pi)         K3e = (1/4) sqrt(105/pi)
#pragma once

namespace gc {

constexpr float kK0 = 0.28209479177387814f;
constexpr float kK1 = 0.48860251190291992f;
constexpr float kK2a = 1.0925484305920792f;
constexpr float kK2b = 0.31539156525252005f;
constexpr float kK2c = 0.54627421529603959f;
constexpr float kK3a = 0.59004358992664352f;
constexpr float kK3b = 2.8906114426405538f;
constexpr float kK3c = 0.45704579946446573f;
constexpr float kK3d = 0.37317633259011540f;
constexpr float kK3e = 1.4453057213202769f;

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float *Y) {
    Y[0] = kK0;
    if (deg < 1) return;
    Y[1] = -kK1 * y;
    Y[2] = kK1 * z;
    Y[3] = -kK1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kK2a * x * y;
    Y[5] = -kK2a * y * z;
    Y[6] = kK2b * (2.f * zz - xx - yy);
    Y[7] = -kK2a * x * z;
    Y[8] = kK2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -kK3a * y * (3.f * xx - yy);
    Y[10] = kK3b * x * y * z;
    Y[11] = -kK3c * y * (4.f * zz - xx - yy);
    Y[12] = kK3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -kK3c * x * (4.f * zz - xx - yy);
    Y[14] = kK3e * z * (xx - yy);
    Y[15] = -kK3a * x * (xx - 3.f * yy);
}

// Gradient of sum_k w[k] Y_k(x, y, z) with respect to (x, y, z), treating the
// polynomials above as functions on R^3 (the caller projects out the radial part).
__device__ __forceinline__ void sh_basis_vjp(int deg, float x, float y, float z, const float *w,
                                             float &gx, float &gy, float &gz) {
    gx = 0.f; gy = 0.f; gz = 0.f;
    if (deg < 1) return;
    gy += -kK1 * w[1];
    gz += kK1 * w[2];
    gx += -kK1 * w[3];
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += kK2a * y * w[4];            gy += kK2a * x * w[4];
    gy += -kK2a * z * w[5];           gz += -kK2a * y * w[5];
    gx += -2.f * kK2b * x * w[6];     gy += -2.f * kK2b * y * w[6];     gz += 4.f * kK2b * z * w[6];
    gx += -kK2a * z * w[7];           gz += -kK2a * x * w[7];
    gx += 2.f * kK2c * x * w[8];      gy += -2.f * kK2c * y * w[8];
    if (deg < 3) return;
    // Y9 = -K3a (3 x^2 y - y^3)
    gx += -kK3a * 6.f * x * y * w[9];
    gy += -kK3a * (3.f * xx - 3.f * yy) * w[9];
    // Y10 = K3b x y z
    gx += kK3b * y * z * w[10]; gy += kK3b * x * z * w[10]; gz += kK3b * x * y * w[10];
    // Y11 = -K3c (4 y z^2 - x^2 y - y^3)
    gx += kK3c * 2.f * x * y * w[11];
    gy += -kK3c * (4.f * zz - xx - 3.f * yy) * w[11];
    gz += -kK3c * 8.f * y * z * w[11];
    // Y12 = K3d (2 z^3 - 3 x^2 z - 3 y^2 z)
    gx += -kK3d * 6.f * x * z * w[12];
    gy += -kK3d * 6.f * y * z * w[12];
    gz += kK3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
    // Y13 = -K3c (4 x z^2 - x^3 - x y^2)
    gx += -kK3c * (4.f * zz - 3.f * xx - yy) * w[13];
    gy += kK3c * 2.f * x * y * w[13];
    gz += -kK3c * 8.f * x * z * w[13];
    // Y14 = K3e (x^2 z - y^2 z)
    gx += kK3e * 2.f * x * z * w[14];
    gy += -kK3e * 2.f * y * z * w[14];
    gz += kK3e * (xx - yy) * w[14];
    // Y15 = -K3a (x^3 - 3 x y^2)
    gx += -kK3a * (3.f * xx - 3.f * yy) * w[15];
    gy += kK3a * 6.f * x * y * w[15];
}

}  // namespace gc
