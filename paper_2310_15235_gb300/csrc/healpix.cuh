// HEALPix RING scheme on the device (Gorski et al. 2005): pixel centres in
// FP64, and the pixel of a direction in FP32 with an FP64 re-check whenever
// the FP32 evaluation lands within a guard band of a pixel boundary.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace trevr2 {

constexpr double kPiD = 3.14159265358979323846;

// Pixel centre of RING pixel p.  Polar rings i (1 <= i < n) hold 4i pixels
// at z = 1 - i^2/(3n^2), phi = pi/(2i) (j + 1/2); the 2n+1 equatorial rings
// hold 4n pixels at z = 2(2n - i)/(3n), phi = pi/(2n)(j + s/2), s = 1 on the
// odd ones counted from z = 2/3; the south cap mirrors the north.
__host__ __device__ inline void hp_pix2vec(int nside, int64_t p, double v[3]) {
  const int64_t n = nside, npix = 12 * n * n, ncap = 2 * n * (n - 1);
  double z, phi;
  auto ring_of = [](int64_t q) {  // ring i with 2i(i-1) <= q < 2i(i+1)
    int64_t i = int64_t((1.0 + sqrt(1.0 + 2.0 * double(q))) * 0.5);
    while (2 * i * (i + 1) <= q) ++i;
    while (i > 1 && 2 * i * (i - 1) > q) --i;
    return i;
  };
  if (p < ncap) {
    int64_t i = ring_of(p);
    int64_t j = p - 2 * i * (i - 1);
    z = 1.0 - double(i * i) / (3.0 * double(n * n));
    phi = kPiD / (2.0 * double(i)) * (double(j) + 0.5);
  } else if (p < npix - ncap) {
    int64_t q = p - ncap;
    int64_t ir = q / (4 * n) + 1;
    int64_t j = q - (ir - 1) * 4 * n;
    z = 2.0 * double(n - ir + 1) / (3.0 * double(n));
    phi = kPiD / (2.0 * double(n)) * (double(j) + ((ir & 1) ? 0.5 : 0.0));
  } else {
    int64_t q = npix - 1 - p;
    int64_t i = ring_of(q);
    int64_t j = p - (npix - 2 * i * (i + 1));
    z = -(1.0 - double(i * i) / (3.0 * double(n * n)));
    phi = kPiD / (2.0 * double(i)) * (double(j) + 0.5);
  }
  double st = sqrt((1.0 - z) * (1.0 + z));
  v[0] = st * cos(phi);
  v[1] = st * sin(phi);
  v[2] = z;
  // phi on a multiple of pi/2 must give exact zeros (lost to pi's rounding)
  for (int a = 0; a < 3; ++a)
    if (fabs(v[a]) < 1e-15) v[a] = 0.0;
}

// FP64 pixel of a direction (any length > 0).
__host__ __device__ inline int hp_vec2pix_f64(int nside, double x, double y, double zc) {
  const int64_t n = nside, npix = 12 * n * n, ncap = 2 * n * (n - 1);
  double z = zc / sqrt(x * x + y * y + zc * zc);
  double phi = atan2(y, x);
  if (phi < 0.0) phi += 2.0 * kPiD;
  double tt = phi / (0.5 * kPiD);
  double za = fabs(z);
  if (za <= 2.0 / 3.0) {
    double t1 = double(n) * (0.5 + tt), t2 = double(n) * z * 0.75;
    int64_t jp = int64_t(floor(t1 - t2)), jm = int64_t(floor(t1 + t2));
    int64_t ir = n + 1 + jp - jm;
    int64_t ip = (jp + jm - n + (1 - (ir & 1)) + 1) / 2;
    ip = ((ip % (4 * n)) + 4 * n) % (4 * n);
    return int(ncap + (ir - 1) * 4 * n + ip);
  }
  double tp = tt - floor(tt);
  double tmp = double(n) * sqrt(3.0 * (1.0 - za));
  int64_t jp = int64_t(floor(tp * tmp)), jm = int64_t(floor((1.0 - tp) * tmp));
  int64_t ir = jp + jm + 1;
  int64_t ip = int64_t(floor(tt * double(ir)));
  ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
  return int(z > 0.0 ? 2 * ir * (ir - 1) + ip : npix - 2 * ir * (ir + 1) + ip);
}

// Distance of x from the nearest integer.
__device__ __forceinline__ float frac_dist(float x) { return fabsf(x - rintf(x)); }

// FP32 pixel of a direction, or -1 when some boundary coordinate of the
// evaluation lies within `eps` of an integer (then the caller re-checks in
// FP64).  eps must bound the FP32 error of the boundary coordinates, which
// are of size <= 4.5 nside.
__device__ __forceinline__ int hp_vec2pix_f32(int nside, float x, float y, float zc, float eps) {
  const int n = nside;
  const float PI_F = 3.14159265358979f;
  float inv = rsqrtf(x * x + y * y + zc * zc);
  float z = zc * inv;
  float phi = atan2f(y, x);
  if (phi < 0.0f) phi += 2.0f * PI_F;
  float tt = phi * (2.0f / PI_F);
  float za = fabsf(z);
  if (fabsf(za - (2.0f / 3.0f)) * float(n) <= eps) return -1;
  if (za < 2.0f / 3.0f) {
    float t1 = float(n) * (0.5f + tt), t2 = float(n) * z * 0.75f;
    float a = t1 - t2, b = t1 + t2;
    if (frac_dist(a) <= eps || frac_dist(b) <= eps) return -1;
    int jp = int(floorf(a)), jm = int(floorf(b));
    int ir = n + 1 + jp - jm;
    int ip = (jp + jm - n + (1 - (ir & 1)) + 1) / 2;
    ip = ((ip % (4 * n)) + 4 * n) % (4 * n);
    return 2 * n * (n - 1) + (ir - 1) * 4 * n + ip;
  }
  if (frac_dist(tt) * float(n) <= eps) return -1;
  float tp = tt - floorf(tt);
  float tmp = float(n) * sqrtf(3.0f * (1.0f - za));
  float a = tp * tmp, b = (1.0f - tp) * tmp;
  if (frac_dist(a) <= eps || frac_dist(b) <= eps) return -1;
  int jp = int(floorf(a)), jm = int(floorf(b));
  int ir = jp + jm + 1;
  float c = tt * float(ir);
  if (frac_dist(c) <= eps) return -1;
  int ip = int(floorf(c));
  ip = ((ip % (4 * ir)) + 4 * ir) % (4 * ir);
  return z > 0.0f ? 2 * ir * (ir - 1) + ip : 12 * n * n - 2 * ir * (ir + 1) + ip;
}

// Guard band for a direction v of length r (normalised units) whose
// components carry an absolute error of at most ~2.1e-7: the FP32 function
// error (a few ulp of coordinates up to 4.5 nside) plus the propagated
// input error (<= 1.6 nside |dv| / r).
__device__ __forceinline__ float hp_guard(int nside, float r) {
  return float(nside) * (4e-6f + 6e-7f / r);
}

}  // namespace trevr2
