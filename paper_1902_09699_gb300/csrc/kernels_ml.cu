// Multilevel transfer kernels for ML-PARSDMM (Sec. "Multilevel PARSDMM";
// Algorithm ML-PARSDMM), internal to libsip.so.
//
// restrict: the coarse model m_l is the mean of each 2 x 2 (x 2) block of
//           fine cells (an anti-alias box filter followed by subsampling).
// prolong:  y_i, v_i and x are interpolated "as images" on the output grid
//           of their own operator: separable linear interpolation in
//           fine-cell coordinates, where fine sample i sits at i (+1/2 on the
//           differenced, staggered axis) and coarse sample j at 2j + 1/2
//           (+1 on the staggered axis); past the ends the two nearest coarse
//           samples are extrapolated linearly, so linear fields are exact.
#include <cstdint>
#include <cuda_runtime.h>

#include "sip_kernels.h"

namespace sip {

template <typename T>
__global__ void k_restrict(int64_t fz, int64_t fx, int64_t fy, int64_t cz, int64_t cx, int64_t cy,
                           const T *__restrict__ mf, T *__restrict__ mc) {
  const int64_t n = cz * cx * cy;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t jz = c % cz, t = c / cz, jx = t % cx, jy = t / cx;
    double sum = 0.0;
    int cnt = 0;
    for (int dy = 0; dy < 2; ++dy) {
      const int64_t iy = (fy > 1 ? 2 * jy : 0) + dy;
      if (iy >= fy || (fy == 1 && dy)) continue;
      for (int dx = 0; dx < 2; ++dx) {
        const int64_t ix = 2 * jx + dx;
        if (ix >= fx) continue;
        for (int dz = 0; dz < 2; ++dz) {
          const int64_t iz = 2 * jz + dz;
          if (iz >= fz) continue;
          sum += (double)mf[iz + fz * (ix + fx * iy)];
          ++cnt;
        }
      }
    }
    mc[c] = (T)(sum / cnt);
  }
}

struct AxisW {
  int64_t j0, j1;
  double f;
};

__device__ __forceinline__ AxisW axis_weights(int64_t i, int64_t nc, bool stag) {
  AxisW a;
  if (nc == 1) {
    a.j0 = a.j1 = 0;
    a.f = 0.0;
    return a;
  }
  const double off = stag ? 0.5 : 0.0;
  const double t = ((double)i + off - 0.5 - 2.0 * off) * 0.5;  // continuous coarse index
  int64_t j0 = (int64_t)floor(t);
  if (j0 < 0) j0 = 0;
  if (j0 > nc - 2) j0 = nc - 2;
  a.j0 = j0;
  a.j1 = j0 + 1;
  a.f = t - (double)j0;
  return a;
}

template <typename T>
__global__ void k_prolong(int64_t cz, int64_t cx, int64_t cy, int64_t fz, int64_t fx, int64_t fy, int stag,
                          const T *__restrict__ uc, T *__restrict__ uf) {
  const int64_t n = fz * fx * fy;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t iz = g % fz, t = g / fz, ix = t % fx, iy = t / fx;
    const AxisW az = axis_weights(iz, cz, stag == 0);
    const AxisW ax = axis_weights(ix, cx, stag == 1);
    const AxisW ay = axis_weights(iy, cy, stag == 2);
    double acc = 0.0;
    for (int by = 0; by < 2; ++by) {
      const double wy = by ? ay.f : 1.0 - ay.f;
      if (wy == 0.0) continue;
      const int64_t jy = by ? ay.j1 : ay.j0;
      for (int bx = 0; bx < 2; ++bx) {
        const double wx = bx ? ax.f : 1.0 - ax.f;
        if (wx == 0.0) continue;
        const int64_t jx = bx ? ax.j1 : ax.j0;
        for (int bz = 0; bz < 2; ++bz) {
          const double wz = bz ? az.f : 1.0 - az.f;
          if (wz == 0.0) continue;
          const int64_t jz = bz ? az.j1 : az.j0;
          acc += wy * wx * wz * (double)uc[jz + cz * (jx + cx * jy)];
        }
      }
    }
    uf[g] = (T)acc;
  }
}

static unsigned grid_for_ml(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_restrict(const Launch &L, const int64_t f[3], const int64_t c[3], const void *mf, void *mc) {
  const int64_t n = c[0] * c[1] * c[2];
  if (L.dtype == SIP_F64)
    k_restrict<double><<<grid_for_ml(n), 256, 0, L.stream>>>(f[0], f[1], f[2], c[0], c[1], c[2], (const double *)mf,
                                                             (double *)mc);
  else
    k_restrict<float><<<grid_for_ml(n), 256, 0, L.stream>>>(f[0], f[1], f[2], c[0], c[1], c[2], (const float *)mf,
                                                            (float *)mc);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const Launch &L, const int64_t c[3], const int64_t f[3], int stag, const void *uc,
                           void *uf) {
  const int64_t n = f[0] * f[1] * f[2];
  if (L.dtype == SIP_F64)
    k_prolong<double><<<grid_for_ml(n), 256, 0, L.stream>>>(c[0], c[1], c[2], f[0], f[1], f[2], stag,
                                                            (const double *)uc, (double *)uf);
  else
    k_prolong<float><<<grid_for_ml(n), 256, 0, L.stream>>>(c[0], c[1], c[2], f[0], f[1], f[2], stag,
                                                           (const float *)uc, (float *)uf);
  return cudaGetLastError();
}

}  // namespace sip
