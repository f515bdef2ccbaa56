// Uniform-grid helpers shared by the collider (collider.cu) and the bare pair
// query (pairs.cu): Morton codes of cells, the cell and integer image of a
// position, the forward half of the 27-cell stencil, and the conservative FP32
// candidate test.
#pragma once
#include "dem_internal.cuh"

namespace dem {
namespace {

__host__ __device__ inline uint32_t spread3(uint32_t x) {  // 8 bits -> every third bit
  x &= 0xffu;
  x = (x | (x << 8)) & 0x0000f00fu;
  x = (x | (x << 4)) & 0x000c30c3u;
  x = (x | (x << 2)) & 0x00249249u;
  return x;
}
__host__ __device__ inline uint32_t morton3(int i, int j, int k) {
  return spread3((uint32_t)i) | (spread3((uint32_t)j) << 1) | (spread3((uint32_t)k) << 2);
}

// global index of cell (i, j, k) of grid g: Morton code (one scene) or row-major
// (sub-scenes), offset by the grid's first cell
__host__ __device__ inline long long cell_index(const Grid &g, int i, int j, int k) {
  return g.base + (g.morton ? (long long)morton3(i, j, k)
                            : ((long long)k * g.n[1] + j) * g.n[0] + i);
}

// cell coordinates (and, periodic, the integer image) of a position
__device__ inline void cell_of(const Grid &g, double x, double y, double z, int c[3], int img[3]) {
  const double p[3] = {x, y, z};
  double u[3] = {x * g.scale[0], y * g.scale[1], z * g.scale[2]};   // fractional (periodic)
  if (g.periodic && g.sheared)   // sheared cell: s = Hinv x
    for (int k = 0; k < 3; ++k)
      u[k] = g.Hinv[3 * k] * x + g.Hinv[3 * k + 1] * y + g.Hinv[3 * k + 2] * z;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int ck;
    if (g.periodic) {
      double s = u[k];
      double fi = floor(s);
      double f = s - fi;
      ck = (int)(f * g.n[k]);
      img[k] = (int)fi;
    } else {
      ck = (int)floor((p[k] - g.lo[k]) * g.scale[k]);
      img[k] = 0;
    }
    c[k] = ck < 0 ? 0 : (ck >= g.n[k] ? g.n[k] - 1 : ck);
  }
}

__device__ inline int neg_shift(int p) {
  int a, b, c;
  unpack_shift(p, a, b, c);
  return pack_shift(-a, -b, -c);
}

// Forward half of the 27-cell stencil: own cell (partners with a higher slot)
// plus the 13 offsets with (dz, dy, dx) lexicographically positive, so every pair
// of neighbouring cells is visited from exactly one side.
template <class F>
__device__ inline void for_half_shell(const Grid &g, const int *__restrict__ count,
                                      const int *__restrict__ start, const int ci[3], int s,
                                      F &&f) {
  for (int dz = 0; dz <= 1; ++dz)
    for (int dy = (dz ? -1 : 0); dy <= 1; ++dy)
      for (int dx = ((dz || dy) ? -1 : 0); dx <= 1; ++dx) {
        const int d[3] = {dx, dy, dz};
        int cj[3], w[3];
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          int c = ci[k] + d[k];
          w[k] = 0;
          if (g.periodic) {
            if (c < 0) { c += g.n[k]; w[k] = -1; }
            else if (c >= g.n[k]) { c -= g.n[k]; w[k] = 1; }
          } else if (c < 0 || c >= g.n[k]) {
            ok = false;
          }
          cj[k] = c;
        }
        if (!ok) continue;
        const bool self = (dx == 0 && dy == 0 && dz == 0);
        const long long m = cell_index(g, cj[0], cj[1], cj[2]);
        const int s0 = start[m], cnt = count[m];
        for (int j = (self ? s + 1 : s0); j < s0 + cnt; ++j) f(j, w);
      }
}

// Per-slot collider record: FP32 position relative to the grid (periodic: the
// wrapped position), radius, packed cell coordinates and the integer image.
struct CellRec {
  float4 *wpos;   // (x, y, z, r)
  int4 *info;     // (cell0 | cell1 << 10 | cell2 << 20, img0, img1, img2)
};

// Conservative FP32 candidate test of (s, j): keeps every pair whose FP64
// distance is below r1 + r2 + reach (the slack covers the FP32 rounding of
// coordinates bounded by the cell size), so the candidate set is a superset of
// the exact one; count and emit evaluate it identically.
__device__ inline bool cand_f32(const Grid &g, const float4 &a, const float4 &b, const int w[3],
                                float slack) {
  float sx = (float)w[0] * g.Lf[0], sy = (float)w[1] * g.Lf[1], sz = (float)w[2] * g.Lf[2];
  if (g.sheared) {   // image shift H w of a sheared cell
    const float f0 = (float)w[0], f1 = (float)w[1], f2 = (float)w[2];
    sx = g.Hf[0] * f0 + g.Hf[1] * f1 + g.Hf[2] * f2;
    sy = g.Hf[3] * f0 + g.Hf[4] * f1 + g.Hf[5] * f2;
    sz = g.Hf[6] * f0 + g.Hf[7] * f1 + g.Hf[8] * f2;
  }
  const float dx = (b.x + sx) - a.x;
  const float dy = (b.y + sy) - a.y;
  const float dz = (b.z + sz) - a.z;
  const float R = (a.w + b.w) + g.reachf + slack;
  return dx * dx + dy * dy + dz * dz < R * R;
}


}  // namespace
}  // namespace dem
