// Collider: the first, approximate pass of the two-pass detection of the
// Yade text (section 2.1.1, eq. 2.1-2.2), run only when a body has moved more
// than the sweep margin ("Verlet distance", eq. 2.3-2.4).
//
// GB300 design (replaces the single-threaded insertion-sort sweep and prune):
//   1. bin every sphere into a uniform grid of cell edge >= 2 r_max + 2 dL
//      (periodic: in the wrapped reference cell, keeping the integer image);
//   2. counting sort over the Morton codes of the cells (atomics only for the
//      per-cell counts and slots), then sort each cell's bodies by id, so the
//      resulting body order ("slots") is deterministic;
//   3. permute the body arrays into that order (spatial locality for every
//      later gather);
//   4. each body scans the 27 neighbour cells and keeps the pairs with
//      |x2 + H c - x1| < r1 + r2 + 2 dL (count, prefix sum, emit: no atomics);
//   5. merge the contact history of the previous table into the new rows by
//      looking each pair up in the old per-body row ranges (the potential /
//      real interaction lifecycle of section 3.1.7), flipping the stored
//      vectors when the slot order of the pair changed;
//   6. build the per-body "down" lists (rows where the body is the second
//      sphere) for the deterministic force gather.
#include "dem_internal.cuh"

namespace dem {

namespace {
constexpr int kT = 256;

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

// cell coordinates (and, periodic, the integer image) of a position
__device__ inline void cell_of(const Grid &g, double x, double y, double z, int c[3], int img[3]) {
  const double p[3] = {x, y, z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int ck;
    if (g.periodic) {
      double s = p[k] * g.scale[k];
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

// Visit the bodies of the 27 neighbour cells of cell ci; f(j, w) receives the
// body slot and the periodic wrap of the neighbour cell.
template <class F>
__device__ inline void for_neighbours(const Grid &g, const int *__restrict__ count,
                                      const int *__restrict__ start, const int ci[3], F &&f) {
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
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
        const uint32_t m = morton3(cj[0], cj[1], cj[2]);
        const int s0 = start[m], cnt = count[m];
        for (int j = s0; j < s0 + cnt; ++j) f(j, w);
      }
}

// Candidate test of the pair (s, j) found from s through a cell wrap w, always
// evaluated in the pair's canonical orientation (lower slot first) so that
// both ends reach the same decision bit for bit.  Returns the packed shift of
// the higher slot.
struct Cand {
  bool keep;
  int cpack;
  bool range_ok;
};
__device__ inline Cand cand_test(const Grid &g, const double4_32a &ps, const int imgs[3], int s,
                                 const double4_32a &pj, int j, const int w[3]) {
  Cand out{false, 0, true};
  int c[3] = {0, 0, 0};
  if (g.periodic) {
    int cj[3], imgj[3];
    cell_of(g, pj.x, pj.y, pj.z, cj, imgj);
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = imgs[k] - imgj[k] + w[k];   // shift of j seen from s
    if (j < s) { c[0] = -c[0]; c[1] = -c[1]; c[2] = -c[2]; }        // shift of s seen from j
  }
  const double4_32a &a = (s < j) ? ps : pj;
  const double4_32a &b = (s < j) ? pj : ps;
  const double h0 = g.L[0] * c[0], h1 = g.L[1] * c[1], h2 = g.L[2] * c[2];
  const double d0 = (b.x + h0) - a.x, d1 = (b.y + h1) - a.y, d2 = (b.z + h2) - a.z;
  const double R = (a.w + b.w) + g.reach;
  out.keep = d0 * d0 + d1 * d1 + d2 * d2 < R * R;
  if (out.keep) {
    out.range_ok = abs(c[0]) <= kShiftMax && abs(c[1]) <= kShiftMax && abs(c[2]) <= kShiftMax;
    out.cpack = pack_shift(c[0], c[1], c[2]);
  }
  return out;
}

__global__ void k_bbox(const double4_32a *__restrict__ pos, long long N, double *partials) {
  __shared__ double sh[6][kT];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < N; i += (long long)gridDim.x * kT) {
    double4_32a p = pos[i];
    lo[0] = fmin(lo[0], p.x - p.w); hi[0] = fmax(hi[0], p.x + p.w);
    lo[1] = fmin(lo[1], p.y - p.w); hi[1] = fmax(hi[1], p.y + p.w);
    lo[2] = fmin(lo[2], p.z - p.w); hi[2] = fmax(hi[2], p.z + p.w);
  }
  for (int k = 0; k < 3; ++k) { sh[k][threadIdx.x] = lo[k]; sh[3 + k][threadIdx.x] = hi[k]; }
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 3; ++k) {
        sh[k][threadIdx.x] = fmin(sh[k][threadIdx.x], sh[k][threadIdx.x + o]);
        sh[3 + k][threadIdx.x] = fmax(sh[3 + k][threadIdx.x], sh[3 + k][threadIdx.x + o]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 6; ++k) partials[6 * blockIdx.x + k] = sh[k][0];
}

__global__ void k_bin(const double4_32a *__restrict__ pos, long long N, Grid g, uint32_t *key,
                      int *count) {
  long long i = (long long)blockIdx.x * kT + threadIdx.x;
  if (i >= N) return;
  double4_32a p = pos[i];
  int c[3], img[3];
  cell_of(g, p.x, p.y, p.z, c, img);
  uint32_t m = morton3(c[0], c[1], c[2]);
  key[i] = m;
  atomicAdd(&count[m], 1);
}

__global__ void k_scatter(long long N, const uint32_t *__restrict__ key,
                          const int *__restrict__ start, int *fill, int *tmp) {
  long long i = (long long)blockIdx.x * kT + threadIdx.x;
  if (i >= N) return;
  uint32_t m = key[i];
  int p = start[m] + atomicAdd(&fill[m], 1);
  tmp[p] = (int)i;
}

// sort the bodies of each cell by id: fixes the order the atomics left open
__global__ void k_cellsort(const int *__restrict__ count, const int *__restrict__ start,
                           long long ncell, const int *__restrict__ id, int *tmp) {
  long long m = (long long)blockIdx.x * kT + threadIdx.x;
  if (m >= ncell) return;
  int cnt = count[m];
  if (cnt < 2) return;
  int s0 = start[m];
  for (int a = s0 + 1; a < s0 + cnt; ++a) {
    int v = tmp[a];
    int key = id[v];
    int b = a - 1;
    while (b >= s0 && id[tmp[b]] > key) {
      tmp[b + 1] = tmp[b];
      --b;
    }
    tmp[b + 1] = v;
  }
}

__global__ void k_reorder(Bodies src, Bodies dst, long long N, long long cap,
                          const int *__restrict__ new_to_old, int *slot_of_id, int has_walls) {
  long long p = (long long)blockIdx.x * kT + threadIdx.x;
  if (p >= N) return;
  int o = new_to_old[p];
  double4_32a x = src.pos[o];
  dst.pos[p] = x;
  dst.vel[p] = src.vel[o];
  dst.angvel[p] = src.angvel[o];
  dst.ori[p] = src.ori[o];
  dst.mprop[p] = src.mprop[o];
  dst.xref[p] = make_double4_32a(x.x, x.y, x.z, 0.0);
  int id = src.id[o];
  dst.id[p] = id;
  dst.mat[p] = src.mat[o];
  dst.flags[p] = src.flags[o];
  slot_of_id[id] = (int)p;
  if (has_walls)
    for (int w = 0; w < 6; ++w) dst.whist[w * cap + p] = src.whist[w * cap + o];
}

__global__ void k_count(Bodies b, long long N, Grid g, const int *__restrict__ count,
                        const int *__restrict__ start, int *cnt_up, int *cnt_down, int *err) {
  long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= N) return;
  const int s = (int)sl;
  const double4_32a ps = b.pos[s];
  int ci[3], imgs[3];
  cell_of(g, ps.x, ps.y, ps.z, ci, imgs);
  int up = 0, down = 0;
  bool bad = false;
  for_neighbours(g, count, start, ci, [&](int j, const int w[3]) {
    if (j == s) return;
    Cand c = cand_test(g, ps, imgs, s, b.pos[j], j, w);
    if (c.keep) {
      if (j > s) ++up; else ++down;
      bad |= !c.range_ok;
    }
  });
  cnt_up[s] = up;
  cnt_down[s] = down;
  if (bad) atomicOr(err, kErrShiftRange);
}

__global__ void k_emit(Bodies b, long long N, Grid g, const int *__restrict__ count,
                       const int *__restrict__ start, Table t) {
  long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= N) return;
  const int s = (int)sl;
  const double4_32a ps = b.pos[s];
  int ci[3], imgs[3];
  cell_of(g, ps.x, ps.y, ps.z, ci, imgs);
  int r = t.row_start[s];
  const int r_end = t.row_start[s + 1];
  for_neighbours(g, count, start, ci, [&](int j, const int w[3]) {
    if (j <= s) return;
    Cand c = cand_test(g, ps, imgs, s, b.pos[j], j, w);
    if (c.keep && r < r_end) {
      t.pair[r] = make_int2(s, j);
      t.cpack[r] = c.cpack;
      ++r;
    }
  });
}

__global__ void k_down(Bodies b, long long N, Grid g, const int *__restrict__ count,
                       const int *__restrict__ start, Table t) {
  long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= N) return;
  const int s = (int)sl;
  const double4_32a ps = b.pos[s];
  int ci[3], imgs[3];
  cell_of(g, ps.x, ps.y, ps.z, ci, imgs);
  int e = t.down_start[s];
  const int e_end = t.down_start[s + 1];
  for_neighbours(g, count, start, ci, [&](int j, const int w[3]) {
    if (j >= s) return;
    Cand c = cand_test(g, ps, imgs, s, b.pos[j], j, w);
    if (!c.keep || e >= e_end) return;
    int row = -1;
    for (int r = t.row_start[j]; r < t.row_start[j + 1]; ++r)
      if (t.pair[r].y == s && t.cpack[r] == c.cpack) { row = r; break; }
    t.down[e++] = row;   // -1 never happens when both ends agree; the gather skips it
  });
}

__global__ void k_merge(Table nt, Table ot, long long N_old, const int *__restrict__ new_to_old) {
  long long k = (long long)blockIdx.x * kT + threadIdx.x;
  if (k >= nt.P) return;
  const int2 pr = nt.pair[k];
  const int cp = nt.cpack[k];
  const int o1 = new_to_old[pr.x], o2 = new_to_old[pr.y];
  const bool flip = o1 > o2;
  const int a = flip ? o2 : o1, bb = flip ? o1 : o2;
  const int want = flip ? neg_shift(cp) : cp;
  long long hit = -1;
  if (bb < N_old && ot.P > 0) {
    for (int r = ot.row_start[a]; r < ot.row_start[a + 1]; ++r)
      if (ot.pair[r].y == bb && ot.cpack[r] == want) { hit = r; break; }
  }
  double4_32a fs = make_double4_32a(0, 0, 0, 0), hn = make_double4_32a(0, 0, 0, 0);
  double tp = 0;
  if (hit >= 0) {
    double4_32a ofs = ot.hfs[hit];
    if (ofs.w != 0.0) {
      double4_32a ohn = ot.hn[hit];
      const double sg = flip ? -1.0 : 1.0;
      fs = make_double4_32a(sg * ofs.x, sg * ofs.y, sg * ofs.z, ofs.w);
      hn = make_double4_32a(sg * ohn.x, sg * ohn.y, sg * ohn.z, ohn.w);
      tp = ot.tanphi[hit];
      ot.found[hit] = 1;
    }
  }
  nt.hfs[k] = fs;
  nt.hn[k] = hn;
  nt.tanphi[k] = tp;
  nt.oF[k] = make_double4_32a(0, 0, 0, 0);
  nt.oM[k] = make_double4_32a(0, 0, 0, 0);
}

__global__ void k_lost(Table ot, int *err) {
  long long r = (long long)blockIdx.x * kT + threadIdx.x;
  if (r >= ot.P) return;
  if (ot.hfs[r].w != 0.0 && !ot.found[r]) atomicOr(err, kErrHistoryLost);
}

inline unsigned blocks(long long n) { return (unsigned)((n + kT - 1) / kT); }
}  // namespace

int bbox_blocks(long long N) {
  long long b = (N + kT - 1) / kT;
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

void launch_bbox(const Bodies &b, long long N, double *partials, int nblk, cudaStream_t st) {
  k_bbox<<<nblk, kT, 0, st>>>(b.pos, N, partials);
}

void launch_bin(const Bodies &b, long long N, const Grid &g, uint32_t *key, int *count,
                cudaStream_t st) {
  if (N > 0) k_bin<<<blocks(N), kT, 0, st>>>(b.pos, N, g, key, count);
}

void launch_scatter(long long N, const uint32_t *key, const int *start, int *fill, int *tmp,
                    cudaStream_t st) {
  if (N > 0) k_scatter<<<blocks(N), kT, 0, st>>>(N, key, start, fill, tmp);
}

void launch_cellsort(const int *count, const int *start, long long ncell, const int *id,
                     int *tmp, cudaStream_t st) {
  k_cellsort<<<blocks(ncell), kT, 0, st>>>(count, start, ncell, id, tmp);
}

void launch_reorder(const Bodies &src, const Bodies &dst, long long N, long long cap,
                    const int *new_to_old, int *slot_of_id, int has_walls, cudaStream_t st) {
  if (N > 0)
    k_reorder<<<blocks(N), kT, 0, st>>>(src, dst, N, cap, new_to_old, slot_of_id, has_walls);
}

void launch_count(const Bodies &b, long long N, const Grid &g, const int *count,
                  const int *start, int *cnt_up, int *cnt_down, int *err, cudaStream_t st) {
  if (N > 0) k_count<<<blocks(N), kT, 0, st>>>(b, N, g, count, start, cnt_up, cnt_down, err);
}

void launch_emit(const Bodies &b, long long N, const Grid &g, const int *count,
                 const int *start, const Table &t, cudaStream_t st) {
  if (N > 0) k_emit<<<blocks(N), kT, 0, st>>>(b, N, g, count, start, t);
}

void launch_down(const Bodies &b, long long N, const Grid &g, const int *count,
                 const int *start, const Table &t, cudaStream_t st) {
  if (N > 0) k_down<<<blocks(N), kT, 0, st>>>(b, N, g, count, start, t);
}

void launch_merge(const Table &nt, const Table &ot, long long N_old, const int *new_to_old,
                  cudaStream_t st) {
  if (nt.P > 0) k_merge<<<blocks(nt.P), kT, 0, st>>>(nt, ot, N_old, new_to_old);
}

void launch_lost(const Table &ot, int *err, cudaStream_t st) {
  if (ot.P > 0) k_lost<<<blocks(ot.P), kT, 0, st>>>(ot, err);
}

}  // namespace dem
