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
//   4. each body scans the forward half of its 27-cell neighbourhood (so each
//      pair is met once) and keeps the pairs with |x2 + H c - x1| < r1 + r2 + 2 dL,
//      tested conservatively in FP32 on wrapped coordinates (count, prefix sum,
//      emit).  A row is oriented by id, not by slot: body 1 is the sphere with the
//      smaller id (the canonical id1 < id2 of the interaction container), and the
//      row is stored in body 1's row range, which is then sorted by the id of
//      body 2;
//   5. merge the contact history of the previous table into the new rows by
//      looking each pair up in the old row range of its body 1 (the potential /
//      real interaction lifecycle of section 3.1.7);
//   6. build the per-body "down" lists (rows where the body is the second
//      sphere), sorted by the id of body 1.
// So a body's rows, down list first, then its own range, run in increasing order
// of partner id; the force gather sums them in that order.  With the orientation
// by id, the FP64 arithmetic of a step depends on the bodies and their contact
// histories only, not on the slot order, the times of the collider runs or the
// other sub-scenes in the arrays: a sub-scene advances bit for bit as it would
//   alone.
#include "dem_internal.cuh"
#include "grid.cuh"

namespace dem {

namespace {
constexpr int kT = 256;

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

// Grid of body i: the one grid, or the grid of its sub-scene.
__device__ __forceinline__ const Grid &grid_of(const Grid *__restrict__ grids,
                                               const int *__restrict__ sid, int multi, long long i) {
  return grids[multi ? sid[i] : 0];
}

// Cell key of every body; bodies of a removed sub-scene (grid with no cells) get
// the sentinel key `dead`, which sorts them behind every live body.
// Order-preserving map of doubles to unsigned integers (sign bit flipped for
// positives, all bits for negatives), so that integer atomics give min / max.
__device__ __forceinline__ unsigned long long ord_key(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Bounding boxes of the sub-scenes: keys[k * cap + q] (k = 0..2 lower, 3..5 upper
// bounds of x - r / x + r), lower keys preset to all ones and upper to zero.  A
// warp whose bodies share one sub-scene (the usual case: bodies are grouped by
// sub-scene) reduces in registers and issues six atomics.
__global__ void k_bbox_sub(const double4_32a *__restrict__ pos, const int *__restrict__ sid,
                           long long N, int cap, unsigned long long *keys) {
  const int lane = threadIdx.x & 31;
  const long long stride = (long long)gridDim.x * kT;
  for (long long base = (long long)blockIdx.x * kT + (threadIdx.x & ~31); base < N; base += stride) {
    const long long i = base + lane;
    int q = -1;
    unsigned long long k[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
    if (i < N) {
      q = sid[i];
      const double4_32a p = pos[i];
      k[0] = ord_key(p.x - p.w); k[1] = ord_key(p.y - p.w); k[2] = ord_key(p.z - p.w);
      k[3] = ord_key(p.x + p.w); k[4] = ord_key(p.y + p.w); k[5] = ord_key(p.z + p.w);
    }
    const int q0 = __shfl_sync(0xffffffffu, q, 0);
    const bool uniform = __all_sync(0xffffffffu, q == q0 || q < 0);
    if (uniform) {
      for (int o = 16; o > 0; o >>= 1)
        for (int c = 0; c < 6; ++c) {
          const unsigned long long v = __shfl_down_sync(0xffffffffu, k[c], o);
          k[c] = c < 3 ? (v < k[c] ? v : k[c]) : (v > k[c] ? v : k[c]);
        }
      if (lane == 0 && q0 >= 0)
        for (int c = 0; c < 6; ++c) {
          if (c < 3) atomicMin(&keys[(long long)c * cap + q0], k[c]);
          else atomicMax(&keys[(long long)c * cap + q0], k[c]);
        }
    } else if (q >= 0) {
      for (int c = 0; c < 6; ++c) {
        if (c < 3) atomicMin(&keys[(long long)c * cap + q], k[c]);
        else atomicMax(&keys[(long long)c * cap + q], k[c]);
      }
    }
  }
}

__global__ void k_bin(const double4_32a *__restrict__ pos, const int *__restrict__ sid, long long N,
                      const Grid *__restrict__ grids, int multi, uint32_t dead, uint32_t *key,
                      int *count) {
  long long i = (long long)blockIdx.x * kT + threadIdx.x;
  if (i >= N) return;
  const Grid &g = grid_of(grids, sid, multi, i);
  uint32_t m = dead;
  if (g.n[0] > 0) {
    const double4_32a p = pos[i];
    int c[3], img[3];
    cell_of(g, p.x, p.y, p.z, c, img);
    m = (uint32_t)cell_index(g, c[0], c[1], c[2]);
  }
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
                          const int *__restrict__ new_to_old, int *slot_of_id, int has_walls,
                          int mixed, const int *__restrict__ id_shift) {
  long long p = (long long)blockIdx.x * kT + threadIdx.x;
  if (p >= N) return;
  int o = new_to_old[p];
  double4_32a x = src.pos[o];
  dst.pos[p] = x;
  const double4_32a v = src.vel[o], w = src.angvel[o];
  dst.vel[p] = v;
  dst.angvel[p] = w;
  if (mixed) {   // the new reference position is x itself: zero offset
    dst.p32[p] = make_float4(0.0f, 0.0f, 0.0f, (float)x.w);
    dst.vw32[2 * p] = make_float4((float)v.x, (float)v.y, (float)v.z, (float)w.x);
    dst.vw32[2 * p + 1] = make_float4((float)w.y, (float)w.z, 0.0f, 0.0f);
    dst.xref32[p] = make_float4((float)x.x, (float)x.y, (float)x.z, 0.0f);
    const double4_32a mp = src.mprop[o];
    dst.mprop32[p] = make_float4((float)mp.x, (float)mp.y, (float)mp.z, (float)mp.w);
    dst.ori32[p] = src.ori32[o];   // the mixed path keeps the orientation in FP32
  }
  dst.ori[p] = src.ori[o];
  dst.mprop[p] = src.mprop[o];
  dst.rdsc[p] = src.rdsc[o];
  dst.xref[p] = make_double4_32a(x.x, x.y, x.z, 0.0);
  const int q = src.sid[o];
  // ids close up over the ranges of removed sub-scenes
  const int id = src.id[o] - (id_shift ? id_shift[q] : 0);
  dst.id[p] = id;
  dst.sid[p] = q;
  dst.mat[p] = src.mat[o];
  dst.flags[p] = src.flags[o];
  slot_of_id[id] = (int)p;
  if (has_walls)
    for (int w = 0; w < 6; ++w) dst.whist[w * cap + p] = src.whist[w * cap + o];
}

__global__ void k_cellrec(const double4_32a *__restrict__ pos, const int *__restrict__ sid,
                          long long N, const Grid *__restrict__ grids, int multi, CellRec cr) {
  long long i = (long long)blockIdx.x * kT + threadIdx.x;
  if (i >= N) return;
  const Grid &g = grid_of(grids, sid, multi, i);
  const double4_32a p = pos[i];
  int c[3], img[3];
  cell_of(g, p.x, p.y, p.z, c, img);
  double x[3] = {p.x, p.y, p.z};
  float f[3];
  for (int k = 0; k < 3; ++k) {
    double shift = g.L[k] * img[k];
    if (g.periodic && g.sheared)   // wrapped position x - H img
      shift = g.H[3 * k] * img[0] + g.H[3 * k + 1] * img[1] + g.H[3 * k + 2] * img[2];
    f[k] = g.periodic ? (float)(x[k] - shift) : (float)(x[k] - g.lo[k]);
  }
  cr.wpos[i] = make_float4(f[0], f[1], f[2], (float)p.w);
  cr.info[i] = make_int4(c[0] | (c[1] << 10) | (c[2] << 20), img[0], img[1], img[2]);
}

__device__ inline void unpack_cell(int v, int c[3]) {
  c[0] = v & 1023;
  c[1] = (v >> 10) & 1023;
  c[2] = (v >> 20) & 1023;
}

// Candidate counts: cnt_up[body 1] and cnt_down[body 2] of every candidate, body 1
// being the sphere with the smaller id (both arrays zeroed before).  Count and emit read
// the partners' records through the read-only path (__ldg): nothing in the walk writes
// them, and the compiler may then issue those loads ahead of the atomics.
__global__ void k_count(CellRec cr, const int *__restrict__ sid, const int *__restrict__ id,
                        long long N, const Grid *__restrict__ grids, int multi,
                        const int *__restrict__ count, const int *__restrict__ start,
                        int *cnt_up, int *cnt_down, int *err, CandList cl) {
  long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= N) return;
  const int s = (int)sl;
  const Grid &g = grid_of(grids, sid, multi, sl);
  const float4 a = cr.wpos[s];
  const int4 inf = cr.info[s];
  const int ids = id[s];
  int ci[3];
  unpack_cell(inf.x, ci);
  bool bad = false;
  int nc = 0;
  unsigned *mine = cl.list + (long long)s * kCandKeep;
  for_half_shell(g, count, start, ci, s, [&](int j, const int w[3]) {
    if (cand_f32(g, a, __ldg(cr.wpos + j), w, g.slack)) {
      if (cl.use && nc < kCandKeep)   // slot and the neighbour cell's wrap (code 0..26)
        mine[nc] = (unsigned)j | ((unsigned)((w[0] + 1) + 3 * (w[1] + 1) + 9 * (w[2] + 1)) << 26);
      ++nc;
      const bool fwd = ids < __ldg(id + j);
      atomicAdd(&cnt_up[fwd ? s : j], 1);
      atomicAdd(&cnt_down[fwd ? j : s], 1);
      if (g.periodic) {
        const int4 ij = __ldg(cr.info + j);
        bad |= abs(inf.y - ij.y + w[0]) > kShiftMax || abs(inf.z - ij.z + w[1]) > kShiftMax ||
               abs(inf.w - ij.w + w[2]) > kShiftMax;
      }
    }
  });
  if (cl.use) cl.n[s] = nc;
  if (bad) atomicOr(err, kErrShiftRange);
}

// Row of candidate (s, j) in the row range of its body 1 (smaller id) at a position the
// atomics pick; w: the wrap of j's neighbour cell as seen from s.
__device__ inline void emit_row(const CellRec &cr, const Bodies &b, const Table &t, int *ufill,
                                const Grid &g, const int4 &inf, int s, int ids, int j,
                                const int w[3]) {
  int c0 = 0, c1 = 0, c2 = 0;   // cell shift of j seen from s
  if (g.periodic) {
    const int4 ij = __ldg(cr.info + j);
    c0 = inf.y - ij.y + w[0]; c1 = inf.z - ij.z + w[1]; c2 = inf.w - ij.w + w[2];
  }
  const int idj = __ldg(b.id + j);
  const bool fwd = ids < idj;
  const int g1 = fwd ? s : j, g2 = fwd ? j : s;
  const int r = t.row_start[g1] + atomicAdd(&ufill[g1], 1);
  if (r < t.row_start[g1 + 1]) {
    t.pair[r] = make_int2(g1, g2);
    t.cpack[r] = fwd ? pack_shift(c0, c1, c2) : pack_shift(-c0, -c1, -c2);   // shift of body 2
    t.found[r] = fwd ? idj : ids;   // sort key: the id of body 2 (scratch until the merge)
  }
}

// Rows of the candidates, each in the row range of its body 1 (smaller id) at a
// position the atomics pick; k_rowsort then fixes the order.  ufill: zeroed.  A walker
// whose candidates all fit the count pass's list places them from it; the others walk
// the cells again with the same test.
__global__ void k_emit(CellRec cr, Bodies b, long long N, const Grid *__restrict__ grids,
                       int multi, const int *__restrict__ count, const int *__restrict__ start,
                       Table t, int *ufill, CandList cl) {
  long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= N) return;
  const int s = (int)sl;
  const Grid &g = grid_of(grids, b.sid, multi, sl);
  const int4 inf = cr.info[s];
  const int ids = b.id[s];
  const int nc = cl.use ? cl.n[s] : kCandKeep + 1;
  if (nc <= kCandKeep) {
    const unsigned *mine = cl.list + (long long)s * kCandKeep;
    for (int k = 0; k < nc; ++k) {
      const unsigned e = mine[k];
      const int j = (int)(e & 0x3ffffffu), code = (int)(e >> 26);
      const int w[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
      emit_row(cr, b, t, ufill, g, inf, s, ids, j, w);
    }
    return;
  }
  const float4 a = cr.wpos[s];
  int ci[3];
  unpack_cell(inf.x, ci);
  for_half_shell(g, count, start, ci, s, [&](int j, const int w[3]) {
    if (cand_f32(g, a, __ldg(cr.wpos + j), w, g.slack)) emit_row(cr, b, t, ufill, g, inf, s, ids, j, w);
  });
}

// Sort each body's own row range by (id of body 2, shift): the order the atomics left
// open becomes the order of the partner ids.  Keys (the partner ids) come from the emit
// in t.found; a range of up to kSortLocal rows is sorted in registers and local memory,
// a longer one in place.
constexpr int kSortLocal = 48;
__global__ void k_rowsort(Table t, long long N) {
  const long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= N) return;
  const int r0 = t.row_start[sl], r1 = t.row_start[sl + 1], n = r1 - r0;
  if (n < 2) return;
  if (n <= kSortLocal) {
    long long key[kSortLocal];   // (partner id, shift as unsigned) | position
    int2 pr[kSortLocal];
    int cp[kSortLocal];
    for (int a = 0; a < n; ++a) {
      pr[a] = t.pair[r0 + a];
      cp[a] = t.cpack[r0 + a];
      key[a] = ((long long)t.found[r0 + a] << 32) | (long long)(unsigned)cp[a];
    }
    int ord[kSortLocal];
    for (int a = 0; a < n; ++a) {
      int q = a - 1;
      const long long kv = key[a];
      while (q >= 0 && key[ord[q]] > kv) {
        ord[q + 1] = ord[q];
        --q;
      }
      ord[q + 1] = a;
    }
    for (int a = 0; a < n; ++a) {
      t.pair[r0 + a] = pr[ord[a]];
      t.cpack[r0 + a] = cp[ord[a]];
    }
    return;
  }
  for (int a = r0 + 1; a < r1; ++a) {
    const int2 pv = t.pair[a];
    const int cv = t.cpack[a];
    const int kv = t.found[a];
    int q = a - 1;
    while (q >= r0) {
      const int kq = t.found[q];
      if (kq < kv || (kq == kv && (unsigned)t.cpack[q] <= (unsigned)cv)) break;
      t.pair[q + 1] = t.pair[q];
      t.cpack[q + 1] = t.cpack[q];
      t.found[q + 1] = kq;
      --q;
    }
    t.pair[q + 1] = pv;
    t.cpack[q + 1] = cv;
    t.found[q + 1] = kv;
  }
}

// After the row sort: t.found[r] = the id of body 1 of row r (the down lists' key).
__global__ void k_rowkey(Table t, const int *__restrict__ id) {
  const long long k = (long long)blockIdx.x * kT + threadIdx.x;
  if (k < t.P) t.found[k] = id[t.pair[k].x];
}

// Down lists: every row is entered in the list of its body 2 (dfill zeroed), at a
// position the atomics pick; k_downsort then fixes the order.
__global__ void k_downfill(Table t, int *dfill) {
  const long long k = (long long)blockIdx.x * kT + threadIdx.x;
  if (k >= t.P) return;
  const int j = t.pair[k].y;
  const int e = t.down_start[j] + atomicAdd(&dfill[j], 1);
  if (e < t.down_start[j + 1]) t.down[e] = (int)k;
}

// Mixed precision: the reference branch vector of every row at this run,
// x2 + Href c - x1 formed in FP64 and rounded once to FP32.  A pass of its own over
// the rows (one row per thread) rather than inside the emit walk, where each thread
// meets its candidates at different iterations and the FP64 work would issue for a
// lane or two at a time.
__global__ void k_ref_branch(Table t, Bodies b, const Grid *__restrict__ grids, int multi) {
  const long long k = (long long)blockIdx.x * kT + threadIdx.x;
  if (k >= t.P) return;
  const int2 pr = t.pair[k];
  const Grid &g = grid_of(grids, b.sid, multi, pr.x);
  const double4_32a p1 = b.pos[pr.x], p2 = b.pos[pr.y];
  double h[3] = {0, 0, 0};
  const int cp = g.periodic ? t.cpack[k] : 0;
  // rows inside the cell have c = 0 and H c = 0 exactly: a warp none of whose rows
  // crosses the cell skips the conversions and products (FP64-pipe instructions)
  if (__any_sync(__activemask(), cp != 0) && g.periodic) {
    int c0, c1, c2;
    unpack_shift(cp, c0, c1, c2);
    h[0] = g.L[0] * c0; h[1] = g.L[1] * c1; h[2] = g.L[2] * c2;
    if (g.sheared)   // Href c of a sheared cell
      for (int q = 0; q < 3; ++q) h[q] = g.H[3 * q] * c0 + g.H[3 * q + 1] * c1 + g.H[3 * q + 2] * c2;
  }
  const double gx = (p2.x + h[0]) - p1.x, gy = (p2.y + h[1]) - p1.y, gz = (p2.z + h[2]) - p1.z;
  t.g32[k] = make_float4((float)gx, (float)gy, (float)gz, 0.0f);
  // the squared gap of the reference configuration, in FP64 before any rounding: the
  // mixed kernel's penetration is this minus the FP32 terms of the offsets, so it keeps
  // FP32's relative precision of the gap rather than of the branch length
  const double R = p1.w + p2.w;
  t.s0[k] = (float)(R * R - (gx * gx + gy * gy + gz * gz));
}

// the down lists were filled in atomic order: sort each body's list by (id of body 1,
// row); rows of one body 1 are ordered by shift within its range already.  Keys come
// from t.found (k_rowkey); short lists are sorted in registers and local memory.
__global__ void k_downsort(Table t, long long N) {
  long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= N) return;
  const int e0 = t.down_start[sl], e1 = t.down_start[sl + 1], n = e1 - e0;
  if (n < 2) return;
  if (n <= kSortLocal) {
    long long key[kSortLocal];   // (id of body 1) << 32 | row
    for (int a = 0; a < n; ++a) {
      const int v = t.down[e0 + a];
      key[a] = ((long long)t.found[v] << 32) | (long long)(unsigned)v;
    }
    for (int a = 1; a < n; ++a) {
      const long long kv = key[a];
      int q = a - 1;
      while (q >= 0 && key[q] > kv) {
        key[q + 1] = key[q];
        --q;
      }
      key[q + 1] = kv;
    }
    for (int a = 0; a < n; ++a) t.down[e0 + a] = (int)(unsigned)(key[a] & 0xffffffffLL);
    return;
  }
  for (int a = e0 + 1; a < e1; ++a) {
    const int v = t.down[a];
    const int kv = t.found[v];
    int b = a - 1;
    while (b >= e0) {
      const int u = t.down[b];
      const int ku = t.found[u];
      if (ku < kv || (ku == kv && u < v)) break;
      t.down[b + 1] = u;
      --b;
    }
    t.down[b + 1] = v;
  }
}

// Integration order: bodies grouped by their number of incident rows, largest
// first, so that the lanes of a warp walk row lists of about the same length
// (the per-body sum is a loop whose trip count is the warp's longest list).  The
// order inside a group is left to the atomics: it changes no result, only which
// lane integrates which body.  Bucket of a body: 63 - min(rows, 63).
__device__ inline int degree_bucket(const Table &t, int s) {
  const int d = (t.row_start[s + 1] - t.row_start[s]) + (t.down_start[s + 1] - t.down_start[s]);
  return kDegreeBuckets - 1 - (d < kDegreeBuckets - 1 ? d : kDegreeBuckets - 1);
}

// Degree order within chunks of kChunk consecutive slots: each chunk's bodies by
// decreasing row count, the chunk itself staying where it is.  The lanes of a warp
// get bodies of about the same row count (so their row walks end together) while
// the bodies a block touches stay spatial neighbours (slot order is Morton order),
// so their records and rows are fetched once into L2 instead of from all over the
// arrays.
constexpr int kChunk = 1024;
__global__ void __launch_bounds__(kChunk) k_degree_chunk(Table t, long long N) {
  __shared__ int cnt[kDegreeBuckets], base[kDegreeBuckets];
  if (threadIdx.x < kDegreeBuckets) cnt[threadIdx.x] = 0;
  __syncthreads();
  const long long c0 = (long long)blockIdx.x * kChunk, sl = c0 + threadIdx.x;
  int b = -1, local = 0;
  if (sl < N) {
    b = degree_bucket(t, (int)sl);
    local = atomicAdd(&cnt[b], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int i = 0; i < kDegreeBuckets; ++i) {
      base[i] = acc;
      acc += cnt[i];
    }
  }
  __syncthreads();
  if (b >= 0) t.ord[c0 + base[b] + local] = (int)sl;
}

__global__ void k_merge(Table nt, Table ot, long long N_old, const int *__restrict__ new_to_old,
                        int mixed) {
  long long k = (long long)blockIdx.x * kT + threadIdx.x;
  if (k >= nt.P) return;
  const int2 pr = nt.pair[k];
  const int cp = nt.cpack[k];
  const int o1 = new_to_old[pr.x], o2 = new_to_old[pr.y];
  // both tables orient a pair by id (ids survive a collider run, or shift by the same
  // amount within a sub-scene), so the old row is in the old range of body 1
  long long hit = -1;
  if (o1 < N_old && o2 < N_old && ot.P > 0) {
    for (int r = ot.row_start[o1]; r < ot.row_start[o1 + 1]; ++r)
      if (ot.pair[r].y == o2 && ot.cpack[r] == cp) { hit = r; break; }
  }
  const double sg = 1.0;
  if (mixed) {
    double4_32a fs = make_double4_32a(0, 0, 0, 0);
    float4 hn = make_float4(0, 0, 0, 0);
    float kn = 0.0f;
    if (hit >= 0) {
      kn = ot.g32[hit].w;
      if (kn != 0.0f) {
        const double4_32a ofs = ot.hfs[hit];
        const float4 ohn = ot.hn32[hit];
        const float sf = (float)sg;
        fs = make_double4_32a(sg * ofs.x, sg * ofs.y, sg * ofs.z, ofs.w);
        hn = make_float4(sf * ohn.x, sf * ohn.y, sf * ohn.z, ohn.w);
        ot.found[hit] = 1;
      }
    }
    const float4 gref = nt.g32[k];
    nt.g32[k] = make_float4(gref.x, gref.y, gref.z, kn);
    nt.hfs[k] = fs;
    nt.hn32[k] = hn;
    nt.oFM32[2 * k] = make_float4(0, 0, 0, 0);
    nt.oFM32[2 * k + 1] = make_float4(0, 0, 0, 0);
    return;
  }
  double4_32a fs = make_double4_32a(0, 0, 0, 0), hn = make_double4_32a(0, 0, 0, 0);
  double tp = 0;
  if (hit >= 0) {
    double4_32a ofs = ot.hfs[hit];
    if (ofs.w != 0.0) {
      double4_32a ohn = ot.hn[hit];
      fs = make_double4_32a(sg * ofs.x, sg * ofs.y, sg * ofs.z, ofs.w);
      hn = make_double4_32a(sg * ohn.x, sg * ohn.y, sg * ohn.z, ohn.w);
      tp = ot.tanphi[hit];
      ot.found[hit] = 1;
    }
  }
  nt.hfs[k] = fs;
  nt.hn[k] = hn;
  nt.tanphi[k] = tp;
  nt.oFM[2 * k] = make_double4_32a(0, 0, 0, 0);
  nt.oFM[2 * k + 1] = make_double4_32a(0, 0, 0, 0);
}

// A real row of the previous table that no candidate carried over: an error only
// if the pair still overlaps at the positions of this collider run (a pair that
// separated within the step is dropped by the contact law anyway; a body may move
// farther than the sweep margin in the step that triggers the run).  ob: the body
// buffer in the old slot order, still holding the current positions.
__global__ void k_lost(Table ot, Bodies ob, const Grid *__restrict__ grids, int multi, int *err,
                       int mixed) {
  long long r = (long long)blockIdx.x * kT + threadIdx.x;
  if (r >= ot.P) return;
  const bool real = mixed ? (ot.g32[r].w != 0.0f) : (ot.hfs[r].w != 0.0);
  if (!real || ot.found[r]) return;
  const int2 pr = ot.pair[r];
  const double4_32a p1 = ob.pos[pr.x], p2 = ob.pos[pr.y];
  const Grid &g = grid_of(grids, ob.sid, multi, pr.x);
  double h[3] = {0, 0, 0};
  if (g.periodic) {
    int c0, c1, c2;
    unpack_shift(ot.cpack[r], c0, c1, c2);
    for (int k = 0; k < 3; ++k) h[k] = g.H[3 * k] * c0 + g.H[3 * k + 1] * c1 + g.H[3 * k + 2] * c2;
  }
  const double dx = (p2.x + h[0]) - p1.x, dy = (p2.y + h[1]) - p1.y, dz = (p2.z + h[2]) - p1.z;
  const double R = p1.w + p2.w;
  if (dx * dx + dy * dy + dz * dz < R * R) atomicOr(err, kErrHistoryLost);
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

void launch_bbox_sub(const Bodies &b, long long N, int cap, unsigned long long *keys,
                     int nsm, cudaStream_t st) {
  if (N <= 0) return;
  const long long need = (N + kT - 1) / kT;
  const long long lim = (long long)nsm * 4;
  k_bbox_sub<<<(unsigned)(need < lim ? need : lim), kT, 0, st>>>(b.pos, b.sid, N, cap, keys);
}

void launch_bin(const Bodies &b, long long N, const Grid *grids, int multi, uint32_t dead,
                uint32_t *key, int *count, cudaStream_t st) {
  if (N > 0) k_bin<<<blocks(N), kT, 0, st>>>(b.pos, b.sid, N, grids, multi, dead, key, count);
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
                    const int *new_to_old, int *slot_of_id, int has_walls, int mixed,
                    const int *id_shift, cudaStream_t st) {
  if (N > 0)
    k_reorder<<<blocks(N), kT, 0, st>>>(src, dst, N, cap, new_to_old, slot_of_id, has_walls,
                                        mixed, id_shift);
}

void launch_cellrec(const Bodies &b, long long N, const Grid *grids, int multi, float4 *wpos,
                    int4 *info, cudaStream_t st) {
  if (N > 0) k_cellrec<<<blocks(N), kT, 0, st>>>(b.pos, b.sid, N, grids, multi, CellRec{wpos, info});
}

void launch_count(float4 *wpos, int4 *info, const int *sid, const int *id, long long N,
                  const Grid *grids, int multi, const int *count, const int *start, int *cnt_up,
                  int *cnt_down, int *err, CandList cl, cudaStream_t st) {
  if (N > 0)
    k_count<<<blocks(N), kT, 0, st>>>(CellRec{wpos, info}, sid, id, N, grids, multi, count, start,
                                      cnt_up, cnt_down, err, cl);
}

void launch_emit(float4 *wpos, int4 *info, const Bodies &b, long long N, const Grid *grids,
                 int multi, const int *count, const int *start, const Table &t, int *ufill,
                 int *dfill, CandList cl, cudaStream_t st) {
  if (N <= 0) return;
  k_emit<<<blocks(N), kT, 0, st>>>(CellRec{wpos, info}, b, N, grids, multi, count, start, t,
                                   ufill, cl);
  k_rowsort<<<blocks(N), kT, 0, st>>>(t, N);
  if (t.P > 0) {
    k_rowkey<<<blocks(t.P), kT, 0, st>>>(t, b.id);
    k_downfill<<<blocks(t.P), kT, 0, st>>>(t, dfill);
  }
}

void launch_ref_branch(const Table &t, const Bodies &b, const Grid *grids, int multi,
                       cudaStream_t st) {
  if (t.P > 0) k_ref_branch<<<blocks(t.P), kT, 0, st>>>(t, b, grids, multi);
}

void launch_downsort(const Table &t, const int *id, long long N, cudaStream_t st) {
  (void)id;   // the keys are in t.found (k_rowkey)
  if (N > 0) k_downsort<<<blocks(N), kT, 0, st>>>(t, N);
}

void launch_degree_order(const Table &t, long long N, int *ws, cudaStream_t st) {
  if (N <= 0) return;
  (void)ws;
  k_degree_chunk<<<(unsigned)((N + kChunk - 1) / kChunk), kChunk, 0, st>>>(t, N);
}

void launch_merge(const Table &nt, const Table &ot, long long N_old, const int *new_to_old,
                  int mixed, cudaStream_t st) {
  if (nt.P > 0) k_merge<<<blocks(nt.P), kT, 0, st>>>(nt, ot, N_old, new_to_old, mixed);
}

namespace {
// Cell flip (section 2.1.6, fig. 6): H' = H M keeps every image when each row's
// shift becomes c' = M^-1 c.  Pass 0 records the largest |c'| component of the rows
// of sub-scene `sub` (all rows without sub-scenes); pass 1 rewrites them.
__global__ void k_flip_shift(Table t, const int *__restrict__ sid, int multi, int sub, int3 m0,
                             int3 m1, int3 m2, int *maxabs, int apply) {
  for (long long k = (long long)blockIdx.x * kT + threadIdx.x; k < t.P;
       k += (long long)gridDim.x * kT) {
    if (multi && sid[t.pair[k].x] != sub) continue;
    int c0, c1, c2;
    unpack_shift(t.cpack[k], c0, c1, c2);
    const int n0 = m0.x * c0 + m0.y * c1 + m0.z * c2;
    const int n1 = m1.x * c0 + m1.y * c1 + m1.z * c2;
    const int n2 = m2.x * c0 + m2.y * c1 + m2.z * c2;
    if (apply) {
      t.cpack[k] = pack_shift(n0, n1, n2);
    } else {
      const int m = max(abs(n0), max(abs(n1), abs(n2)));
      if (m > kShiftMax) atomicMax(maxabs, m);
    }
  }
}
}  // namespace

void launch_flip_shift(const Table &t, const int *sid, int multi, int sub, const int Minv[9],
                       int *maxabs, int apply, cudaStream_t st) {
  if (t.P <= 0) return;
  const long long b = std::min<long long>(blocks(t.P), 4096);
  k_flip_shift<<<(unsigned)b, kT, 0, st>>>(t, sid, multi, sub, make_int3(Minv[0], Minv[1], Minv[2]),
                                          make_int3(Minv[3], Minv[4], Minv[5]),
                                          make_int3(Minv[6], Minv[7], Minv[8]), maxabs, apply);
}

void launch_lost(const Table &ot, const Bodies &ob, const Grid *grids, int multi, int *err,
                 int mixed, cudaStream_t st) {
  if (ot.P > 0) k_lost<<<blocks(ot.P), kT, 0, st>>>(ot, ob, grids, multi, err, mixed);
}

}  // namespace dem
