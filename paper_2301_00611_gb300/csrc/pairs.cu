// Bare collider query: all pairs of spheres closer than r_i + r_j + margin in a
// caller-provided configuration (device arrays in, device arrays out) -- the
// collision detection of section 2.1.1 (both passes: bounding-volume filter,
// then the exact sphere test) without a scene.
//
// Same grid as the scene collider: spheres are binned by Morton cell, sorted
// by a counting sort, and each one scans the forward half of its 27-cell
// neighbourhood.  The FP32 candidate test only filters; the kept pairs pass the
// exact FP64 test |x_j + H c - x_i| < (r_i + r_j) + margin, evaluated with
// round-to-nearest operations in the order written (shift, branch vector,
// squared length left to right), in the orientation i < j of the caller's
// indices, so the result is bit-for-bit the set that definition gives.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dem_internal.cuh"
#include "grid.cuh"
#include "dem.h"

namespace dem {

namespace {
constexpr int kT = 256;

inline unsigned blocks(long long n) { return (unsigned)((n + kT - 1) / kT); }

// positions + radii into one record; per-block extent (min x, max x per axis, max r)
__global__ void k_pack(const double *__restrict__ pos, const double *__restrict__ rad, long long n,
                       double4_32a *out, double *partials, int *err) {
  __shared__ double sh[7][kT];
  double v[7] = {1e300, 1e300, 1e300, -1e300, -1e300, -1e300, 0};
  for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2], r = rad[i];
    if (!(r > 0) || !isfinite(x + y + z + r)) atomicOr(err, 1);
    out[i] = make_double4_32a(x, y, z, r);
    v[0] = fmin(v[0], x); v[1] = fmin(v[1], y); v[2] = fmin(v[2], z);
    v[3] = fmax(v[3], x); v[4] = fmax(v[4], y); v[5] = fmax(v[5], z);
    v[6] = fmax(v[6], r);
  }
  for (int q = 0; q < 7; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = fmin(sh[q][threadIdx.x], sh[q][threadIdx.x + o]);
      for (int q = 3; q < 7; ++q) sh[q][threadIdx.x] = fmax(sh[q][threadIdx.x], sh[q][threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 7; ++q) partials[7 * blockIdx.x + q] = sh[q][0];
}

__global__ void k_bin_q(const double4_32a *__restrict__ p, long long n, Grid g, uint32_t *key,
                        int *count) {
  long long i = (long long)blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  const double4_32a q = p[i];
  int c[3], img[3];
  cell_of(g, q.x, q.y, q.z, c, img);
  const uint32_t m = morton3(c[0], c[1], c[2]);
  key[i] = m;
  atomicAdd(&count[m], 1);
}

__global__ void k_scatter_q(long long n, const uint32_t *__restrict__ key,
                            const int *__restrict__ start, int *fill, int *order) {
  long long i = (long long)blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  const uint32_t m = key[i];
  order[start[m] + atomicAdd(&fill[m], 1)] = (int)i;
}

// cells sorted by index: the atomics above left the order inside a cell open
__global__ void k_cellsort_q(const int *__restrict__ count, const int *__restrict__ start,
                             long long ncell, int *order) {
  long long m = (long long)blockIdx.x * kT + threadIdx.x;
  if (m >= ncell) return;
  const int cnt = count[m];
  if (cnt < 2) return;
  const int s0 = start[m];
  for (int a = s0 + 1; a < s0 + cnt; ++a) {
    const int v = order[a];
    int b = a - 1;
    while (b >= s0 && order[b] > v) {
      order[b + 1] = order[b];
      --b;
    }
    order[b + 1] = v;
  }
}

__global__ void k_sorted_rec(const double4_32a *__restrict__ p, const int *__restrict__ order,
                             long long n, Grid g, double4_32a *sp, CellRec cr) {
  long long s = (long long)blockIdx.x * kT + threadIdx.x;
  if (s >= n) return;
  const double4_32a q = p[order[s]];
  sp[s] = q;
  int c[3], img[3];
  cell_of(g, q.x, q.y, q.z, c, img);
  const double x[3] = {q.x, q.y, q.z};
  float f[3];
  for (int k = 0; k < 3; ++k)
    f[k] = g.periodic ? (float)(x[k] - g.L[k] * img[k]) : (float)(x[k] - g.lo[k]);
  cr.wpos[s] = make_float4(f[0], f[1], f[2], (float)q.w);
  cr.info[s] = make_int4(c[0] | (c[1] << 10) | (c[2] << 20), img[0], img[1], img[2]);
}

// exact test in the caller's orientation (a has the lower index), shift c of b
__device__ inline bool exact_pair(const double4_32a &a, const double4_32a &b, const int c[3],
                                  const Grid &g, double margin) {
  double h0 = 0, h1 = 0, h2 = 0;
  if (g.periodic) {
    h0 = __dmul_rn(g.L[0], (double)c[0]);
    h1 = __dmul_rn(g.L[1], (double)c[1]);
    h2 = __dmul_rn(g.L[2], (double)c[2]);
  }
  const double d0 = __dsub_rn(__dadd_rn(b.x, h0), a.x);
  const double d1 = __dsub_rn(__dadd_rn(b.y, h1), a.y);
  const double d2 = __dsub_rn(__dadd_rn(b.z, h2), a.z);
  const double l2 = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
  const double R = __dadd_rn(__dadd_rn(a.w, b.w), margin);
  return l2 < __dmul_rn(R, R);
}

template <bool Emit>
__global__ void k_pairs(const double4_32a *__restrict__ sp, const int *__restrict__ order,
                        CellRec cr, long long n, Grid g, const int *__restrict__ count,
                        const int *__restrict__ start, double margin, int *cnt,
                        const int *__restrict__ off, long long cap, int *I, int *J, int *C) {
  long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= n) return;
  const int s = (int)sl;
  const float4 a = cr.wpos[s];
  const int4 inf = cr.info[s];
  int ci[3];
  ci[0] = inf.x & 1023; ci[1] = (inf.x >> 10) & 1023; ci[2] = (inf.x >> 20) & 1023;
  const int is = order[s];
  long long out = Emit ? (long long)off[s] : 0;
  int k = 0;
  for_half_shell(g, count, start, ci, s, [&](int j, const int w[3]) {
    if (!cand_f32(g, a, cr.wpos[j], w, g.slack)) return;
    int c[3] = {0, 0, 0};
    if (g.periodic) {
      const int4 ij = cr.info[j];
      c[0] = inf.y - ij.y + w[0]; c[1] = inf.z - ij.z + w[1]; c[2] = inf.w - ij.w + w[2];
    }
    const int ij_ = order[j];
    const bool fwd = is < ij_;
    if (!fwd) { c[0] = -c[0]; c[1] = -c[1]; c[2] = -c[2]; }
    const bool keep = fwd ? exact_pair(sp[s], sp[j], c, g, margin) : exact_pair(sp[j], sp[s], c, g, margin);
    if (!keep) return;
    if (Emit) {
      const long long r = out + k;
      if (r < cap) {
        I[r] = fwd ? is : ij_;
        J[r] = fwd ? ij_ : is;
        if (C) { C[3 * r] = c[0]; C[3 * r + 1] = c[1]; C[3 * r + 2] = c[2]; }
      }
    }
    ++k;
  });
  if (!Emit) cnt[s] = k;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// bounded wait on the caller's stream (DEM_TIMEOUT_S, default 120 s)
cudaError_t bounded_wait(cudaStream_t st, bool *timed_out) {
  *timed_out = false;
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(ev, st);
  if (e != cudaSuccess) { cudaEventDestroy(ev); return e; }
  const char *env = std::getenv("DEM_TIMEOUT_S");
  double lim = env ? std::atof(env) : 120.0;
  if (!(lim > 0)) lim = 120.0;
  const double deadline = now_s() + lim;
  while (true) {
    e = cudaEventQuery(ev);
    if (e != cudaErrorNotReady) break;
    if (now_s() > deadline) { *timed_out = true; break; }
    std::this_thread::yield();
  }
  cudaEventDestroy(ev);
  return e == cudaErrorNotReady ? cudaSuccess : e;
}
}  // namespace

// Grid of a pair query: cell edge >= 2 r_max + margin, at most max_side cells per axis.
dem_status pair_grid(int periodic, const double *H, const double lo[3], const double hi[3],
                     double rmax, double margin, Grid &g, std::string &err,
                     int max_side = kMaxGridSide) {
  const double hmin = 2 * rmax + margin;
  g = Grid{};
  g.periodic = periodic;
  g.reach = margin;
  double ext = 0;
  for (int k = 0; k < 3; ++k) {
    if (periodic) {
      const double L = H[4 * k];
      const int n = (int)std::floor(L / hmin);
      if (n < 3) {
        err = "periodic cell edge shorter than 3 * (2 r_max + margin)";
        return DEM_ERR_GEOMETRY;
      }
      g.n[k] = std::min(n, max_side);
      g.L[k] = L;
      g.scale[k] = 1.0 / L;
      ext = std::max(ext, L);
    } else {
      const double e = std::max(hi[k] - lo[k] + 2 * rmax, hmin);
      const int n = std::max(1, std::min((int)std::floor(e / hmin), max_side));
      g.n[k] = n;
      g.lo[k] = lo[k] - rmax;
      g.scale[k] = n / e;
      ext = std::max(ext, e);
    }
    g.Lf[k] = (float)g.L[k];
  }
  g.reachf = (float)margin;
  g.slack = (float)(8.0 * ext * std::ldexp(1.0, -23) + 1e-5 * hmin);
  unsigned B = 1;
  while ((int)B < std::max(g.n[0], std::max(g.n[1], g.n[2]))) B <<= 1;
  g.B = (int)B;
  g.base = 0;
  g.morton = 1;
  return DEM_OK;
}

// Scratch of one query, carved from caller-chosen memory (see pairs_run).
struct PairScratch {
  double4_32a *packed, *sorted;
  double *partials;
  uint32_t *key;
  int *count, *start, *fill, *order, *cnt, *off, *err, *ws;
  float4 *wpos;
  int4 *info;
};

size_t pair_scratch_bytes(long long n, long long ncell) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  long long nb = std::min<long long>(1024, std::max<long long>(1, (n + kT - 1) / kT));
  size_t b = 0;
  b += 2 * up(sizeof(double4_32a) * n);
  b += up(sizeof(double) * 7 * nb);
  b += up(sizeof(uint32_t) * n);
  b += up(sizeof(int) * ncell) + up(sizeof(int) * (ncell + 1)) + up(sizeof(int) * ncell);
  b += up(sizeof(int) * n) * 2 + up(sizeof(int) * (n + 1)) + up(sizeof(int) * 4);
  b += up(scan_workspace_bytes(std::max<long long>(ncell + 1, n + 1)));
  b += up(sizeof(float4) * n) + up(sizeof(int4) * n);
  return b;
}

PairScratch carve(char *base, long long n, long long ncell) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  long long nb = std::min<long long>(1024, std::max<long long>(1, (n + kT - 1) / kT));
  PairScratch s{};
  char *p = base;
  s.packed = (double4_32a *)p; p += up(sizeof(double4_32a) * n);
  s.sorted = (double4_32a *)p; p += up(sizeof(double4_32a) * n);
  s.partials = (double *)p; p += up(sizeof(double) * 7 * nb);
  s.key = (uint32_t *)p; p += up(sizeof(uint32_t) * n);
  s.count = (int *)p; p += up(sizeof(int) * ncell);
  s.start = (int *)p; p += up(sizeof(int) * (ncell + 1));
  s.fill = (int *)p; p += up(sizeof(int) * ncell);
  s.order = (int *)p; p += up(sizeof(int) * n);
  s.cnt = (int *)p; p += up(sizeof(int) * n);
  s.off = (int *)p; p += up(sizeof(int) * (n + 1));
  s.err = (int *)p; p += up(sizeof(int) * 4);
  s.ws = (int *)p; p += up(scan_workspace_bytes(std::max<long long>(ncell + 1, n + 1)));
  s.wpos = (float4 *)p; p += up(sizeof(float4) * n);
  s.info = (int4 *)p;
  return s;
}

// First phase of a query: pack the inputs and measure their extent.  Returns the
// number of extent partials written to host[] (7 per block).
int pairs_extent(const double *pos, const double *rad, long long n, const PairScratch &S,
                 cudaStream_t st) {
  const int nb = (int)std::min<long long>(1024, std::max<long long>(1, (n + kT - 1) / kT));
  k_pack<<<nb, kT, 0, st>>>(pos, rad, n, S.packed, S.partials, S.err);
  return nb;
}

// Launches of the second phase (bin, sort, count, scan, emit) on zeroed counters.
dem_status pairs_run_nowait(long long n, const Grid &g, double margin, const PairScratch &S,
                            long long cap, int *I, int *J, int *C, cudaStream_t st) {
  const long long ncell = (long long)g.B * g.B * g.B;
  k_bin_q<<<blocks(n), kT, 0, st>>>(S.packed, n, g, S.key, S.count);
  exclusive_scan(S.count, S.start, ncell, S.ws, st);
  k_scatter_q<<<blocks(n), kT, 0, st>>>(n, S.key, S.start, S.fill, S.order);
  k_cellsort_q<<<blocks(ncell), kT, 0, st>>>(S.count, S.start, ncell, S.order);
  CellRec cr{S.wpos, S.info};
  k_sorted_rec<<<blocks(n), kT, 0, st>>>(S.packed, S.order, n, g, S.sorted, cr);
  k_pairs<false><<<blocks(n), kT, 0, st>>>(S.sorted, S.order, cr, n, g, S.count, S.start, margin,
                                           S.cnt, nullptr, 0, nullptr, nullptr, nullptr);
  exclusive_scan(S.cnt, S.off, n, S.ws, st);
  k_pairs<true><<<blocks(n), kT, 0, st>>>(S.sorted, S.order, cr, n, g, S.count, S.start, margin,
                                          nullptr, S.off, cap, I, J, C);
  return cudaGetLastError() == cudaSuccess ? DEM_OK : DEM_ERR_CUDA;
}

// Second phase: bin, sort, count, scan, emit.  *total receives the pair count.
dem_status pairs_run(long long n, const Grid &g, double margin, const PairScratch &S,
                     long long cap, int *I, int *J, int *C, long long *total, cudaStream_t st,
                     std::string &err) {
  const long long ncell = (long long)g.B * g.B * g.B;
  cudaMemsetAsync(S.count, 0, sizeof(int) * ncell, st);
  cudaMemsetAsync(S.fill, 0, sizeof(int) * ncell, st);
  k_bin_q<<<blocks(n), kT, 0, st>>>(S.packed, n, g, S.key, S.count);
  exclusive_scan(S.count, S.start, ncell, S.ws, st);
  k_scatter_q<<<blocks(n), kT, 0, st>>>(n, S.key, S.start, S.fill, S.order);
  k_cellsort_q<<<blocks(ncell), kT, 0, st>>>(S.count, S.start, ncell, S.order);
  CellRec cr{S.wpos, S.info};
  k_sorted_rec<<<blocks(n), kT, 0, st>>>(S.packed, S.order, n, g, S.sorted, cr);
  k_pairs<false><<<blocks(n), kT, 0, st>>>(S.sorted, S.order, cr, n, g, S.count, S.start, margin,
                                           S.cnt, nullptr, 0, nullptr, nullptr, nullptr);
  exclusive_scan(S.cnt, S.off, n, S.ws, st);
  k_pairs<true><<<blocks(n), kT, 0, st>>>(S.sorted, S.order, cr, n, g, S.count, S.start, margin,
                                          nullptr, S.off, cap, I, J, C);
  // wait (bounded) for the kernels first: a device-to-pageable copy returns only
  // once it is done, so issued before the wait it would block without a limit
  cudaError_t e = cudaGetLastError();
  bool to = false;
  if (e == cudaSuccess) e = bounded_wait(st, &to);
  if (to) { err = "timed out waiting for the GPU"; return DEM_ERR_TIMEOUT; }
  int tot = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, S.off + n, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { err = std::string("pair query: ") + cudaGetErrorString(e); return DEM_ERR_CUDA; }
  *total = tot;
  return DEM_OK;
}

// Host side of the first phase: wait for the extent, reduce it, check the inputs.
dem_status pairs_extent_host(const PairScratch &S, int nb, double *host7, double lo[3],
                             double hi[3], double *rmax, cudaStream_t st, std::string &err) {
  int bad = 0;
  // the bounded wait comes before the copies to pageable memory (which would block)
  cudaError_t e = cudaGetLastError();
  bool to = false;
  if (e == cudaSuccess) e = bounded_wait(st, &to);
  if (to) { err = "timed out waiting for the GPU"; return DEM_ERR_TIMEOUT; }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host7, S.partials, sizeof(double) * 7 * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, S.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { err = std::string("pair query: ") + cudaGetErrorString(e); return DEM_ERR_CUDA; }
  if (bad) { err = "non-finite position or non-positive radius"; return DEM_ERR_NONFINITE; }
  for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
  *rmax = 0;
  for (int b = 0; b < nb; ++b) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], host7[7 * b + k]);
      hi[k] = std::max(hi[k], host7[7 * b + 3 + k]);
    }
    *rmax = std::max(*rmax, host7[7 * b + 6]);
  }
  return DEM_OK;
}

}  // namespace dem

namespace dem {
void set_global_error(const std::string &msg);
}

using namespace dem;

extern "C" dem_status dem_find_pairs(const double *pos_dev, const double *radius_dev, long long n,
                                     int periodic, const double *cell_h, double margin,
                                     long long cap, int *id1_dev, int *id2_dev,
                                     int *cell_dist_dev, long long *count, void *cuda_stream) {
  std::string err;
  auto fail = [&](dem_status c, const std::string &m) { set_global_error(m); return c; };
  if (!count || n < 0 || cap < 0 || !(margin >= 0) || (n > 0 && (!pos_dev || !radius_dev)) ||
      (cap > 0 && (!id1_dev || !id2_dev)))
    return fail(DEM_ERR_INVALID_ARG, "bad pair-query arguments");
  if (periodic && (!cell_h || cell_h[1] != 0 || cell_h[2] != 0 || cell_h[3] != 0 ||
                   cell_h[5] != 0 || cell_h[6] != 0 || cell_h[7] != 0 || !(cell_h[0] > 0) ||
                   !(cell_h[4] > 0) || !(cell_h[8] > 0)))
    return fail(DEM_ERR_INVALID_ARG, "the periodic cell must be diagonal with positive edges");
  if (n > 0x7fffffffLL) return fail(DEM_ERR_CAPACITY, "more than 2^31-1 spheres");
  *count = 0;
  set_global_error("");
  if (n < 2) return DEM_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // phase 1: extent (scratch sized for the largest grid this n can need)
  const long long ncell_max = (long long)kMaxGridSide * kMaxGridSide * kMaxGridSide;
  (void)ncell_max;
  char *mem = nullptr;
  size_t bytes1 = pair_scratch_bytes(n, 1);
  if (cudaMallocAsync((void **)&mem, bytes1, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(DEM_ERR_OOM, "device allocation failed");
  }
  PairScratch S1 = carve(mem, n, 1);
  cudaMemsetAsync(S1.err, 0, sizeof(int), st);
  const int nb = pairs_extent(pos_dev, radius_dev, n, S1, st);
  std::vector<double> host7(7 * nb);
  double lo[3], hi[3], rmax = 0;
  dem_status r = pairs_extent_host(S1, nb, host7.data(), lo, hi, &rmax, st, err);
  if (r) { cudaFreeAsync(mem, st); return fail(r, err); }
  Grid g;
  if ((r = pair_grid(periodic, cell_h, lo, hi, rmax, margin, g, err))) {
    cudaFreeAsync(mem, st);
    return fail(r, err);
  }
  // phase 2: scratch for this grid; keep the packed inputs of phase 1
  const long long ncell = (long long)g.B * g.B * g.B;
  char *mem2 = nullptr;
  if (cudaMallocAsync((void **)&mem2, pair_scratch_bytes(n, ncell), st) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(mem, st);
    return fail(DEM_ERR_OOM, "device allocation failed");
  }
  PairScratch S = carve(mem2, n, ncell);
  cudaMemcpyAsync(S.packed, S1.packed, sizeof(double4_32a) * n, cudaMemcpyDeviceToDevice, st);
  long long total = 0;
  r = pairs_run(n, g, margin, S, cap, id1_dev, id2_dev, cell_dist_dev, &total, st, err);
  cudaFreeAsync(mem2, st);
  cudaFreeAsync(mem, st);
  if (r) return fail(r, err);
  *count = total;
  return DEM_OK;
}

// ---------------------------------------------------------------------------
// Pair query without allocation.
//
// The scratch of dem_find_pairs_noalloc lives in one file-scope device array
// of fixed size, present on every GPU that loads this library until the process
// exits.  Host code cannot pass the array's name to a kernel (in host code the
// name is only a host-side stand-in); the device address is fetched with
// cudaGetSymbolAddress once per device, with that device current, on the first
// call there.
namespace dem {
namespace {
constexpr long long kNoAllocMaxSpheres = 1LL << 16;   // 65,536 spheres
constexpr int kNoAllocMaxSide = 64;                     // grid cells per axis
constexpr long long kNoAllocMaxCells = (long long)kNoAllocMaxSide * kNoAllocMaxSide * kNoAllocMaxSide;
constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }
// the layout of carve() at the maximum sizes, with room for the scan workspace
constexpr size_t kNoAllocBytes =
    2 * up256(32 * kNoAllocMaxSpheres) + up256(8 * 7 * 1024) + up256(4 * kNoAllocMaxSpheres) +
    up256(4 * kNoAllocMaxCells) + up256(4 * (kNoAllocMaxCells + 1)) + up256(4 * kNoAllocMaxCells) +
    2 * up256(4 * kNoAllocMaxSpheres) + up256(4 * (kNoAllocMaxSpheres + 1)) + up256(16) +
    up256(16384) + up256(16 * kNoAllocMaxSpheres) + up256(16 * kNoAllocMaxSpheres);

__device__ __align__(256) unsigned char g_pairs_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_dev[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (set up on first use)
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pairs_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

// bounded wait that creates nothing: poll the stream until its work is done
cudaError_t bounded_stream_wait(cudaStream_t st, bool *timed_out) {
  *timed_out = false;
  const char *env = std::getenv("DEM_TIMEOUT_S");
  double lim = env ? std::atof(env) : 120.0;
  if (!(lim > 0)) lim = 120.0;
  const double deadline = now_s() + lim;
  while (true) {
    cudaError_t e = cudaStreamQuery(st);
    if (e != cudaErrorNotReady) return e;
    if (now_s() > deadline) { *timed_out = true; return cudaSuccess; }
    std::this_thread::yield();
  }
}
}  // namespace
}  // namespace dem

extern "C" dem_status dem_find_pairs_noalloc(const double *pos_dev, const double *radius_dev,
                                             long long n, int periodic, const double *cell_h,
                                             double margin, long long cap, int *id1_dev,
                                             int *id2_dev, int *cell_dist_dev, long long *count,
                                             void *cuda_stream) {
  std::string err;
  auto fail = [&](dem_status c, const std::string &m) { set_global_error(m); return c; };
  if (!count || n < 0 || cap < 0 || !(margin >= 0) || (n > 0 && (!pos_dev || !radius_dev)) ||
      (cap > 0 && (!id1_dev || !id2_dev)))
    return fail(DEM_ERR_INVALID_ARG, "bad pair-query arguments");
  if (periodic && (!cell_h || cell_h[1] != 0 || cell_h[2] != 0 || cell_h[3] != 0 ||
                   cell_h[5] != 0 || cell_h[6] != 0 || cell_h[7] != 0 || !(cell_h[0] > 0) ||
                   !(cell_h[4] > 0) || !(cell_h[8] > 0)))
    return fail(DEM_ERR_INVALID_ARG, "the periodic cell must be diagonal with positive edges");
  if (n > kNoAllocMaxSpheres)
    return fail(DEM_ERR_CAPACITY, "dem_find_pairs_noalloc takes at most 65536 spheres; use "
                                  "dem_find_pairs for larger configurations");
  *count = 0;
  set_global_error("");
  // set-up first (also for n < 2): the lookup loads this file's device module, and
  // with it the scratch array, on the current device
  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(DEM_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
  }
  if (n < 2) return DEM_OK;
  if (pair_scratch_bytes(n, kNoAllocMaxCells) > kNoAllocBytes)
    return fail(DEM_ERR_CAPACITY, "internal: pair-query scratch exceeds its static size");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // one layout for both phases, carved at the largest grid; the previous call's
  // contents are stale: the error word and the cell counters are cleared here
  PairScratch S = carve((char *)base, n, kNoAllocMaxCells);
  cudaMemsetAsync(S.err, 0, sizeof(int), st);
  const int nb = pairs_extent(pos_dev, radius_dev, n, S, st);
  double host7[7 * 256];
  int bad = 0;
  // poll (bounded) until the kernels are done, and only then copy to the host: a
  // device-to-pageable copy returns only once it is done, so it must not be the wait
  e = cudaGetLastError();
  bool to = false;
  if (e == cudaSuccess) e = bounded_stream_wait(st, &to);
  if (to) return fail(DEM_ERR_TIMEOUT, "timed out waiting for the GPU");
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host7, S.partials, sizeof(double) * 7 * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, S.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(DEM_ERR_CUDA, std::string("pair query: ") + cudaGetErrorString(e));
  if (bad) return fail(DEM_ERR_NONFINITE, "non-finite position or non-positive radius");
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double rmax = 0;
  for (int b = 0; b < nb; ++b) {
    for (int k = 0; k < 3; ++k) {
      lo[k] = std::min(lo[k], host7[7 * b + k]);
      hi[k] = std::max(hi[k], host7[7 * b + 3 + k]);
    }
    rmax = std::max(rmax, host7[7 * b + 6]);
  }
  Grid g;
  dem_status r = pair_grid(periodic, cell_h, lo, hi, rmax, margin, g, err, kNoAllocMaxSide);
  if (r) return fail(r, err);
  // pairs_run's own wait creates an event; the no-allocation path repeats its
  // launches with the polling wait instead
  const long long ncell = (long long)g.B * g.B * g.B;
  cudaMemsetAsync(S.count, 0, sizeof(int) * ncell, st);
  cudaMemsetAsync(S.fill, 0, sizeof(int) * ncell, st);
  long long total = 0;
  r = pairs_run_nowait(n, g, margin, S, cap, id1_dev, id2_dev, cell_dist_dev, st);
  if (r) return fail(r, "pair query launch failed");
  int tot = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = bounded_stream_wait(st, &to);
  if (to) return fail(DEM_ERR_TIMEOUT, "timed out waiting for the GPU");
  if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, S.off + n, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(DEM_ERR_CUDA, std::string("pair query: ") + cudaGetErrorString(e));
  total = tot;
  *count = total;
  return DEM_OK;
}
