// Exclusive prefix sum of int arrays (collider cell offsets, per-body CSR
// offsets).  Tile scan: each block scans 2048 items through shared memory
// (coalesced loads, per-thread serial scan of 8 items, warp-shuffle scan of
// the thread totals), block totals are scanned recursively and added back.
// out has n + 1 entries: out[n] is the total.  Deterministic (integers).
#include "dem_internal.cuh"

namespace dem {

namespace {
constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;

__global__ void __launch_bounds__(kThreads) k_scan_tile(const int *__restrict__ in,
                                                        int *__restrict__ out, long long n,
                                                        int *__restrict__ sums) {
  __shared__ int tile[kTile];
  __shared__ int warp_tot[kThreads / 32];
  const long long base = (long long)blockIdx.x * kTile;
  const int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    long long g = base + i * kThreads + t;
    tile[i * kThreads + t] = (g < n) ? in[g] : 0;
  }
  __syncthreads();
  int v[kItems];
  int run = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    v[i] = run;
    run += tile[t * kItems + i];
  }
  // inclusive warp scan of the per-thread totals
  const int lane = t & 31, wid = t >> 5;
  int x = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = (lane < kThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kThreads / 32) warp_tot[lane] = w;  // inclusive
  }
  __syncthreads();
  const int thread_off = (x - run) + (wid > 0 ? warp_tot[wid - 1] : 0);
#pragma unroll
  for (int i = 0; i < kItems; ++i) tile[t * kItems + i] = v[i] + thread_off;
  if (t == kThreads - 1) sums[blockIdx.x] = thread_off + run;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    long long g = base + i * kThreads + t;
    if (g < n) out[g] = tile[i * kThreads + t];
  }
}

__global__ void k_add_offsets(int *__restrict__ out, long long n, const int *__restrict__ off) {
  long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[g] += off[g / kTile];
}

__global__ void k_set_total(int *out, long long n, const int *total) { out[n] = *total; }

long long nblocks(long long n) { return (n + kTile - 1) / kTile; }
}  // namespace

size_t scan_workspace_bytes(long long n) {
  size_t bytes = 0;
  while (true) {
    long long nb = nblocks(n);
    bytes += (size_t)(2 * nb + 2) * sizeof(int);
    if (nb <= 1) break;
    n = nb;
  }
  return bytes + 256;
}

void exclusive_scan(const int *in, int *out, long long n, int *ws, cudaStream_t st) {
  if (n <= 0) {
    cudaMemsetAsync(out, 0, sizeof(int), st);
    return;
  }
  long long nb = nblocks(n);
  int *sums = ws;
  k_scan_tile<<<(unsigned)nb, kThreads, 0, st>>>(in, out, n, sums);
  if (nb == 1) {
    k_set_total<<<1, 1, 0, st>>>(out, n, sums);
    return;
  }
  int *scanned = ws + nb;              // nb + 1 entries
  exclusive_scan(sums, scanned, nb, ws + 2 * nb + 2, st);
  k_add_offsets<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, scanned);
  k_set_total<<<1, 1, 0, st>>>(out, n, scanned + nb);
}

}  // namespace dem
