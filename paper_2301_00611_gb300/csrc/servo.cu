// Reductions of the cell controllers over the contact table: the stress servo's sums
// (PeriTriaxController: sigma_aa V = sum F_a (-l n_a) and K_a V = sum kn (l n_a)^2,
// every globUpdate steps) and the Peri3dController's Love-Weber tensor
// (sum F_a (-l n_b), every step).  Both read each table row once and are bound by HBM:
// kServoBlocks blocks (two per SM of the 152-SM part) of kServoThreads threads stride
// over the rows, each thread loading the kn words of several rows (kRun for FP32
// tables, kRun / 2 for FP64) before any row's operands (so that many loads are in
// flight), and every block reduces in a fixed
// order (warp shuffles, then the warps in order) to one partial, which the cell
// advance sums in block order: the sums are the same from run to run.
//
// FP64 tables: every product and sum in FP64.  Mixed tables: the operands of a row
// (force, normal, the two branch lengths, kn) are FP32 values; their products are
// formed in FP32 and summed in FP32 over the kRun rows a thread takes at a time, and
// each such run sum is added to FP64 accumulators.  A run sum of the stiffness terms
// (all positive) carries at most (kRun + 3) FP32 units of relative error; the stress
// terms, at most that many units of the sum of their magnitudes.  Forming the same
// products in FP64 took about 25 FP64-pipe instructions per real row, which on this
// part made the pass FP64-pipe bound instead of HBM bound.
#include "dem_internal.cuh"

namespace dem {

namespace {
constexpr int kServoThreads = 512;
constexpr int kRun = 8;

template <int K>
__device__ inline void reduce_store(double (&v)[K], double *partials) {
  __shared__ double sh[K][kServoThreads / 32];
  for (int q = 0; q < K; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < K; ++q) sh[q][threadIdx.x >> 5] = v[q];
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0;
    for (int w = 0; w < kServoThreads / 32; ++w) s += sh[threadIdx.x][w];
    partials[K * blockIdx.x + threadIdx.x] = s;
  }
}

// kn of row k (0 for a row that is not a real contact)
__device__ inline float kn_mixed(const Table &t, long long k) {
  return reinterpret_cast<const float *>(t.g32)[4 * k + 3];
}
__device__ inline double kn_fp64(const Table &t, long long k) {
  return reinterpret_cast<const double *>(t.hfs)[4 * k + 3];
}

// Hertz-Mindlin tangent stiffness 3/2 kno pen^1/2 (pen from the FP64 radii)
__device__ inline double hertz_tangent(const Bodies &b, const Table &t, long long k,
                                       double kno, double l) {
  const int2 pr = t.pair[k];
  const double pen = (b.pos[pr.x].w + b.pos[pr.y].w) - l;
  return 1.5 * kno * sqrt(pen > 0 ? pen : 0.0);
}

// The products of one row, FP32 operands (mixed tables)
template <bool kHertz>
__device__ inline void servo_row_f32(const Table &t, const Bodies &b, long long k, float kn,
                                     float (&a)[6]) {
  const float4 f = t.oFM32[2 * k], m = t.oFM32[2 * k + 1], h = t.hn32[k];
  if (kHertz) kn = (float)hertz_tangent(b, t, k, kn, (double)f.w + (double)m.w);
  const float l = f.w + m.w;
  const float bl0 = l * h.x, bl1 = l * h.y, bl2 = l * h.z;
  a[0] -= f.x * bl0; a[1] -= f.y * bl1; a[2] -= f.z * bl2;
  a[3] += kn * (bl0 * bl0); a[4] += kn * (bl1 * bl1); a[5] += kn * (bl2 * bl2);
}

// The products of one row, FP64 operands
template <bool kHertz>
__device__ inline void servo_row_f64(const Table &t, const Bodies &b, long long k, double kn,
                                     double (&v)[6]) {
  const double4_32a f = t.oFM[2 * k], m = t.oFM[2 * k + 1], h = t.hn[k];
  const double l = f.w + m.w;
  if (kHertz) kn = hertz_tangent(b, t, k, kn, l);
  const double F[3] = {f.x, f.y, f.z}, n[3] = {h.x, h.y, h.z};
  for (int q = 0; q < 3; ++q) {
    v[q] += F[q] * (-l * n[q]);
    const double bl = l * n[q];
    v[3 + q] += kn * (bl * bl);
  }
}

template <bool kMixed, bool kHertz>
__global__ void __launch_bounds__(kServoThreads, 2)
k_servo_partials(Table t, Bodies b, const DevStatus *ds, double *partials) {
  constexpr int R = kMixed ? kRun : kRun / 2;   // rows whose kn words load together
  double v[6] = {0, 0, 0, 0, 0, 0};
  if (!ds->pending) {
    const long long stride = (long long)gridDim.x * kServoThreads;
    for (long long k0 = (long long)blockIdx.x * kServoThreads + threadIdx.x; k0 < t.P;
         k0 += R * stride) {
      if (kMixed) {
        float kn[R], a[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const long long k = k0 + j * stride;
          kn[j] = k < t.P ? kn_mixed(t, k) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (kn[j] != 0.0f) servo_row_f32<kHertz>(t, b, k0 + j * stride, kn[j], a);
        for (int q = 0; q < 6; ++q) v[q] += (double)a[q];
      } else {
        double kn[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const long long k = k0 + j * stride;
          kn[j] = k < t.P ? kn_fp64(t, k) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (kn[j] != 0.0) servo_row_f64<kHertz>(t, b, k0 + j * stride, kn[j], v);
      }
    }
  }
  reduce_store<6>(v, partials);
}

template <bool kMixed>
__global__ void __launch_bounds__(kServoThreads, 2)
k_p3d_partials(Table t, const DevStatus *ds, double *partials) {
  constexpr int R = kMixed ? kRun : kRun / 2;
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (!ds->pending) {
    const long long stride = (long long)gridDim.x * kServoThreads;
    for (long long k0 = (long long)blockIdx.x * kServoThreads + threadIdx.x; k0 < t.P;
         k0 += R * stride) {
      if (kMixed) {
        float kn[R], a[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const long long k = k0 + j * stride;
          kn[j] = k < t.P ? kn_mixed(t, k) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          if (kn[j] == 0.0f) continue;
          const long long k = k0 + j * stride;
          const float4 f = t.oFM32[2 * k], m = t.oFM32[2 * k + 1], h = t.hn32[k];
          const float l = f.w + m.w;
          const float F[3] = {f.x, f.y, f.z}, bl[3] = {l * h.x, l * h.y, l * h.z};
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) a[3 * p + q] -= F[p] * bl[q];
        }
        for (int q = 0; q < 9; ++q) v[q] += (double)a[q];
      } else {
        double kn[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const long long k = k0 + j * stride;
          kn[j] = k < t.P ? kn_fp64(t, k) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < R; ++j) {
          if (kn[j] == 0.0) continue;
          const long long k = k0 + j * stride;
          const double4_32a f = t.oFM[2 * k], m = t.oFM[2 * k + 1], h = t.hn[k];
          const double l = f.w + m.w;
          const double F[3] = {f.x, f.y, f.z}, n[3] = {h.x, h.y, h.z};
          for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) v[3 * p + q] += F[p] * (-l * n[q]);
        }
      }
    }
  }
  reduce_store<9>(v, partials);
}
}  // namespace

void launch_servo_partials(const Table &t, const Bodies &b, const DevStatus *ds, int mixed,
                           int law, double *partials, cudaStream_t st) {
  const dim3 g(kServoBlocks), bl(kServoThreads);
  if (mixed)
    law ? k_servo_partials<true, true><<<g, bl, 0, st>>>(t, b, ds, partials)
        : k_servo_partials<true, false><<<g, bl, 0, st>>>(t, b, ds, partials);
  else
    law ? k_servo_partials<false, true><<<g, bl, 0, st>>>(t, b, ds, partials)
        : k_servo_partials<false, false><<<g, bl, 0, st>>>(t, b, ds, partials);
}

void launch_p3d_partials(const Table &t, const DevStatus *ds, int mixed, double *partials,
                         cudaStream_t st) {
  if (mixed)
    k_p3d_partials<true><<<kServoBlocks, kServoThreads, 0, st>>>(t, ds, partials);
  else
    k_p3d_partials<false><<<kServoBlocks, kServoThreads, 0, st>>>(t, ds, partials);
}

}  // namespace dem
