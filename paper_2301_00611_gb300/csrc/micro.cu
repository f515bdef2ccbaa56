// Micromechanics of the contact network (utils reference of the Yade text):
//   fabricTensor              F = (1/n_c) sum n (x) n over the sphere-sphere contacts
//   normalShearStressTensors  the cell stress split into the part carried by normal
//                             forces, -(1/V) sum l N n (x) n, and by shear forces,
//                             -(1/V) sum l n (x) Fs (l = current centroid distance,
//                             N = normal force, compression negative)
//   bodyStressTensors         per sphere (1/V_b) sum x (x) f over its contacts, x the
//                             contact point relative to the centre, f the force on it
// Post-processing of the table the step leaves behind: block partial sums in a
// fixed tree (summed on the host in block order) and a per-body fixed-order gather,
// so every result is reproducible bit for bit.
#include "dem_internal.cuh"

namespace dem {

namespace {
constexpr int kT = 128;

template <int K>
__device__ inline void block_sum_store(double (&v)[K], double *partials) {
  __shared__ double sh[K][kT];
  for (int q = 0; q < K; ++q) sh[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int q = 0; q < K; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < K; ++q) partials[K * blockIdx.x + q] = sh[q][0];
}

// One real row: normal n, force on body 2 F, its shear part Fs, arms d1, d2.
struct RowOut {
  double n[3], F[3], Fs[3], d1, d2;
};

__device__ inline bool row_out(const Table &t, long long k, int mixed, RowOut &o) {
  if (mixed) {
    if (t.g32[k].w == 0.0f) return false;
    const float4 h = t.hn32[k], f = t.oFM32[2 * k], m = t.oFM32[2 * k + 1];
    const double4_32a s = t.hfs[k];
    o.n[0] = h.x; o.n[1] = h.y; o.n[2] = h.z;
    o.F[0] = f.x; o.F[1] = f.y; o.F[2] = f.z;
    o.Fs[0] = s.x; o.Fs[1] = s.y; o.Fs[2] = s.z;
    o.d1 = f.w; o.d2 = m.w;
  } else {
    const double4_32a s = t.hfs[k];
    if (s.w == 0.0) return false;
    const double4_32a h = t.hn[k], f = t.oFM[2 * k], m = t.oFM[2 * k + 1];
    o.n[0] = h.x; o.n[1] = h.y; o.n[2] = h.z;
    o.F[0] = f.x; o.F[1] = f.y; o.F[2] = f.z;
    o.Fs[0] = s.x; o.Fs[1] = s.y; o.Fs[2] = s.z;
    o.d1 = f.w; o.d2 = m.w;
  }
  return true;
}

// partials per block: count, fabric sum (9), sum l N n n (9), sum l n Fs (9)
constexpr int kMicro = 28;

__global__ void __launch_bounds__(kT) k_micro_rows(Table t, int mixed, double *partials) {
  double v[kMicro];
  for (int q = 0; q < kMicro; ++q) v[q] = 0;
  for (long long k = (long long)blockIdx.x * kT + threadIdx.x; k < t.P;
       k += (long long)gridDim.x * kT) {
    RowOut o;
    if (!row_out(t, k, mixed, o)) continue;
    const double l = o.d1 + o.d2;   // current centroid distance (d1 + d2 = l)
    const double N = (o.F[0] - o.Fs[0]) * o.n[0] + (o.F[1] - o.Fs[1]) * o.n[1] +
                     (o.F[2] - o.Fs[2]) * o.n[2];
    v[0] += 1.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        v[1 + 3 * i + j] += o.n[i] * o.n[j];
        v[10 + 3 * i + j] += l * N * o.n[i] * o.n[j];
        v[19 + 3 * i + j] += l * o.n[i] * o.Fs[j];
      }
  }
  block_sum_store<kMicro>(v, partials);
}

// Per body: sum of (contact point - centre) (x) (force on the body) over its rows in the
// fixed gather order, then its wall contacts; divided by the sphere volume.
__global__ void __launch_bounds__(kT) k_body_stress(Bodies b, Table t, long long N, long long cap,
                                                    int mixed, int walls, int multi,
                                                    const CellState *__restrict__ cs,
                                                    const Mat *__restrict__ mats, double *out) {
  const long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= N) return;
  const int s = (int)sl;
  double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  RowOut o;
  // in increasing partner id, as the force gather: the rows where the body is body 2,
  // then those where it is body 1
  for (int e = t.down_start[s]; e < t.down_start[s + 1]; ++e) {   // body 2: x = -d2 n, f = F
    if (!row_out(t, t.down[e], mixed, o)) continue;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) S[3 * i + j] -= o.d2 * o.n[i] * o.F[j];
  }
  for (int k = t.row_start[s]; k < t.row_start[s + 1]; ++k) {   // body 1: x = d1 n, f = -F
    if (!row_out(t, k, mixed, o)) continue;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) S[3 * i + j] -= o.d1 * o.n[i] * o.F[j];
  }
  const double r = b.pos[s].w;
  const uint8_t fl = b.flags[s];
  if (walls && (fl & 0x7e)) {
    // normal stiffness constant of the sphere-wall contact (FrictPhys: both springs
    // 2 r times the Young moduli; Hertz-Mindlin: kno with an infinite wall radius)
    const CellState &c = cs[multi ? b.sid[s] : 0];
    const Mat mw = mats[c.wall_mat], ms = mats[b.mat[s]];
    double kn, kso;
    if (c.law) {
      mindlin_phys(ms, r, mw, -1.0, kn, kso);
    } else {
      const double k1 = mw.young * (2 * r), k2 = ms.young * (2 * r);
      kn = k1 * k2 / (k1 + k2);
    }
    for (int wi = 0; wi < 6; ++wi) {   // n along axis wi/2, toward the sphere
      if (!(fl & (2 << wi))) continue;
      const double4_32a h = b.whist[wi * cap + s];
      const int ax = wi >> 1;
      const double sn = h.w >= 0 ? 1.0 : -1.0, Fn = fabs(h.w);
      double f[3] = {h.x, h.y, h.z};
      f[ax] += sn * Fn;
      const double xa = -sn * (r - 0.5 * wall_pen(Fn, kn, c.law));   // contact point - centre
      for (int j = 0; j < 3; ++j) S[3 * ax + j] += xa * f[j];
    }
  }
  const double V = (4.0 / 3.0) * 3.14159265358979323846 * r * r * r;
  for (int q = 0; q < 9; ++q) out[9 * sl + q] = S[q] / V;
}
}  // namespace

int micro_blocks(long long P) {
  long long b = (P + kT - 1) / kT;
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

void launch_micro_rows(const Table &t, int mixed, double *partials, cudaStream_t st) {
  k_micro_rows<<<micro_blocks(t.P), kT, 0, st>>>(t, mixed, partials);
}

void launch_body_stress(const Bodies &b, const Table &t, long long N, long long cap, int mixed,
                        int walls, int multi, const CellState *cs, const Mat *mats, double *out,
                        cudaStream_t st) {
  if (N > 0)
    k_body_stress<<<(unsigned)((N + kT - 1) / kT), kT, 0, st>>>(b, t, N, cap, mixed, walls, multi,
                                                                cs, mats, out);
}

}  // namespace dem
