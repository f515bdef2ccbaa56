// Mixed-precision variant of the fused contact kernel (same method as
// contact.cu: Ig2_Sphere_Sphere_ScGeom + Ip2_FrictMat_FrictMat_FrictPhys +
// Law2_ScGeom_FrictPhys_CundallStrack, sections 2.1.2-2.1.4).
//
// Precision split:
//   FP32  geometry and law: the branch vector is rebuilt each step from a
//         per-row FP32 reference branch vector (xref2 + Href c - xref1, formed in
//         FP64 at the collider run and rounded once) plus the FP32 offsets of
//         both bodies from their own FP64 positions at that run, plus the FP32
//         change of the cell shift (H - Href) c; the contact test and the
//         penetration from the squared gap (reference gap formed in FP64 at the
//         run, corrected by the FP32 offset terms); normal, penetration, relative
//         velocity, stiffnesses, normal force, output force and torque arms.
//   FP64  the shear-force history: the transport into the new contact frame
//         (-Fs x (n- x n) - Fs x (dt/2 n.(w1+w2) n)) and the shear increment are
//         formed in FP32 and accumulated into the FP64 spring, and the Coulomb cap
//         rescales the FP64 spring.
// Every length is an offset bounded by the cell size, so FP32 keeps about
// 1e-7 relative resolution of the branch length whatever the cell extent.
//
// Traffic per real row: 172 B read (row 28 + history 48 + two bodies 96),
// 80 B written; per non-real row 64 B read -- about 60% of the FP64 kernel's.
// GB300's FP64 pipe issues ~2 instructions per clock per SM and also carries
// every double<->float conversion, so at the HBM rate (~21 B per clock per SM) a
// real row affords ~25 FP64-pipe instructions: this kernel uses ~12 (three
// conversions in, three out, three accumulating adds, three for the output).
#include "dem_internal.cuh"

namespace dem {

namespace {
constexpr int kQ = 64;   // per-warp queue of real rows (< 32 left over + 32 new)

// Queued real row: its index, FP32 branch vector, squared length, radii, sub-scene,
// and the squared gap (r1 + r2)^2 - |d|^2 from the reference gap.
struct QRowF {
  float dx, dy, dz, l2, r1, r2;
  long long k;
  int q;
  float gap2;
};

// What a row needs of its (sub-)scene's cell state in FP32, plus the FP64 step.
struct RowCellF {
  double dt;
  float dH[3], W[3];   // diagonals (the full matrices are read when the cell is sheared)
  int periodic, law, sheared;
};
__device__ __forceinline__ RowCellF row_cell_f(const CellState &c) {
  RowCellF r;
  r.dt = c.dt;
  r.periodic = c.periodic;
  r.law = c.law;
  r.sheared = c.sheared;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.dH[i] = c.periodic ? c.dHf[4 * i] : 0.0f;
    r.W[i] = c.periodic ? c.Wf[4 * i] : 0.0f;
  }
  return r;
}

// One real row in mixed precision (Ip2 on creation, shear transport, Law2, outputs).
template <int kFeat>
__device__ __forceinline__ void real_row_mixed(const Table &t, const Bodies &b,
                                               const Mat *__restrict__ mats, const QRowF &e,
                                               const RowCellF &rc,
                                               const CellState *__restrict__ cq) {
  const double dt = rc.dt;
  const float *Wd = rc.W;
  const long long k = e.k;
  const int2 pr = t.pair[k];
  const float dx = e.dx, dy = e.dy, dz = e.dz, l2 = e.l2, r1 = e.r1, r2 = e.r2;
  const float R = r1 + r2;
  const float dtf = (float)dt;
  const float l = sqrtf(l2);
  const float il = 1.0f / l;
  const float nx = dx * il, ny = dy * il, nz = dz * il;
  // R - l = (R^2 - l^2) / (R + l): the penetration from the squared gap, which keeps
  // FP32's relative precision of the penetration itself (R - l in FP32 would lose it
  // to the rounding of l, a number of the size of R)
  const float pen = e.gap2 / (R + l);
  const float4 g = t.g32[k];
  float kn = g.w;
  double4_32a fsd = t.hfs[k];
  float4 hn = t.hn32[k];
  float ks;
  double tanphi;
  if (kn == 0.0f) {   // Ip2 on a new contact
    const Mat &m1 = mats[b.mat[pr.x]], &m2 = mats[b.mat[pr.y]];
    if ((kFeat & 1) && rc.law) {     // MindlinPhys constants kno, kso (formed once per contact in FP64)
      double kno, kso;
      mindlin_phys(m1, r1, m2, r2, kno, kso);
      kn = (float)kno;
      ks = (float)kso;
    } else {          // FrictPhys
      const float k1 = (float)m1.young * (2 * r1), k2 = (float)m2.young * (2 * r2);
      kn = k1 * k2 / (k1 + k2);
      const float s1 = (float)(m1.young * m1.poisson) * (2 * r1);
      const float s2 = (float)(m2.young * m2.poisson) * (2 * r2);
      ks = s1 * s2 / (s1 + s2);
    }
    tanphi = fmin(m1.tanphi, m2.tanphi);
    fsd = make_double4_32a(0, 0, 0, tanphi);
    hn = make_float4(nx, ny, nz, ks);
    t.g32[k] = make_float4(g.x, g.y, g.z, kn);
  } else {
    ks = hn.w;
    tanphi = fsd.w;
  }
  float cx = 0, cy = 0, cz = 0;
  if (rc.periodic) {
    int i0, i1, i2;
    unpack_shift(t.cpack[k], i0, i1, i2);
    cx = (float)i0; cy = (float)i1; cz = (float)i2;
  }
  const float4 va1 = b.vw32[2 * pr.x], vb1 = b.vw32[2 * pr.x + 1];
  const float4 va2 = b.vw32[2 * pr.y], vb2 = b.vw32[2 * pr.y + 1];
  const float w1x = va1.w, w1y = vb1.x, w1z = vb1.y;
  const float w2x = va2.w, w2y = vb2.x, w2z = vb2.y;
  float v2x = va2.x + Wd[0] * cx, v2y = va2.y + Wd[1] * cy, v2z = va2.z + Wd[2] * cz;
  if ((kFeat & 2) && rc.sheared) {   // W c with the full image velocity matrix
    const float *Wf = cq->Wf;
    v2x = va2.x + (Wf[0] * cx + Wf[1] * cy + Wf[2] * cz);
    v2y = va2.y + (Wf[3] * cx + Wf[4] * cy + Wf[5] * cz);
    v2z = va2.z + (Wf[6] * cx + Wf[7] * cy + Wf[8] * cz);
  }
  // 2 (first, in FP32). mutual motion: ratchet-free v12, its part perpendicular to n
  const float rx = r2 * w2x + r1 * w1x, ry = r2 * w2y + r1 * w1y, rz = r2 * w2z + r1 * w1z;
  const float f = R * il;
  const float ux = f * (v2x - va1.x) - (ry * nz - rz * ny);
  const float uy = f * (v2y - va1.y) - (rz * nx - rx * nz);
  const float uz = f * (v2z - va1.z) - (rx * ny - ry * nx);
  const float vn = nx * ux + ny * uy + nz * uz;
  const float sq = ((kFeat & 1) && rc.law) ? sqrtf(pen) : 1.0f;   // Hertz-Mindlin pen^1/2 factor
  const float kd = (ks * sq) * dtf;
  const float ix = kd * (ux - vn * nx), iy = kd * (uy - vn * ny), iz = kd * (uz - vn * nz);
  // 1. transport of the stored shear force into the new frame: the rotation vector
  //    b = n- x n + (dt/2 n.(w1+w2)) n and the change -Fs x b - ks dt v12_perp are
  //    formed in FP32 from an FP32 copy of the spring and accumulated into the FP64
  //    spring (as NewtonIntegrator accumulates FP32 increments into FP64 velocities):
  //    the stored force never drifts from repeated FP32 rounding
  const float tw = 0.5f * dtf * (nx * (w1x + w2x) + ny * (w1y + w2y) + nz * (w1z + w2z));
  const float bx = (hn.y * nz - hn.z * ny) + tw * nx;
  const float by = (hn.z * nx - hn.x * nz) + tw * ny;
  const float bz = (hn.x * ny - hn.y * nx) + tw * nz;
  const float sx0 = (float)fsd.x, sy0 = (float)fsd.y, sz0 = (float)fsd.z;
  double fx = fsd.x - (double)((sy0 * bz - sz0 * by) + ix);
  double fy = fsd.y - (double)((sz0 * bx - sx0 * bz) + iy);
  double fz = fsd.z - (double)((sx0 * by - sy0 * bx) + iz);
  // Law2: normal force, Coulomb test in FP32; the cap rescales the FP64 spring
  const float Fn = ((kFeat & 1) && rc.law) ? kn * pen * sq : kn * pen;
  const float maxFs = Fn * (float)tanphi;
  float sx = (float)fx, sy = (float)fy, sz = (float)fz;
  const float fs2 = sx * sx + sy * sy + sz * sz;
  if (fs2 > maxFs * maxFs) {
    const float sc = maxFs * rsqrtf(fs2);
    const double scd = (double)sc;
    fx *= scd; fy *= scd; fz *= scd;
    sx *= sc; sy *= sc; sz *= sc;
  }
  const float Fx = Fn * nx + sx, Fy = Fn * ny + sy, Fz = Fn * nz + sz;
  const float d1 = r1 - 0.5f * pen, d2 = r2 - 0.5f * pen;
  t.hfs[k] = make_double4_32a(fx, fy, fz, tanphi);
  t.hn32[k] = make_float4(nx, ny, nz, ks);
  t.oFM32[2 * k] = make_float4(Fx, Fy, Fz, d1);
  t.oFM32[2 * k + 1] = make_float4(-(ny * Fz - nz * Fy), -(nz * Fx - nx * Fz), -(nx * Fy - ny * Fx), d2);
}

// Same per-warp queue of real rows as the FP64 kernel: the FP32 geometry test on
// tiles of 32 consecutive rows, the law on 32 queued real rows at a time.
template <int kT, int kFeat, bool kDesc>
__global__ void __launch_bounds__(kT) k_contact_mixed(const StepDesc *__restrict__ d,
                                                      Table tp, Bodies bp,
                                                      const CellState *__restrict__ cs,
                                                      const DevStatus *__restrict__ ds,
                                                      const Mat *__restrict__ mats, int multi) {
  constexpr int kWarps = kT / 32;
  const Table &t = kDesc ? d->t : tp;
  const Bodies &b = kDesc ? d->b : bp;
  if (ds->pending) return;
  __shared__ QRowF q[kWarps][kQ];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  QRowF *wq = q[wi];
  const RowCellF rc0 = row_cell_f(cs[0]);
  const long long P = t.P;
  const long long stride = (long long)gridDim.x * kT;
  int cnt = 0;
  for (long long base = (long long)blockIdx.x * kT + wi * 32; base < P; base += stride) {
    const long long k = base + lane;
    bool real = false;
    float dx = 0, dy = 0, dz = 0, l2 = 0, r1 = 0, r2 = 0, gap2 = 0;
    int sq = 0;
    if (k < P) {
      const int2 pr = t.pair[k];
      const float4 g = t.g32[k];
      const float4 a = b.p32[pr.x];
      const float4 c = b.p32[pr.y];
      if (multi) sq = b.sid[pr.x];
      float cx = 0, cy = 0, cz = 0, dH0 = 0, dH1 = 0, dH2 = 0;
      float hx = 0, hy = 0, hz = 0;
      if (multi ? cs[sq].periodic : rc0.periodic) {
        int i0, i1, i2;
        unpack_shift(t.cpack[k], i0, i1, i2);
        cx = (float)i0; cy = (float)i1; cz = (float)i2;
        if ((kFeat & 2) && (multi ? cs[sq].sheared : rc0.sheared)) {   // (H - Href) c, full
          const float *D = cs[sq].dHf;
          hx = D[0] * cx + D[1] * cy + D[2] * cz;
          hy = D[3] * cx + D[4] * cy + D[5] * cz;
          hz = D[6] * cx + D[7] * cy + D[8] * cz;
        } else {
          dH0 = multi ? cs[sq].dHf[0] : rc0.dH[0];
          dH1 = multi ? cs[sq].dHf[4] : rc0.dH[1];
          dH2 = multi ? cs[sq].dHf[8] : rc0.dH[2];
          hx = dH0 * cx; hy = dH1 * cy; hz = dH2 * cz;
        }
      }
      // branch vector: reference branch at the collider run + the change e of both
      // offsets and of the cell shift since then; the contact test and the penetration
      // take the squared gap (r1 + r2)^2 - |g + e|^2 = s0 - 2 g.e - e.e, with s0 formed in
      // FP64 at the collider run: every FP32 term is then of the size of the gap or of
      // the motion since the run, not of the branch length
      const float ex = (c.x - a.x) + hx, ey = (c.y - a.y) + hy, ez = (c.z - a.z) + hz;
      dx = g.x + ex;
      dy = g.y + ey;
      dz = g.z + ez;
      l2 = dx * dx + dy * dy + dz * dz;
      r1 = a.w; r2 = c.w;
      gap2 = t.s0[k] - (2.0f * (g.x * ex + g.y * ey + g.z * ez) + (ex * ex + ey * ey + ez * ez));
      real = gap2 > 0.0f;
      if (!real && g.w != 0.0f) {   // contact lost: back to a potential interaction
        t.g32[k] = make_float4(g.x, g.y, g.z, 0.0f);
        t.hfs[k] = make_double4_32a(0, 0, 0, 0);
        const float4 z = make_float4(0, 0, 0, 0);
        t.hn32[k] = z; t.oFM32[2 * k] = z; t.oFM32[2 * k + 1] = z;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, real);
    if (real) {
      const int at = cnt + __popc(m & ((1u << lane) - 1u));
      wq[at] = QRowF{dx, dy, dz, l2, r1, r2, k, sq, gap2};
    }
    cnt += __popc(m);
    __syncwarp();
    if (cnt >= 32) {
      const QRowF e = wq[lane];
      real_row_mixed<kFeat>(t, b, mats, e, multi ? row_cell_f(cs[e.q]) : rc0, cs + e.q);
      __syncwarp();
      if (lane < cnt - 32) wq[lane] = wq[lane + 32];
      cnt -= 32;
      __syncwarp();
    }
  }
  if (lane < cnt) {
    const QRowF e = wq[lane];
    real_row_mixed<kFeat>(t, b, mats, e, multi ? row_cell_f(cs[e.q]) : rc0, cs + e.q);
  }
}
}  // namespace

void launch_contact_mixed(const StepDesc *d, const StepDesc &h, bool desc, long long rows,
                          const CellState *cs, const DevStatus *ds, const Mat *mats, int multi,
                          int feat, int nsm, int block, int per_sm, cudaStream_t st) {
  if (rows <= 0) return;
  long long need = (rows + block - 1) / block;
  long long cap = (long long)nsm * per_sm;   // persistent grid: per_sm blocks per SM
  unsigned grid = (unsigned)(need < cap ? need : cap);
#define DEM_C(B, F, D) k_contact_mixed<B, F, D><<<grid, B, 0, st>>>(d, h.t, h.b, cs, ds, mats, multi)
#define DEM_CB(F, D) if (block == 128) DEM_C(128, F, D); else DEM_C(256, F, D);
#define DEM_CF(D) switch (feat & 3) { case 0: DEM_CB(0, D) break; case 1: DEM_CB(1, D) break; \
                                      case 2: DEM_CB(2, D) break; default: DEM_CB(3, D) }
  if (desc) { DEM_CF(true) } else { DEM_CF(false) }
#undef DEM_CF
#undef DEM_CB
#undef DEM_C
}

}  // namespace dem
