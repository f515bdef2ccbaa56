// Fused contact kernel: one thread per row of the contact table runs, in one
// pass over the row, what the Yade InteractionLoop runs as three functors
// (section 1.1.2 "Engines", InteractionLoop):
//   Ig2_Sphere_Sphere_ScGeom  exact test |x2 + H c - x1| < r1 + r2, normal
//                             (eq. 2.7), penetration, contact point (eq. 2.8),
//                             shear-force transport into the new frame and the
//                             ratchet-free relative velocity (section 2.1.3 and
//                             the ScGeom class reference);
//   Ip2_FrictMat_FrictMat_FrictPhys  on a new contact: kn, ks from series
//                             springs k_i = E_i 2 r_i (resp. E_i nu_i 2 r_i),
//                             tan(phi) = min (section 2.1.2);
//   Law2_ScGeom_FrictPhys_CundallStrack  Fn = kn pen, shear increment, Coulomb
//                             cap |Fs| <= Fn tan(phi) (section 2.1.4).
// It writes the force on body 2 and the two torque arms; the per-body sum is a
// gather in the integrator (no atomics, fixed order).
//
// Readings of the text (shared with the oracle): the shear force is stored as
// acting on body 2 and incremented by -ks dt v12_perp; both rotation
// increments use the previous shear force; a new contact starts from Fs = 0,
// n_prev = n; the exact test is evaluated with round-to-nearest operations in
// the oracle's order so that both sides decide contact identically.
//
// Roofline: FP64 arithmetic on GB300 runs at 1/58 of the FP32 rate (measured),
// so this kernel is bound by the FP64 pipe (ncu: ~88% of its issue rate busy)
// rather than by its ~400 bytes of real-row traffic; square roots and divisions
// are taken from rsqrt to shorten the FP64 instruction stream.
#include "dem_internal.cuh"

namespace dem {

namespace {
constexpr int kT = 256;

__global__ void __launch_bounds__(kT) k_contact(Table t, Bodies b, const CellState *__restrict__ cs,
                                                const DevStatus *__restrict__ ds,
                                                const Mat *__restrict__ mats, int periodic) {
  if (ds->pending) return;
  const double dt = cs->dt;
  double H[9], W[9];
#pragma unroll
  for (int q = 0; q < 9; q += 4) {
    H[q] = periodic ? cs->H[q] : 0.0;
    W[q] = periodic ? cs->W[q] : 0.0;
  }
  const long long P = t.P;
  for (long long k = (long long)blockIdx.x * kT + threadIdx.x; k < P;
       k += (long long)gridDim.x * kT) {
    const int2 pr = t.pair[k];
    const double4_32a p1 = b.pos[pr.x];
    const double4_32a p2 = b.pos[pr.y];
    double c0 = 0, c1 = 0, c2 = 0;
    double h0 = 0, h1 = 0, h2 = 0;
    if (periodic) {
      int i0, i1, i2;
      unpack_shift(t.cpack[k], i0, i1, i2);
      c0 = i0; c1 = i1; c2 = i2;
      // the cell is diagonal (enforced at the C ABI): H c has one term per axis, the
      // same value the full product gives (the off-diagonal terms are exact zeros)
      h0 = __dmul_rn(H[0], c0);
      h1 = __dmul_rn(H[4], c1);
      h2 = __dmul_rn(H[8], c2);
    }
    // branch vector and the exact test (eq. 2.2, second pass; R1 of the oracle)
    const double dx = __dsub_rn(__dadd_rn(p2.x, h0), p1.x);
    const double dy = __dsub_rn(__dadd_rn(p2.y, h1), p1.y);
    const double dz = __dsub_rn(__dadd_rn(p2.z, h2), p1.z);
    const double l2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double R = __dadd_rn(p1.w, p2.w);
    double4_32a fs = t.hfs[k];
    if (!(l2 < __dmul_rn(R, R))) {
      if (fs.w != 0.0) {  // contact lost (u_N > 0): back to a potential interaction
        const double4_32a z = make_double4_32a(0, 0, 0, 0);
        t.hfs[k] = z; t.hn[k] = z; t.oF[k] = z; t.oM[k] = z;
      }
      continue;
    }
    double4_32a hn = t.hn[k];
    // 1/l from rsqrt (one FP64 pipe sequence instead of a square root and a division);
    // l = l2 / l within an ulp or two of the correctly rounded root
    const double il = rsqrt(l2);
    const double l = l2 * il;
    const double nx = dx * il, ny = dy * il, nz = dz * il;   // eq. 2.7
    const double pen = R - l;                                  // penetrationDepth
    const double r1 = p1.w, r2 = p2.w;
    double kn = fs.w, ks = hn.w, tanphi;
    if (kn == 0.0) {
      // Ip2_FrictMat_FrictMat_FrictPhys (new contact)
      const Mat m1 = mats[b.mat[pr.x]], m2 = mats[b.mat[pr.y]];
      const double k1 = m1.young * (2 * r1), k2 = m2.young * (2 * r2);
      kn = k1 * k2 / (k1 + k2);
      const double s1 = m1.young * m1.poisson * (2 * r1), s2 = m2.young * m2.poisson * (2 * r2);
      ks = s1 * s2 / (s1 + s2);
      tanphi = fmin(m1.tanphi, m2.tanphi);
      t.tanphi[k] = tanphi;
      fs = make_double4_32a(0, 0, 0, kn);
      hn = make_double4_32a(nx, ny, nz, ks);
    } else {
      tanphi = t.tanphi[k];
    }
    const double4_32a v1 = b.vel[pr.x], w1 = b.angvel[pr.x];
    double4_32a v2 = b.vel[pr.y];
    const double4_32a w2 = b.angvel[pr.y];
    if (periodic) {  // velocity of the image of body 2 (shift c moves with the cell)
      v2.x += W[0] * c0;
      v2.y += W[4] * c1;
      v2.z += W[8] * c2;
    }
    // 1. motion of the contact frame: -Fs x (n- x n) - Fs x (dt/2 n.(w1+w2) n)
    const double ax = hn.y * nz - hn.z * ny;
    const double ay = hn.z * nx - hn.x * nz;
    const double az = hn.x * ny - hn.y * nx;
    const double tw = 0.5 * dt * (nx * (w1.x + w2.x) + ny * (w1.y + w2.y) + nz * (w1.z + w2.z));
    const double bx = ax + tw * nx, by = ay + tw * ny, bz = az + tw * nz;
    double fx = fs.x - (fs.y * bz - fs.z * by);
    double fy = fs.y - (fs.z * bx - fs.x * bz);
    double fz = fs.z - (fs.x * by - fs.y * bx);
    // 2. mutual motion: ratchet-free v12 (ScGeom), its part perpendicular to n
    const double rx = r2 * w2.x + r1 * w1.x, ry = r2 * w2.y + r1 * w1.y, rz = r2 * w2.z + r1 * w1.z;
    const double f = R * il;
    const double ux = f * (v2.x - v1.x) - (ry * nz - rz * ny);
    const double uy = f * (v2.y - v1.y) - (rz * nx - rx * nz);
    const double uz = f * (v2.z - v1.z) - (rx * ny - ry * nx);
    const double vn = nx * ux + ny * uy + nz * uz;
    const double kd = ks * dt;
    fx -= kd * (ux - vn * nx);
    fy -= kd * (uy - vn * ny);
    fz -= kd * (uz - vn * nz);
    // Law2: normal force and Coulomb cap
    const double Fn = kn * pen;
    const double maxFs = Fn * tanphi;
    const double fs2 = fx * fx + fy * fy + fz * fz;
    if (fs2 > maxFs * maxFs) {
      const double sc = maxFs * rsqrt(fs2);
      fx *= sc; fy *= sc; fz *= sc;
    }
    const double Fx = Fn * nx + fx, Fy = Fn * ny + fy, Fz = Fn * nz + fz;
    // torques: T1 = (C - x1) x (-F) = d1 * M, T2 = (C - x2') x F = d2 * M, M = -(n x F)
    const double d1 = r1 - 0.5 * pen, d2 = r2 - 0.5 * pen;
    const double Mx = -(ny * Fz - nz * Fy), My = -(nz * Fx - nx * Fz), Mz = -(nx * Fy - ny * Fx);
    t.hfs[k] = make_double4_32a(fx, fy, fz, kn);
    t.hn[k] = make_double4_32a(nx, ny, nz, ks);
    t.oF[k] = make_double4_32a(Fx, Fy, Fz, d1);
    t.oM[k] = make_double4_32a(Mx, My, Mz, d2);
  }
}
}  // namespace

void launch_contact(const Table &t, const Bodies &b, const CellState *cs, const DevStatus *ds,
                    const Mat *mats, int periodic, int nsm, cudaStream_t st) {
  if (t.P <= 0) return;
  long long need = (t.P + kT - 1) / kT;
  long long cap = (long long)nsm * 8;
  unsigned grid = (unsigned)(need < cap ? need : cap);
  k_contact<<<grid, kT, 0, st>>>(t, b, cs, ds, mats, periodic);
}

}  // namespace dem
