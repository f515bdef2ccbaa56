// Per-body kernel of the step: force/torque gather over the body's contact
// rows in one fixed order (the ForceContainer sum made reproducible, cf. the
// summation-order example of section 2.1.7 "Result indeterminism"),
// sphere-wall contacts (Ig2_Wall_Sphere_ScGeom with the same law), gravity,
// Cundall non-viscous damping (eq. 2.9), leapfrog for position and spherical
// rotation (section 2.1.5), the orientation quaternion q+ = dq(w dt) q, the
// homoDeform = 2 velocity terms of a deforming periodic cell (Cell class
// reference), and the collider trigger (eq. 2.3-2.4) -- all fused in one pass
// over the body arrays.
//
// Also here: the one-thread cell/clock advance (F+ = (I + grad(v) dt) F,
// section 2.1.6), the force-only gather used by queries, and the statistics
// reductions (block partial sums in a fixed tree, summed on the host in
// block order, so every statistic is reproducible bit for bit).
#include "dem_internal.cuh"

namespace dem {

namespace {
constexpr int kT = 256;

// The step scaled by the damping factor of eq. 2.9, dt (1 - lam sgn(a b)), with
// dt_m = dt (1 - lam) and dt_p = dt (1 + lam): sgn(a b) is read from the sign bits and
// zero tests of a and b on the integer pipe (no FP64 product or compare).  It differs
// from sgn(fl(a b)) only if the product underflows to zero.
__device__ inline double damped_dt(double a, double b, double dt, double dt_m, double dt_p) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const bool zero = ((ia << 1) == 0) | ((ib << 1) == 0);
  return zero ? dt : ((ia ^ ib) < 0 ? dt_p : dt_m);
}
__device__ inline float damp_factor_f(float p, float lam) {
  return p > 0.0f ? 1.0f - lam : (p < 0.0f ? 1.0f + lam : 1.0f);
}
// finiteness by exponent bits (integer pipe)
__device__ inline bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}

// Fixed-order gather of a body's contact forces and torques, in increasing partner id:
// its rows as body 2 (force +F, torque d2 M; partners of smaller id) in down-list
// order, then its rows as body 1 (force -F, torque d1 M; partners of larger id) in row
// order.  The order depends on the ids only (not on the slots or the collider runs),
// so a body's sums are the same bits whatever the layout of the arrays.  Both lists
// run as one loop over their concatenation, so the trip count is the body's row count
// (which the degree ordering makes nearly uniform across a warp) rather than two loops
// whose lengths differ lane by lane; the sign is applied as a multiplication by -1 or
// +1, which is exact, so the sums are the same as two separate loops would give.  Two
// rows are loaded before either is added (more loads in flight, same order of the
// additions).
__device__ inline void gather_rows(const Table &t, int s, double F[3], double T[3]) {
  const int e0 = t.down_start[s], nd = t.down_start[s + 1] - e0;
  const int r0 = t.row_start[s] - nd, n = nd + (t.row_start[s + 1] - t.row_start[s]);
  int j = 0;
  for (; j + 1 < n; j += 2) {
    const bool a1 = j >= nd, b1 = j + 1 >= nd;   // body 1 of the row
    const int ka = a1 ? r0 + j : t.down[e0 + j];
    const int kb = b1 ? r0 + j + 1 : t.down[e0 + j + 1];
    const double4_32a fa = t.oFM[2 * ka], ma = t.oFM[2 * ka + 1], fb = t.oFM[2 * kb], mb = t.oFM[2 * kb + 1];
    const double sa = a1 ? -1.0 : 1.0, da = a1 ? fa.w : ma.w;
    const double sb = b1 ? -1.0 : 1.0, db = b1 ? fb.w : mb.w;
    F[0] += sa * fa.x; F[1] += sa * fa.y; F[2] += sa * fa.z;
    T[0] += da * ma.x; T[1] += da * ma.y; T[2] += da * ma.z;
    F[0] += sb * fb.x; F[1] += sb * fb.y; F[2] += sb * fb.z;
    T[0] += db * mb.x; T[1] += db * mb.y; T[2] += db * mb.z;
  }
  if (j < n) {
    const bool a1 = j >= nd;
    const int ka = a1 ? r0 + j : t.down[e0 + j];
    const double4_32a f = t.oFM[2 * ka], m = t.oFM[2 * ka + 1];
    const double sa = a1 ? -1.0 : 1.0, da = a1 ? f.w : m.w;
    F[0] += sa * f.x; F[1] += sa * f.y; F[2] += sa * f.z;
    T[0] += da * m.x; T[1] += da * m.y; T[2] += da * m.z;
  }
}

// Mixed precision: the same fixed-order gather over FP32 row outputs, summed in FP32
// (the contact forces are FP32 results; the sum feeds an FP64 velocity update).
__device__ inline void gather_rows_f32(const Table &t, int s, float F[3], float T[3]) {
  float f0 = 0, f1 = 0, f2 = 0, t0 = 0, t1 = 0, t2 = 0;
  const int e0 = t.down_start[s], nd = t.down_start[s + 1] - e0;
  const int r0 = t.row_start[s] - nd, n = nd + (t.row_start[s + 1] - t.row_start[s]);
  int j = 0;
  for (; j + 1 < n; j += 2) {
    const bool a1 = j >= nd, b1 = j + 1 >= nd;
    const int ka = a1 ? r0 + j : t.down[e0 + j];
    const int kb = b1 ? r0 + j + 1 : t.down[e0 + j + 1];
    const float4 fa = t.oFM32[2 * ka], ma = t.oFM32[2 * ka + 1], fb = t.oFM32[2 * kb], mb = t.oFM32[2 * kb + 1];
    const float sa = a1 ? -1.0f : 1.0f, da = a1 ? fa.w : ma.w;
    const float sb = b1 ? -1.0f : 1.0f, db = b1 ? fb.w : mb.w;
    f0 += sa * fa.x; f1 += sa * fa.y; f2 += sa * fa.z;
    t0 += da * ma.x; t1 += da * ma.y; t2 += da * ma.z;
    f0 += sb * fb.x; f1 += sb * fb.y; f2 += sb * fb.z;
    t0 += db * mb.x; t1 += db * mb.y; t2 += db * mb.z;
  }
  if (j < n) {
    const bool a1 = j >= nd;
    const int ka = a1 ? r0 + j : t.down[e0 + j];
    const float4 f = t.oFM32[2 * ka], m = t.oFM32[2 * ka + 1];
    const float sa = a1 ? -1.0f : 1.0f, da = a1 ? f.w : m.w;
    f0 += sa * f.x; f1 += sa * f.y; f2 += sa * f.z;
    t0 += da * m.x; t1 += da * m.y; t2 += da * m.z;
  }
  F[0] = f0; F[1] = f1; F[2] = f2;
  T[0] = t0; T[1] = t1; T[2] = t2;
}

// Physics of a sphere-wall contact: FrictPhys with equivalent wall radius = sphere
// radius, or (law 1) the Hertz-Mindlin constants with an infinite wall radius; wall
// material = the scene's wall material (material 0 by default).
__device__ inline void wall_phys(const Mat *mats, int wmat, int mat, double r, double &kn,
                                 double &ks, double &tanphi, int law = 0) {
  const Mat mw = mats[wmat], ms = mats[mat];
  tanphi = fmin(mw.tanphi, ms.tanphi);
  if (law) {
    mindlin_phys(ms, r, mw, -1.0, kn, ks);
    return;
  }
  const double k1 = mw.young * (2 * r), k2 = ms.young * (2 * r);
  kn = k1 * k2 / (k1 + k2);
  const double s1 = mw.young * mw.poisson * (2 * r), s2 = ms.young * ms.poisson * (2 * r);
  ks = s1 * s2 / (s1 + s2);
}

// Mixed precision integrator: FP32 force sum, walls, damping and orientation;
// FP64 only where the velocity and position accumulate (v += dv, x += dt v) and in
// the offset of the new position from its reference (rounded once to FP32 for the
// contact kernel).  Every quantity it needs in FP32 is read from the FP32 mirrors
// the previous step wrote, so the FP64 pipe (conversions included) carries ~27
// instructions per body.
// kFeat: bit 0 some sub-scene has walls, bit 1 some periodic cell is sheared (full 3x3
// products); each variant carries only the branches it needs.
template <int kB, int kFeat, bool kDesc>
__global__ void __launch_bounds__(kB) k_integrate_mixed(const StepDesc *__restrict__ d, StepDesc hp,
                                                        const CellState *__restrict__ cs,
                                                        DevStatus *ds, const Mat *__restrict__ mats) {
  if (ds->pending) return;
  const Bodies &b = kDesc ? d->b : hp.b;
  const Table &t = kDesc ? d->t : hp.t;
  const SceneConst &sc = kDesc ? d->sc : hp.sc;
  const long long cap = kDesc ? d->cap : hp.cap;
  const long long sl = (long long)blockIdx.x * kB + threadIdx.x;
  if (sl >= sc.N) return;
  const int s = sc.ordered ? t.ord[sl] : (int)sl;
  const CellState &c = cs[sc.multi ? b.sid[s] : 0];
  const double dt = c.dt;
  const float dtf = (float)dt;
  float F[3], T[3];
  gather_rows_f32(t, s, F, T);   // fixed order, FP32 sums
  const float4 va = b.vw32[2 * s], vb = b.vw32[2 * s + 1];   // v-, w- in FP32
  const float4 off = b.p32[s];                                // x - xref, r
  const float4 xr = b.xref32[s];
  const float4 mp = b.mprop32[s];                             // m, I, 1/m, 1/I
  uint8_t flags = b.flags[s];
  const float vv[3] = {va.x, va.y, va.z}, ww[3] = {va.w, vb.x, vb.y};
  const float xf[3] = {xr.x + off.x, xr.y + off.y, xr.z + off.z};
  const float r = off.w;

  if ((kFeat & 1) && c.wall_mask) {   // sphere-wall contacts: the FP64 kernel's law, in FP32
    const float dtl = (float)c.dt_law;   // the contact law's step (see CellState::dt_law)
    const double4_32a pd = b.pos[s];
    const double xd[3] = {pd.x, pd.y, pd.z};
    for (int wi = 0; wi < 6; ++wi) {
      if (!(c.wall_mask & (1 << wi))) continue;
      const int ax = wi >> 1;
      const double distd = xd[ax] - ((wi & 1) ? c.box_hi[ax] : c.box_lo[ax]);
      const float dist = (float)distd;
      const bool was = flags & (2 << wi);
      if (!(fabsf(dist) < r)) {
        if (was) {
          b.whist[wi * cap + s] = make_double4_32a(0, 0, 0, 0);
          flags &= ~(2 << wi);
        }
        continue;
      }
      const float sn = dist >= 0 ? 1.0f : -1.0f;
      float n[3] = {0, 0, 0};
      n[ax] = sn;
      // the penetration in FP64 and rounded once: r - |dist| in FP32 would keep the
      // precision of r, not of the (much smaller) penetration
      const float pen = (float)(pd.w - fabs(distd));   // FP64 radius and distance
      double knd, ksd, tpd;
      wall_phys(mats, c.wall_mat, b.mat[s], (double)r, knd, ksd, tpd, c.law);
      const float sqp = c.law ? sqrtf(pen) : 1.0f;   // Hertz-Mindlin: pen^1/2 factors
      const float kn = (float)knd * sqp, ks = (float)ksd * sqp, tanphi = (float)tpd;
      float fs[3] = {0, 0, 0};
      if (was) {
        const double4_32a h = b.whist[wi * cap + s];
        fs[0] = (float)h.x; fs[1] = (float)h.y; fs[2] = (float)h.z;
      }
      const float tw = 0.5f * dtl * (sn * ww[ax]);
      const float tn[3] = {tw * n[0], tw * n[1], tw * n[2]};
      const float c0 = fs[1] * tn[2] - fs[2] * tn[1];
      const float c1 = fs[2] * tn[0] - fs[0] * tn[2];
      const float c2 = fs[0] * tn[1] - fs[1] * tn[0];
      fs[0] -= c0; fs[1] -= c1; fs[2] -= c2;
      const float rr[3] = {r * ww[0], r * ww[1], r * ww[2]};
      const float cr[3] = {rr[1] * n[2] - rr[2] * n[1], rr[2] * n[0] - rr[0] * n[2],
                           rr[0] * n[1] - rr[1] * n[0]};
      const float fac = (r + r) / (2 * r - pen);
      float u[3];
      for (int q = 0; q < 3; ++q) u[q] = fac * vv[q] - cr[q];
      const float vn = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
      for (int q = 0; q < 3; ++q) fs[q] -= ks * (dtl * (u[q] - vn * n[q]));
      const float Fn = kn * pen;
      const float maxFs = Fn * tanphi;
      const float fs2 = fs[0] * fs[0] + fs[1] * fs[1] + fs[2] * fs[2];
      if (fs2 > maxFs * maxFs) {
        const float scl = maxFs * rsqrtf(fs2);
        fs[0] *= scl; fs[1] *= scl; fs[2] *= scl;
      }
      const float F2[3] = {Fn * n[0] + fs[0], Fn * n[1] + fs[1], Fn * n[2] + fs[2]};
      const float arm = -(r - 0.5f * pen);
      const float a[3] = {arm * n[0], arm * n[1], arm * n[2]};
      F[0] += F2[0]; F[1] += F2[1]; F[2] += F2[2];
      T[0] += a[1] * F2[2] - a[2] * F2[1];
      T[1] += a[2] * F2[0] - a[0] * F2[2];
      T[2] += a[0] * F2[1] - a[1] * F2[0];
      b.whist[wi * cap + s] = make_double4_32a(fs[0], fs[1], fs[2], sn * Fn);
      flags |= (2 << wi);
    }
  }

  float dv[3] = {0, 0, 0}, dw[3] = {0, 0, 0};
  const bool fixed = flags & 1;
  if (!fixed) {
    const float lam = (float)c.damping;
    float vref[3] = {vv[0], vv[1], vv[2]};
    if (c.periodic) {
      if ((kFeat & 2) && c.sheared) {
        for (int q = 0; q < 3; ++q)
          vref[q] -= (float)c.Lprev[3 * q] * xf[0] + (float)c.Lprev[3 * q + 1] * xf[1] +
                     (float)c.Lprev[3 * q + 2] * xf[2];
      } else {
        for (int q = 0; q < 3; ++q) vref[q] -= (float)c.Lprev[4 * q] * xf[q];
      }
    }
    float im = mp.z, iI = mp.w;   // inverse inertial mass and moment
    if (c.dscale) {   // density scaling: inertia times f (the weight keeps the true mass)
      const float rf = (float)b.rdsc[s];
      im *= rf;
      iI *= rf;
    }
    for (int q = 0; q < 3; ++q) {
      const float Ft = F[q] + mp.x * (float)c.gravity[q];
      const float acc = Ft * im;
      const float Fd = Ft * damp_factor_f(Ft * (vref[q] + 0.5f * dtf * acc), lam);
      dv[q] = dtf * Fd * im;
      const float aacc = T[q] * iI;
      const float Td = T[q] * damp_factor_f(T[q] * (ww[q] + 0.5f * dtf * aacc), lam);
      dw[q] = dtf * Td * iI;
    }
    if (c.periodic) {   // homoDeform = 2
      if ((kFeat & 2) && c.sheared) {
        for (int q = 0; q < 3; ++q) {
          float a = 0, bq = 0;
          for (int j = 0; j < 3; ++j) {
            a += (float)c.dL[3 * q + j] * xf[j];
            bq += (float)c.L[3 * q + j] * vv[j];
          }
          dv[q] += a + dtf * bq;
        }
      } else {
        for (int q = 0; q < 3; ++q)
          dv[q] += (float)c.dL[4 * q] * xf[q] + dtf * ((float)c.L[4 * q] * vv[q]);
      }
    }
  }
  // FP64 accumulation of velocity, spin and position
  const double4_32a v = b.vel[s], w = b.angvel[s], p = b.pos[s];
  const double vn_[3] = {v.x + (double)dv[0], v.y + (double)dv[1], v.z + (double)dv[2]};
  const double wn_[3] = {w.x + (double)dw[0], w.y + (double)dw[1], w.z + (double)dw[2]};
  const double xn[3] = {p.x + dt * vn_[0], p.y + dt * vn_[1], p.z + dt * vn_[2]};
  b.pos[s] = make_double4_32a(xn[0], xn[1], xn[2], p.w);
  b.vel[s] = make_double4_32a(vn_[0], vn_[1], vn_[2], 0.0);
  b.angvel[s] = make_double4_32a(wn_[0], wn_[1], wn_[2], 0.0);
  if (flags != b.flags[s]) b.flags[s] = flags;
  const float vnf[3] = {(float)vn_[0], (float)vn_[1], (float)vn_[2]};
  const float wnf[3] = {(float)wn_[0], (float)wn_[1], (float)wn_[2]};
  b.vw32[2 * s] = make_float4(vnf[0], vnf[1], vnf[2], wnf[0]);
  b.vw32[2 * s + 1] = make_float4(wnf[1], wnf[2], 0.0f, 0.0f);
  const double4_32a xrd = b.xref[s];
  const float ox = (float)(xn[0] - xrd.x), oy = (float)(xn[1] - xrd.y), oz = (float)(xn[2] - xrd.z);
  b.p32[s] = make_float4(ox, oy, oz, r);

  // orientation in FP32: q+ = dq(w+ dt) q, series of cos x and sin x / x for x < 1e-2
  const float w2 = wnf[0] * wnf[0] + wnf[1] * wnf[1] + wnf[2] * wnf[2];
  if (w2 > 0.0f) {
    const float4 q0 = b.ori32[s];
    const float x2 = 0.25f * (dtf * dtf) * w2;
    float ch, sx;
    if (x2 < 1e-4f) {
      ch = 1.0f - 0.5f * x2 * (1.0f - x2 * (1.0f / 12.0f));
      sx = 1.0f - x2 * (1.0f / 6.0f) * (1.0f - x2 * (1.0f / 20.0f));
    } else {
      const float x = sqrtf(x2);
      float sh;
      sincosf(x, &sh, &ch);
      sx = sh / x;
    }
    const float hs = 0.5f * dtf * sx;
    const float dq0 = ch, dq1 = hs * wnf[0], dq2 = hs * wnf[1], dq3 = hs * wnf[2];
    b.ori32[s] = make_float4(dq0 * q0.x - dq1 * q0.y - dq2 * q0.z - dq3 * q0.w,
                             dq0 * q0.y + dq1 * q0.x + dq2 * q0.w - dq3 * q0.z,
                             dq0 * q0.z - dq1 * q0.w + dq2 * q0.x + dq3 * q0.y,
                             dq0 * q0.w + dq1 * q0.z - dq2 * q0.y + dq3 * q0.x);
  }
  // collider trigger on the FP32 offset (slightly early to cover its rounding)
  float ux = ox - c.Ef[0] * xr.x, uy = oy - c.Ef[4] * xr.y, uz = oz - c.Ef[8] * xr.z;
  if ((kFeat & 2) && c.sheared) {   // E xref with the full affine strain
    const float *Ef = c.Ef;
    ux = ox - (Ef[0] * xr.x + Ef[1] * xr.y + Ef[2] * xr.z);
    uy = oy - (Ef[3] * xr.x + Ef[4] * xr.y + Ef[5] * xr.z);
    uz = oz - (Ef[6] * xr.x + Ef[7] * xr.y + Ef[8] * xr.z);
  }
  if (!(ux * ux + uy * uy + uz * uz <= (float)(0.998 * c.thr2))) {
    if (!ds->request) ds->request = 1;
  }
  if (!(isfinite(ox + oy + oz) && isfinite(vnf[0] + vnf[1] + vnf[2]) &&
        isfinite(wnf[0] + wnf[1] + wnf[2])))
    atomicOr(&ds->error, kErrNonFinite);
}

template <int kB, int kFeat, bool kDesc>
__global__ void __launch_bounds__(kB) k_integrate(const StepDesc *__restrict__ d, StepDesc hp,
                                                  const CellState *__restrict__ cs,
                                                  DevStatus *ds, const Mat *__restrict__ mats) {
  if (ds->pending) return;
  const Bodies &b = kDesc ? d->b : hp.b;
  const Table &t = kDesc ? d->t : hp.t;
  const SceneConst &sc = kDesc ? d->sc : hp.sc;
  const long long cap = kDesc ? d->cap : hp.cap;
  const long long sl = (long long)blockIdx.x * kB + threadIdx.x;
  if (sl >= sc.N) return;
  const int s = sc.ordered ? t.ord[sl] : (int)sl;
  const CellState &c = cs[sc.multi ? b.sid[s] : 0];
  const double dt = c.dt;
  double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
  gather_rows(t, s, F, T);

  const double4_32a p = b.pos[s];
  const double4_32a v = b.vel[s];
  const double4_32a w = b.angvel[s];
  const double4_32a mp = b.mprop[s];   // m, I, 1/m, 1/I
  uint8_t flags = b.flags[s];
  const double x[3] = {p.x, p.y, p.z}, vv[3] = {v.x, v.y, v.z}, ww[3] = {w.x, w.y, w.z};
  const double r = p.w;

  if ((kFeat & 1) && c.wall_mask) {
    for (int wi = 0; wi < 6; ++wi) {
      if (!(c.wall_mask & (1 << wi))) continue;
      const int ax = wi >> 1;
      const double wc = (wi & 1) ? c.box_hi[ax] : c.box_lo[ax];
      const double dist = x[ax] - wc;
      const bool was = flags & (2 << wi);
      if (!(fabs(dist) < r)) {
        if (was) {
          b.whist[wi * cap + s] = make_double4_32a(0, 0, 0, 0);
          flags &= ~(2 << wi);
        }
        continue;
      }
      const double sn = dist >= 0 ? 1.0 : -1.0;
      double n[3] = {0, 0, 0};
      n[ax] = sn;
      const double pen = r - fabs(dist);
      double kn, ks, tanphi;
      wall_phys(mats, c.wall_mat, b.mat[s], r, kn, ks, tanphi, c.law);
      if (c.law) {   // Hertz-Mindlin: Fn = kno pen^3/2, ks = kso pen^1/2
        const double sq = sqrt(pen);
        kn *= sq;
        ks *= sq;
      }
      double fs[3] = {0, 0, 0};
      if (was) {
        const double4_32a h = b.whist[wi * cap + s];
        fs[0] = h.x; fs[1] = h.y; fs[2] = h.z;
      }
      // frame motion: n- x n = 0 (the normal is fixed); twist dt/2 n.(0 + w), with the
      // contact law's step (see CellState::dt_law)
      const double tw = 0.5 * c.dt_law * (sn * ww[ax]);
      const double tn[3] = {tw * n[0], tw * n[1], tw * n[2]};
      const double c0 = fs[1] * tn[2] - fs[2] * tn[1];
      const double c1 = fs[2] * tn[0] - fs[0] * tn[2];
      const double c2 = fs[0] * tn[1] - fs[1] * tn[0];
      fs[0] -= c0; fs[1] -= c1; fs[2] -= c2;
      // ratchet-free relative velocity with refR1 = refR2 = r, l = 2r - pen, wall at rest
      const double rr[3] = {r * ww[0], r * ww[1], r * ww[2]};
      const double cr[3] = {rr[1] * n[2] - rr[2] * n[1], rr[2] * n[0] - rr[0] * n[2],
                            rr[0] * n[1] - rr[1] * n[0]};
      const double fac = (r + r) / (2 * r - pen);
      double u[3];
      for (int q = 0; q < 3; ++q) u[q] = fac * vv[q] - cr[q];
      const double vn = n[0] * u[0] + n[1] * u[1] + n[2] * u[2];
      for (int q = 0; q < 3; ++q) fs[q] -= ks * (c.dt_law * (u[q] - vn * n[q]));
      const double Fn = kn * pen;
      const double maxFs = Fn * tanphi;
      const double fs2 = fs[0] * fs[0] + fs[1] * fs[1] + fs[2] * fs[2];
      if (fs2 > maxFs * maxFs) {
        const double scl = maxFs / sqrt(fs2);
        fs[0] *= scl; fs[1] *= scl; fs[2] *= scl;
      }
      const double F2[3] = {Fn * n[0] + fs[0], Fn * n[1] + fs[1], Fn * n[2] + fs[2]};
      const double arm = -(r - 0.5 * pen);   // C - x = arm * n
      const double a[3] = {arm * n[0], arm * n[1], arm * n[2]};
      F[0] += F2[0]; F[1] += F2[1]; F[2] += F2[2];
      T[0] += a[1] * F2[2] - a[2] * F2[1];
      T[1] += a[2] * F2[0] - a[0] * F2[2];
      T[2] += a[0] * F2[1] - a[1] * F2[0];
      b.whist[wi * cap + s] = make_double4_32a(fs[0], fs[1], fs[2], sn * Fn);
      flags |= (2 << wi);
    }
  }

  double vn_[3], wn_[3];
  const bool fixed = flags & 1;
  if (!fixed) {
    const double lam = c.damping;
    double vref[3] = {vv[0], vv[1], vv[2]};
    if (c.periodic) {   // fluctuation velocity for eq. 2.9 in a deforming cell
      const double *Lp = c.Lprev;
      if ((kFeat & 2) && c.sheared) {   // Lprev x, rows summed as the oracle writes them
        for (int q = 0; q < 3; ++q)
          vref[q] -= Lp[3 * q] * x[0] + Lp[3 * q + 1] * x[1] + Lp[3 * q + 2] * x[2];
      } else {   // diagonal matrices: only their diagonals enter
        for (int q = 0; q < 3; ++q) vref[q] -= Lp[4 * q] * x[q];
      }
    }
    // eq. 2.9 with the damping factor folded into the step: v+ = v- + dt (1 -+ lam) a,
    // a = F / m, the sign decided on F (v- + dt/2 a) (products and sums of the same
    // terms as the oracle's dt F (1 -+ lam) / m, in another rounding order)
    const double hdt = 0.5 * dt, dt_m = dt * (1.0 - lam), dt_p = dt * (1.0 + lam);
    double im = mp.z, iI = mp.w;   // inverse inertial mass and moment
    if (c.dscale) {   // density scaling: inertia times f (the weight keeps the true mass)
      const double rf = b.rdsc[s];
      im *= rf;
      iI *= rf;
    }
    for (int q = 0; q < 3; ++q) {
      const double Ft = F[q] + mp.x * c.gravity[q];
      const double a = Ft * im;
      vn_[q] = vv[q] + damped_dt(Ft, vref[q] + hdt * a, dt, dt_m, dt_p) * a;
      const double al = T[q] * iI;
      wn_[q] = ww[q] + damped_dt(T[q], ww[q] + hdt * al, dt, dt_m, dt_p) * al;
    }
    if (c.periodic) {   // homoDeform = 2
      const double *dL = c.dL, *L = c.L;
      if ((kFeat & 2) && c.sheared) {
        for (int q = 0; q < 3; ++q)
          vn_[q] += (dL[3 * q] * x[0] + dL[3 * q + 1] * x[1] + dL[3 * q + 2] * x[2]) +
                    dt * (L[3 * q] * vv[0] + L[3 * q + 1] * vv[1] + L[3 * q + 2] * vv[2]);
      } else {
        if (c.dl_zero) {   // gradient unchanged since the last step: only dt L v-
          for (int q = 0; q < 3; ++q) vn_[q] += c.dtL[q] * vv[q];
        } else {
          for (int q = 0; q < 3; ++q) vn_[q] += dL[4 * q] * x[q] + dt * (L[4 * q] * vv[q]);
        }
      }
    }
  } else {
    for (int q = 0; q < 3; ++q) { vn_[q] = vv[q]; wn_[q] = ww[q]; }
  }
  const double xn[3] = {x[0] + dt * vn_[0], x[1] + dt * vn_[1], x[2] + dt * vn_[2]};
  b.pos[s] = make_double4_32a(xn[0], xn[1], xn[2], r);
  b.vel[s] = make_double4_32a(vn_[0], vn_[1], vn_[2], 0.0);
  b.angvel[s] = make_double4_32a(wn_[0], wn_[1], wn_[2], 0.0);
  if (flags != b.flags[s]) b.flags[s] = flags;

  // orientation: q+ = dq(w+ dt) q, dq = (cos x, (sin x / x) * w dt / 2), x = |w| dt / 2.
  // For x < 1e-2 the Maclaurin series of cos x and sin x / x truncated after the x^4
  // term (first omitted terms x^6/720 and x^6/5040, below 1.4e-15) needs no square
  // root, division or sincos; larger angles use sincos.
  const double w2 = wn_[0] * wn_[0] + wn_[1] * wn_[1] + wn_[2] * wn_[2];
  if (!is_zero_bits(w2)) {   // w2 > 0 (a sum of squares)
    const double4_32a q0 = b.ori[s];
    const double x2 = 0.25 * (dt * dt) * w2;
    double ch, sx;   // cos x, sin x / x
    if (lt_nonneg(x2, 1e-4)) {
      ch = 1.0 - 0.5 * x2 * (1.0 - x2 * (1.0 / 12.0));
      sx = 1.0 - x2 * (1.0 / 6.0) * (1.0 - x2 * (1.0 / 20.0));
    } else {
      const double x = sqrt(x2);
      double sh;
      sincos(x, &sh, &ch);
      sx = sh / x;
    }
    const double hs = 0.5 * dt * sx;
    const double dw = ch, dx = hs * wn_[0], dy = hs * wn_[1], dz = hs * wn_[2];
    b.ori[s] = make_double4_32a(dw * q0.x - dx * q0.y - dy * q0.z - dz * q0.w,
                                dw * q0.y + dx * q0.x + dy * q0.w - dz * q0.z,
                                dw * q0.z - dx * q0.w + dy * q0.x + dz * q0.y,
                                dw * q0.w + dx * q0.z - dy * q0.y + dz * q0.x);
  }

  // collider trigger: displacement since the last run, minus the affine part
  const double4_32a xr = b.xref[s];
  const double *E = c.E;   // diagonal cell: x+ - (1 + E) xref, one fused step per axis
  double ux = xn[0] - c.Ep1[0] * xr.x;
  double uy = xn[1] - c.Ep1[1] * xr.y;
  double uz = xn[2] - c.Ep1[2] * xr.z;
  if ((kFeat & 2) && c.sheared) {   // E xref with the full affine strain
    ux = (xn[0] - xr.x) - (E[0] * xr.x + E[1] * xr.y + E[2] * xr.z);
    uy = (xn[1] - xr.y) - (E[3] * xr.x + E[4] * xr.y + E[5] * xr.z);
    uz = (xn[2] - xr.z) - (E[6] * xr.x + E[7] * xr.y + E[8] * xr.z);
  }
  if (lt_nonneg(c.thr2, ux * ux + uy * uy + uz * uz)) {   // displacement^2 > bound^2
    if (!ds->request) ds->request = 1;
  }
  bool ok = true;
  for (int q = 0; q < 3; ++q) ok &= finite_bits(xn[q]) & finite_bits(vn_[q]) & finite_bits(wn_[q]);
  if (!ok) atomicOr(&ds->error, kErrNonFinite);
}

// Row-major 3x3 helpers evaluated with round-to-nearest operations in a fixed
// order (the same order the oracle writes them), so the cell history is
// reproducible on every platform.
__device__ inline void m_mul_rn(const double *A, const double *B, double *O) {
  double Tm[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      Tm[3 * r + c] = __dadd_rn(__dadd_rn(__dmul_rn(A[3 * r], B[c]), __dmul_rn(A[3 * r + 1], B[3 + c])),
                                __dmul_rn(A[3 * r + 2], B[6 + c]));
  for (int q = 0; q < 9; ++q) O[q] = Tm[q];
}

// The next cell H+ = (I + L dt) H, the affine strain since the collider run and
// the displacement bound that follow from it (periodic cells).
// H+ = (I + L dt) H, the affine strain E = (H+ - Href) Href^-1 since the collider run
// and the displacement bound that follow from it, computed on local copies (one
// thread: keeping the matrices in registers avoids a chain of dependent global loads)
__device__ void derive_next_local(CellState *__restrict__ cs, const double (&H)[9],
                                  const double (&L)[9], double dt) {
  double A[9], Hn[9], D[9], Hri[9], E[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    A[q] = __dadd_rn((q % 4 == 0) ? 1.0 : 0.0, __dmul_rn(L[q], dt));
    Hri[q] = cs->Hrefinv[q];
  }
  m_mul_rn(A, H, Hn);
#pragma unroll
  for (int q = 0; q < 9; ++q) D[q] = Hn[q] - cs->Href[q];
  m_mul_rn(D, Hri, E);
  double e2 = 0;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    e2 += E[q] * E[q];
    cs->Hnext[q] = Hn[q];
    cs->E[q] = E[q];
  }
  const double eff = cs->verlet - sqrt(e2) * (cs->rmax + cs->verlet);
  cs->thr2 = eff > 0 ? eff * eff : -1.0;
#pragma unroll
  for (int q = 0; q < 9; ++q) cs->Ef[q] = (float)E[q];
  for (int k = 0; k < 3; ++k) {
    cs->Ep1[k] = 1.0 + E[4 * k];
    cs->dtL[k] = dt * L[4 * k];
  }
}

// Whether a double is nonzero (either sign), tested on its bits by the integer pipe.
__device__ inline bool nonzero_bits(double x) { return (__double_as_longlong(x) << 1) != 0; }
__device__ inline bool offdiag_nonzero(const double *M) {
  return nonzero_bits(M[1]) | nonzero_bits(M[2]) | nonzero_bits(M[3]) | nonzero_bits(M[5]) |
         nonzero_bits(M[6]) | nonzero_bits(M[7]);
}

// derive_next_local for a cell whose matrices are all diagonal: the same values (every
// off-diagonal term of the products is an exact zero, which leaves the diagonal sums
// unchanged, and the off-diagonal entries in memory stay zero) with a fifth of the FP64
// instructions.  One thread runs this, and each FP64 warp instruction occupies the
// SM's FP64 pipe as long as a full warp's would.
__device__ void derive_next_diag(CellState *__restrict__ cs, const double (&H)[9],
                                 const double (&L)[9], double dt) {
  double E[3], e2 = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int q = 4 * k;
    const double Hn = __dmul_rn(__dadd_rn(1.0, __dmul_rn(L[q], dt)), H[q]);
    E[k] = __dmul_rn(Hn - cs->Href[q], cs->Hrefinv[q]);
    cs->Hnext[q] = Hn;
    cs->E[q] = E[k];
  }
  for (int k = 0; k < 3; ++k) e2 += E[k] * E[k];
  const double eff = cs->verlet - sqrt(e2) * (cs->rmax + cs->verlet);
  cs->thr2 = eff > 0 ? eff * eff : -1.0;
  for (int k = 0; k < 3; ++k) {
    cs->Ef[4 * k] = (float)E[k];
    cs->Ep1[k] = 1.0 + E[k];
    cs->dtL[k] = dt * L[4 * k];
  }
}

__device__ void derive_next(CellState *__restrict__ cs) {
  double H[9], L[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) { H[q] = cs->H[q]; L[q] = cs->L[q]; }
  derive_next_local(cs, H, L, cs->dt);
}

// ---- Peri3dController (class reference): one thread, FP64, after the cell update
__device__ inline bool m_inv_dev(const double *M, double *O) {
  const double d = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                   M[2] * (M[3] * M[7] - M[4] * M[6]);
  if (d == 0.0 || !isfinite(d)) return false;
  double T[9];
  T[0] = (M[4] * M[8] - M[5] * M[7]) / d; T[1] = (M[2] * M[7] - M[1] * M[8]) / d;
  T[2] = (M[1] * M[5] - M[2] * M[4]) / d; T[3] = (M[5] * M[6] - M[3] * M[8]) / d;
  T[4] = (M[0] * M[8] - M[2] * M[6]) / d; T[5] = (M[2] * M[3] - M[0] * M[5]) / d;
  T[6] = (M[3] * M[7] - M[4] * M[6]) / d; T[7] = (M[1] * M[6] - M[0] * M[7]) / d;
  T[8] = (M[0] * M[4] - M[1] * M[3]) / d;
  for (int q = 0; q < 9; ++q) O[q] = T[q];
  return true;
}

__device__ inline void m_tr(const double *A, double *O) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) O[3 * r + c] = A[3 * c + r];
}

// value of component i on its time function at progress p: piecewise linear from
// (0, 0) through the couples scaled by the last one, the goal beyond it
__device__ double p3d_value(const P3d &P, int i, double p) {
  const int n = P.npath[i];
  const double tl = P.path[i][n - 1][0], vl = P.path[i][n - 1][1];
  double t0 = 0, v0 = 0;
  for (int j = 0; j < n; ++j) {
    const double t1 = P.path[i][j][0] / tl, v1 = P.path[i][j][1] / vl;
    if (p <= t1) {
      const double a = t1 > t0 ? (p - t0) / (t1 - t0) : 1.0;
      return P.goal[i] * (v0 + a * (v1 - v0));
    }
    t0 = t1;
    v0 = v1;
  }
  return P.goal[i];
}

// Controller update at the end of a step: stress of the step's contacts (cell Hp),
// strain of the transformation T = H H0^-1 T0 = U P (polar decomposition) in global
// axes, the next rates and the velocity gradient (T+ T^-1 - I) / dt with
// T+ = U (P + U^T dt E(rate) U).  Returns false when the controller did not update.
__device__ bool p3d_update(P3d &P, const double *part, const double (&Hp)[9],
                           const double (&H)[9], double dt, double (&L)[9]) {
  const int VO[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {2, 0}, {0, 1}};
  double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < kServoBlocks; ++b)
    for (int q = 0; q < 9; ++q) S[q] += part[9 * b + q];
  const double V = fabs(Hp[0] * (Hp[4] * Hp[8] - Hp[5] * Hp[7]) - Hp[1] * (Hp[3] * Hp[8] - Hp[5] * Hp[6]) +
                        Hp[2] * (Hp[3] * Hp[7] - Hp[4] * Hp[6]));
  double T1[9], T[9], U[9], X[9], Xi[9], Ut[9], Pm[9], Pc[9];
  m_mul_rn(H, P.H0inv, T1);
  m_mul_rn(T1, P.T0, T);
  for (int q = 0; q < 9; ++q) X[q] = T[q];
  for (int it = 0; it < 60; ++it) {   // X <- (X + X^-T) / 2 converges to U
    if (!m_inv_dev(X, Xi)) break;
    double d = 0;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        const double y = 0.5 * (X[3 * r + c] + Xi[3 * c + r]);
        d += fabs(y - X[3 * r + c]);
        U[3 * r + c] = y;
      }
    for (int q = 0; q < 9; ++q) X[q] = U[q];
    if (d < 1e-15) break;
  }
  for (int q = 0; q < 9; ++q) U[q] = X[q];
  m_tr(U, Ut);
  m_mul_rn(Ut, T, Pm);
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Pc[3 * r + c] = 0.5 * (Pm[3 * r + c] + Pm[3 * c + r]);
  double G1[9], G[9], E1[9];
  for (int q = 0; q < 9; ++q) E1[q] = Pc[q] - ((q % 4 == 0) ? 1.0 : 0.0);
  m_mul_rn(U, E1, G1);
  m_mul_rn(G1, Ut, G);
  double sig[6], eps[6], emax = 0;
  for (int i = 0; i < 6; ++i) {
    const int a = VO[i][0], b = VO[i][1];
    sig[i] = 0.5 * (S[3 * a + b] + S[3 * b + a]) / V;
    eps[i] = a == b ? G[3 * a + a] : G[3 * a + b] + G[3 * b + a];
    P.stress[i] = sig[i];
    P.strain[i] = eps[i];
    emax = fmax(emax, fabs(eps[i]));
  }
  if (P.done) return false;
  const long long k = ++P.k;
  if (k >= P.nsteps || emax >= P.max_strain) {
    P.done = 1;
    return false;
  }
  const double p = (double)k / (double)P.nsteps, pn = (double)(k + 1) / (double)P.nsteps;
  double rate[6], err[6], rmax = 0;
  for (int i = 0; i < 6; ++i) rmax = fmax(rmax, fabs(P.rate[i]));
  for (int i = 0; i < 6; ++i) {
    rate[i] = P.rate[i];
    err[i] = 0;
    if (!(P.mask & (1 << i))) rate[i] = (p3d_value(P, i, pn) - eps[i]) / dt;
    else err[i] = sig[i] - p3d_value(P, i, p);
  }
  if (P.first) {   // isotropic elastic estimate: D_SS de_S = dsig_S - D_SE de_E
    const double E = P.young, nu = P.poisson;
    const double lam = E * nu / ((1 + nu) * (1 - 2 * nu)), Gm = E / (2 * (1 + nu));
    double D[6][6];
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) D[i][j] = 0;
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) D[i][j] = lam;
      D[i][i] = lam + 2 * Gm;
      D[3 + i][3 + i] = Gm;
    }
    int idx[6], m = 0;
    for (int i = 0; i < 6; ++i)
      if (P.mask & (1 << i)) idx[m++] = i;
    double A[6][7];
    for (int r = 0; r < m; ++r) {
      const int i = idx[r];
      double rhs = p3d_value(P, i, pn) - sig[i];
      for (int j = 0; j < 6; ++j)
        if (!(P.mask & (1 << j))) rhs -= D[i][j] * rate[j] * dt;
      for (int c = 0; c < m; ++c) A[r][c] = D[i][idx[c]];
      A[r][m] = rhs;
    }
    for (int c = 0; c < m; ++c) {
      int piv = c;
      for (int r = c + 1; r < m; ++r)
        if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
      for (int q = 0; q <= m; ++q) {
        const double tq = A[c][q];
        A[c][q] = A[piv][q];
        A[piv][q] = tq;
      }
      for (int r = 0; r < m; ++r) {
        if (r == c) continue;
        const double f = A[r][c] / A[c][c];
        for (int q = c; q <= m; ++q) A[r][q] -= f * A[c][q];
      }
    }
    for (int r = 0; r < m; ++r) rate[idx[r]] = A[r][m] / A[r][r] / dt;
    P.first = 0;
  } else {   // stress error extrapolated one step decides the sign of mod x max |rate|
    for (int i = 0; i < 6; ++i) {
      if (!(P.mask & (1 << i))) continue;
      const double pred = 2 * err[i] - P.err[i];
      if (pred > 0) rate[i] -= rmax * P.mod;
      else if (pred < 0) rate[i] += rmax * P.mod;
    }
  }
  double Ed[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < 6; ++i) {
    rate[i] = fmin(fmax(rate[i], -P.max_rate), P.max_rate);
    P.rate[i] = rate[i];
    P.err[i] = err[i];
    const int a = VO[i][0], b = VO[i][1];
    if (a == b) {
      Ed[3 * a + a] = dt * rate[i];
    } else {
      Ed[3 * a + b] = 0.5 * dt * rate[i];
      Ed[3 * b + a] = 0.5 * dt * rate[i];
    }
  }
  double A1[9], A2[9], Pn[9], Tn[9], Ti[9];
  m_mul_rn(Ut, Ed, A1);
  m_mul_rn(A1, U, A2);
  for (int q = 0; q < 9; ++q) Pn[q] = Pc[q] + A2[q];
  m_mul_rn(U, Pn, Tn);
  if (!m_inv_dev(T, Ti)) return false;
  m_mul_rn(Tn, Ti, L);
  for (int q = 0; q < 9; ++q) L[q] = (L[q] - ((q % 4 == 0) ? 1.0 : 0.0)) / dt;
  return true;
}

// Advance of one (sub-)scene's cell and clock.
__device__ void cell_advance(CellState *__restrict__ cs, const double *servo, P3d *p3d = nullptr) {
  const double dt = cs->dt;
  if (cs->periodic) {
    double Hp[9], H[9], Lp[9], L[9], dL[9], W[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      Hp[q] = cs->H[q];
      H[q] = cs->Hnext[q];
      Lp[q] = cs->L[q];
      L[q] = Lp[q];
      dL[q] = 0.0;   // L - Lprev after the assignment above
    }
    if (servo) {
      // PeriTriaxController: new diagonal gradient from this step's contacts (their
      // stress and stiffness in the cell Hprev they were computed in), effective from
      // the next step; the partials are summed in block order
      double acc[6] = {0, 0, 0, 0, 0, 0};
      for (int b = 0; b < kServoBlocks; ++b)
        for (int q = 0; q < 6; ++q) acc[q] += servo[6 * b + q];
      const double V = fabs(Hp[0] * (Hp[4] * Hp[8] - Hp[5] * Hp[7]) -
                            Hp[1] * (Hp[3] * Hp[8] - Hp[5] * Hp[6]) +
                            Hp[2] * (Hp[3] * Hp[7] - Hp[4] * Hp[6]));
      for (int a = 0; a < 3; ++a) {
        double rate;
        if (cs->stress_mask & (1 << a)) {
          const double sa = acc[a] / V, Ka = acc[3 + a] / V;
          const double want = (1 - cs->grow_damping) * (cs->goal[a] - sa);
          if (Ka > 0) rate = want / (Ka * (dt * cs->glob_update));
          else rate = want > 0 ? cs->max_rate[a] : (want < 0 ? -cs->max_rate[a] : 0.0);
          rate = fmin(fmax(rate, -cs->max_rate[a]), cs->max_rate[a]);
        } else {
          rate = cs->goal[a];
        }
        L[4 * a] = rate;
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) dL[q] = L[q] - Lp[q];
    }
    if (p3d && p3d->has_next) {
      // the controller's gradient (k_p3d_update), effective from the next step like
      // Cell.velGrad
      for (int q = 0; q < 9; ++q) {
        L[q] = p3d->Lnext[q];
        dL[q] = L[q] - Lp[q];
      }
      p3d->has_next = 0;
    }
    // a cell that stays diagonal (every matrix of the state and the new gradient) takes
    // the diagonal products only: the same values, far fewer FP64 instructions
    const bool diag = !cs->sheared && !offdiag_nonzero(L);
    if (diag) {
#pragma unroll
      for (int q = 0; q < 9; ++q) W[q] = (q % 4 == 0) ? __dmul_rn(Lp[q], Hp[q]) : 0.0;
    } else {
      m_mul_rn(Lp, Hp, W);
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      cs->Hprev[q] = Hp[q];
      cs->H[q] = H[q];
      cs->Lprev[q] = Lp[q];
      cs->L[q] = L[q];
      cs->dL[q] = dL[q];
      cs->W[q] = W[q];
    }
    cs->dl_zero = !(nonzero_bits(dL[0]) | nonzero_bits(dL[4]) | nonzero_bits(dL[8]) |
                    offdiag_nonzero(dL));
    if (diag) {
      derive_next_diag(cs, H, L, dt);
      for (int k = 0; k < 3; ++k) {
        cs->dHf[4 * k] = (float)(H[4 * k] - cs->Href[4 * k]);
        cs->Wf[4 * k] = (float)W[4 * k];
      }
    } else {
      derive_next_local(cs, H, L, dt);
      bool off = offdiag_nonzero(H) | offdiag_nonzero(Hp) | offdiag_nonzero(L) |
                 offdiag_nonzero(Lp) | offdiag_nonzero(cs->Href);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        cs->dHf[q] = (float)(H[q] - cs->Href[q]);
        cs->Wf[q] = (float)W[q];
      }
      cs->sheared = off ? 1 : 0;
    }
  }
  cs->iter += 1;
  cs->time = __dadd_rn(cs->time, dt);
  cs->dt_law = dt;
}

// Peri3dController update of sub-scene 0 (one thread), between the integration and
// the cell advance of a step that was not skipped: the gradient it computes is
// picked up by that cell advance.
__global__ void k_p3d_update(const CellState *cs, const DevStatus *ds, P3d *p3d, const double *part) {
  if (ds->pending || !p3d->on) return;
  double Hp[9], H[9], L[9];
  for (int q = 0; q < 9; ++q) {
    Hp[q] = cs->H[q];
    H[q] = cs->Hnext[q];
  }
  if (p3d_update(*p3d, part, Hp, H, cs->dt, L)) {
    for (int q = 0; q < 9; ++q) p3d->Lnext[q] = L[q];
    p3d->has_next = 1;
  }
}

// One thread per sub-scene.  Every block reads "pending" before it counts itself
// in; the last block to arrive (so every block has read it) turns a collider
// request into "pending" and counts the step, so no block can see the flag of the
// step it is advancing.
__global__ void k_cell_advance(CellState *cs, int nsub, DevStatus *ds, const double *servo,
                               P3d *p3d) {
  const bool skip = *(volatile int *)&ds->pending;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (!skip && q < nsub && cs[q].alive)
    cell_advance(cs + q, q == 0 ? servo : nullptr, q == 0 ? p3d : nullptr);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int arrived = atomicAdd(&ds->arrive, 1);
    if (arrived == (int)gridDim.x - 1) {
      ds->arrive = 0;
      if (!skip) {
        ds->steps += 1;
        if (*(volatile int *)&ds->request) ds->pending = 1;
      }
    }
  }
}

__global__ void k_gather_forces(Bodies b, Table t, const Mat *__restrict__ mats,
                                const CellState *__restrict__ cs, SceneConst sc, long long cap,
                                double4_32a *Fo, double4_32a *To, int mixed) {
  const long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl >= sc.N) return;
  const int s = (int)sl;
  double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
  if (mixed) {
    float Ff[3], Tf[3];
    gather_rows_f32(t, s, Ff, Tf);
    for (int q = 0; q < 3; ++q) { F[q] = Ff[q]; T[q] = Tf[q]; }
  } else {
    gather_rows(t, s, F, T);
  }
  const uint8_t flags = b.flags[s];
  if (sc.walls && (flags & 0x7e)) {
    const CellState &c = cs[sc.multi ? b.sid[s] : 0];
    const int wmat = c.wall_mat;
    const double r = b.pos[s].w;
    for (int wi = 0; wi < 6; ++wi) {
      if (!(flags & (2 << wi))) continue;
      const double4_32a h = b.whist[wi * cap + s];
      const int ax = wi >> 1;
      const double sn = h.w >= 0 ? 1.0 : -1.0;
      const double Fn = fabs(h.w);
      double kn, ks, tanphi;
      wall_phys(mats, wmat, b.mat[s], r, kn, ks, tanphi, c.law);
      const double pen = wall_pen(Fn, kn, c.law);
      double n[3] = {0, 0, 0};
      n[ax] = sn;
      const double F2[3] = {Fn * n[0] + h.x, Fn * n[1] + h.y, Fn * n[2] + h.z};
      const double arm = -(r - 0.5 * pen);
      const double a[3] = {arm * n[0], arm * n[1], arm * n[2]};
      F[0] += F2[0]; F[1] += F2[1]; F[2] += F2[2];
      T[0] += a[1] * F2[2] - a[2] * F2[1];
      T[1] += a[2] * F2[0] - a[0] * F2[2];
      T[2] += a[0] * F2[1] - a[1] * F2[0];
    }
  }
  Fo[s] = make_double4_32a(F[0], F[1], F[2], 0);
  To[s] = make_double4_32a(T[0], T[1], T[2], 0);
}

// ---- deterministic block reductions of K doubles
template <int K>
__device__ inline void block_reduce_store(double (&v)[K], double *partials) {
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

// ke, sum |F contact| over free bodies, number of free bodies
__global__ void k_body_stats(Bodies b, const double4_32a *__restrict__ F, long long N, double *partials) {
  double v[3] = {0, 0, 0};
  for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < N; i += (long long)gridDim.x * kT) {
    const double4_32a u = b.vel[i], w = b.angvel[i], mp = b.mprop[i];
    v[0] += 0.5 * mp.x * (u.x * u.x + u.y * u.y + u.z * u.z) + 0.5 * mp.y * (w.x * w.x + w.y * w.y + w.z * w.z);
    if (!(b.flags[i] & 1)) {
      const double4_32a f = F[i];
      v[1] += sqrt(f.x * f.x + f.y * f.y + f.z * f.z);
      v[2] += 1.0;
    }
  }
  block_reduce_store<3>(v, partials);
}

// real sphere-sphere rows: count, sum |F|, Love-Weber stress sum F_i (x1 - x2')_j
__global__ void k_row_stats(Table t, double *partials, int mixed) {
  double v[11] = {0};
  for (long long k = (long long)blockIdx.x * kT + threadIdx.x; k < t.P; k += (long long)gridDim.x * kT) {
    double4_32a f, m, n;
    if (mixed) {
      if (t.g32[k].w == 0.0f) continue;
      const float4 a = t.oFM32[2 * k], c = t.oFM32[2 * k + 1], h = t.hn32[k];
      f = make_double4_32a(a.x, a.y, a.z, a.w);
      m = make_double4_32a(c.x, c.y, c.z, c.w);
      n = make_double4_32a(h.x, h.y, h.z, h.w);
    } else {
      if (t.hfs[k].w == 0.0) continue;
      f = t.oFM[2 * k]; m = t.oFM[2 * k + 1]; n = t.hn[k];
    }
    const double l = f.w + m.w;
    v[0] += 1.0;
    v[1] += sqrt(f.x * f.x + f.y * f.y + f.z * f.z);
    const double F3[3] = {f.x, f.y, f.z}, br[3] = {-l * n.x, -l * n.y, -l * n.z};
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) v[2 + 3 * a + c] += F3[a] * br[c];
  }
  block_reduce_store<11>(v, partials);
}

// wall contacts: count, sum |F|
__global__ void k_wall_stats(Bodies b, SceneConst sc, const Mat *__restrict__ mats, long long cap,
                             double *partials) {
  double v[2] = {0, 0};
  for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < sc.N; i += (long long)gridDim.x * kT) {
    const uint8_t fl = b.flags[i];
    if (!(fl & 0x7e)) continue;
    for (int wi = 0; wi < 6; ++wi) {
      if (!(fl & (2 << wi))) continue;
      const double4_32a h = b.whist[wi * cap + i];
      const int ax = wi >> 1;
      const double sn = h.w >= 0 ? 1.0 : -1.0;
      double F2[3] = {h.x, h.y, h.z};
      F2[ax] += sn * fabs(h.w);
      v[0] += 1.0;
      v[1] += sqrt(F2[0] * F2[0] + F2[1] * F2[1] + F2[2] * F2[2]);
    }
  }
  block_reduce_store<2>(v, partials);
}

inline unsigned blocks(long long n) { return (unsigned)((n + kT - 1) / kT); }

// GlobalStiffnessTimeStepper (section 2.1.5, eq. 2.12-2.14): per body the diagonal of
// its translational stiffness sum (kn - ks) n_i^2 + ks and rotational stiffness
// sum ks d^2 (1 - n_i^2) over its real contacts (spheres and walls, d = r - pen/2),
// the smallest sqrt(2) sqrt(m / K) over its degrees of freedom, and the minimum over
// the bodies of each sub-scene into keys[sub] (bit patterns of positive doubles
// order like the values, so an integer atomic min is exact and order-free).
__device__ inline void stiff_add(double Kt[3], double Kr[3], double kn, double ks, const double n[3],
                                 double d, int law, double pen) {
  if (law) {   // Hertz-Mindlin tangents: k_n = 3/2 kno pen^1/2, k_s = kso pen^1/2
    const double sq = sqrt(pen);
    kn = 1.5 * kn * sq;
    ks = ks * sq;
  }
  for (int i = 0; i < 3; ++i) {
    const double ni2 = n[i] * n[i];
    Kt[i] += (kn - ks) * ni2 + ks;
    Kr[i] += ks * d * d * (1.0 - ni2);
  }
}

__global__ void k_stiffness(Bodies b, Table t, const CellState *__restrict__ cs,
                            const Mat *__restrict__ mats, long long N, long long cap, int mixed,
                            int multi, int walls, unsigned long long *keys) {
  const long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  const int lane = threadIdx.x & 31;
  unsigned long long key = 0x7ff0000000000000ull;   // +inf: no contact
  int q = -1;
  if (sl < N) {
    const int s = (int)sl;
    q = multi ? b.sid[s] : 0;
    const int law = cs[q].law;
    const double rs = b.pos[s].w;
    double Kt[3] = {0, 0, 0}, Kr[3] = {0, 0, 0};
    auto row = [&](long long k, bool first) {
      double kn, ks, n[3], d;
      if (mixed) {
        const float4 g = t.g32[k];
        if (g.w == 0.0f) return;
        const float4 h = t.hn32[k];
        kn = g.w; ks = h.w; n[0] = h.x; n[1] = h.y; n[2] = h.z;
        d = first ? t.oFM32[2 * k].w : t.oFM32[2 * k + 1].w;
      } else {
        const double4_32a f = t.hfs[k];
        if (f.w == 0.0) return;
        const double4_32a h = t.hn[k];
        kn = f.w; ks = h.w; n[0] = h.x; n[1] = h.y; n[2] = h.z;
        d = first ? t.oFM[2 * k].w : t.oFM[2 * k + 1].w;
      }
      stiff_add(Kt, Kr, kn, ks, n, d, law, 2.0 * (rs - d));   // d = r - pen/2
    };
    // increasing partner id, as the force gather
    for (int e = t.down_start[s]; e < t.down_start[s + 1]; ++e) row(t.down[e], false);
    for (int k = t.row_start[s]; k < t.row_start[s + 1]; ++k) row(k, true);
    const uint8_t fl = b.flags[s];
    const double4_32a p = b.pos[s];
    const double r = p.w;
    const CellState &c = cs[q];
    if (walls && c.wall_mask) {
      // this step's wall contacts (the integrator evaluates them after this kernel):
      // the same test on the same positions, pen = r - |x_a - w|
      double kn, ks, tp;
      wall_phys(mats, c.wall_mat, b.mat[s], r, kn, ks, tp, c.law);
      const double x[3] = {p.x, p.y, p.z};
      for (int wi = 0; wi < 6; ++wi) {
        if (!(c.wall_mask & (1 << wi))) continue;
        const int ax = wi >> 1;
        const double dist = x[ax] - ((wi & 1) ? c.box_hi[ax] : c.box_lo[ax]);
        if (!(fabs(dist) < r)) continue;
        double n[3] = {0, 0, 0};
        n[ax] = 1.0;   // only n_i^2 enters
        stiff_add(Kt, Kr, kn, ks, n, r - 0.5 * (r - fabs(dist)), c.law, r - fabs(dist));
      }
    }
    if (!(fl & 1)) {
      const double4_32a mp = b.mprop[s];   // m, I (true values)
      double best = INFINITY;
      for (int i = 0; i < 3; ++i) {
        if (Kt[i] > 0) best = fmin(best, sqrt(2.0) * sqrt(mp.x / Kt[i]));
        if (Kr[i] > 0) best = fmin(best, sqrt(2.0) * sqrt(mp.y / Kr[i]));
      }
      key = (unsigned long long)__double_as_longlong(best);
      // density scaling on an update step of this sub-scene: f = (target / (safety t_b))^2,
      // kept as 1/f; a body without contacts keeps its factor
      if (c.dscale && best < INFINITY && (c.iter % c.tstep_interval) == 0) {
        const double q_ = (c.tstep_safety * best) / c.target_dt;
        b.rdsc[s] = q_ * q_;
      }
    }
  }
  // one atomic per warp when its bodies share a sub-scene (the usual case)
  const int q0 = __shfl_sync(0xffffffffu, q, 0);
  if (__all_sync(0xffffffffu, q == q0 || q < 0)) {
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_down_sync(0xffffffffu, key, o);
      key = v < key ? v : key;
    }
    if (lane == 0 && q0 >= 0 && key != 0x7ff0000000000000ull) atomicMin(&keys[q0], key);
  } else if (q >= 0 && key != 0x7ff0000000000000ull) {
    atomicMin(&keys[q], key);
  }
}

// Apply the new step to the sub-scenes due for an update this step (iteration
// count a multiple of their interval), re-derive the next cell with it, and reset
// every key.
__global__ void k_dt_apply(CellState *cs, int nsub, const DevStatus *ds, unsigned long long *keys) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nsub) return;
  const unsigned long long key = keys[q];
  keys[q] = 0x7ff0000000000000ull;
  if (ds->pending) return;
  CellState *c = cs + q;
  if (!c->alive || !c->tstep || (c->iter % c->tstep_interval) != 0) return;
  double dt = key == 0x7ff0000000000000ull ? c->tstep_default
                                           : c->tstep_safety * __longlong_as_double((long long)key);
  if (c->tstep_max > 0 && dt > c->tstep_max) dt = c->tstep_max;
  if (c->dscale) dt = c->target_dt;   // density scaling: every body is scaled to this step
  c->dt_law = c->dt;   // the walls' law of this step still uses the step's old dt
  c->dt = dt;
  if (c->periodic) derive_next(c);
}
}  // namespace

namespace {
__global__ void k_dscale_reset(Bodies b, long long N, int multi, int sub) {
  const long long sl = (long long)blockIdx.x * kT + threadIdx.x;
  if (sl < N && (!multi || b.sid[sl] == sub)) b.rdsc[sl] = 1.0;
}
}  // namespace

void launch_dscale_reset(const Bodies &b, long long N, int multi, int sub, cudaStream_t st) {
  if (N > 0) k_dscale_reset<<<(unsigned)((N + kT - 1) / kT), kT, 0, st>>>(b, N, multi, sub);
}

void launch_integrate(const StepDesc *d, const StepDesc &h, bool desc, const CellState *cs,
                      DevStatus *ds, const Mat *mats, int mixed, int block, cudaStream_t st) {
  const long long N = h.sc.N;
  if (N <= 0) return;
  const int feat = (h.sc.walls ? 1 : 0) | (h.sc.sheared ? 2 : 0);
  // kernels without the sphere-wall or sheared-cell branches when no sub-scene needs them
#define DEM_I(K, B, F, D) K<B, F, D><<<(unsigned)((N + B - 1) / B), B, 0, st>>>(d, h, cs, ds, mats)
#define DEM_I_F(K, B, D) switch (feat) { case 0: DEM_I(K, B, 0, D); break; case 1: DEM_I(K, B, 1, D); break; \
                                         case 2: DEM_I(K, B, 2, D); break; default: DEM_I(K, B, 3, D); }
#define DEM_I_B(K, D) if (block == 128) { DEM_I_F(K, 128, D) } else if (block == 512) { DEM_I_F(K, 512, D) } else { DEM_I_F(K, 256, D) }
  if (mixed) {
    if (desc) { DEM_I_B(k_integrate_mixed, true) } else { DEM_I_B(k_integrate_mixed, false) }
  } else {
    if (desc) { DEM_I_B(k_integrate, true) } else { DEM_I_B(k_integrate, false) }
  }
#undef DEM_I_B
#undef DEM_I_F
#undef DEM_I
}

void launch_cell_advance(CellState *cs, int nsub, DevStatus *ds, const double *servo_partials,
                         cudaStream_t st, P3d *p3d, const double *p3d_partials) {
  const int threads = nsub < 128 ? 32 * ((nsub + 31) / 32) : 128;
  if (p3d) k_p3d_update<<<1, 1, 0, st>>>(cs, ds, p3d, p3d_partials);
  k_cell_advance<<<(nsub + threads - 1) / threads, threads, 0, st>>>(cs, nsub, ds, servo_partials,
                                                                     p3d);
}

void launch_timestepper(const Bodies &b, const Table &t, CellState *cs, int nsub,
                        const DevStatus *ds, const Mat *mats, long long N, long long cap,
                        int mixed, int multi, int walls, unsigned long long *keys,
                        cudaStream_t st) {
  if (N > 0)
    k_stiffness<<<blocks(N), kT, 0, st>>>(b, t, cs, mats, N, cap, mixed, multi, walls, keys);
  k_dt_apply<<<(nsub + 127) / 128, 128, 0, st>>>(cs, nsub, ds, keys);
}

void launch_gather_forces(const Bodies &b, const Table &t, const Mat *mats, const CellState *cs,
                          const SceneConst &sc, long long cap, double4_32a *F, double4_32a *T,
                          int mixed, cudaStream_t st) {
  if (sc.N > 0)
    k_gather_forces<<<blocks(sc.N), kT, 0, st>>>(b, t, mats, cs, sc, cap, F, T, mixed);
}

__global__ void k_gather_ids(const int *__restrict__ slot_of_id, long long n,
                             const double4_32a *__restrict__ src, double4_32a *dst) {
  const long long i = (long long)blockIdx.x * kT + threadIdx.x;
  if (i < n) dst[i] = src[slot_of_id[i]];
}
__global__ void k_gather_ids_f(const int *__restrict__ slot_of_id, long long n,
                               const float4 *__restrict__ src, float4 *dst) {
  const long long i = (long long)blockIdx.x * kT + threadIdx.x;
  if (i < n) dst[i] = src[slot_of_id[i]];
}

void launch_gather_ids(const int *slot_of_id, long long n, const double4_32a *src,
                       double4_32a *dst, cudaStream_t st) {
  if (n > 0) k_gather_ids<<<blocks(n), kT, 0, st>>>(slot_of_id, n, src, dst);
}
void launch_gather_ids_f(const int *slot_of_id, long long n, const float4 *src, float4 *dst,
                         cudaStream_t st) {
  if (n > 0) k_gather_ids_f<<<blocks(n), kT, 0, st>>>(slot_of_id, n, src, dst);
}

int stats_blocks(long long n) {
  long long b = (n + kT - 1) / kT;
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

void launch_body_stats(const Bodies &b, const double4_32a *F, long long N, double *partials,
                       cudaStream_t st) {
  k_body_stats<<<stats_blocks(N), kT, 0, st>>>(b, F, N, partials);
}

void launch_row_stats(const Table &t, const Bodies &b, double *partials, int mixed,
                      cudaStream_t st) {
  (void)b;
  k_row_stats<<<stats_blocks(t.P), kT, 0, st>>>(t, partials, mixed);
}

void launch_wall_stats(const Bodies &b, const SceneConst &sc, const Mat *mats, long long cap,
                           double *partials, cudaStream_t st) {
  k_wall_stats<<<stats_blocks(sc.N), kT, 0, st>>>(b, sc, mats, cap, partials);
}

}  // namespace dem
