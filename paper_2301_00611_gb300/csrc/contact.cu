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
// so this kernel is bound by the FP64 pipe rather than by its ~400 bytes of
// real-row traffic.  Two choices follow: real rows are queued per warp so that
// the law runs with every lane busy (non-real rows, ~45% of the table, would
// otherwise idle lanes through it), and square roots and divisions are taken
// from an FP32 estimate of 1/sqrt refined in FP64 to shorten the FP64 instruction stream.
#include "dem_internal.cuh"

namespace dem {

namespace {
constexpr int kQ = 64;   // per-warp queue of real rows (< 32 left over + 32 new)

// 1/sqrt(x) for x > 0 with four FP64-pipe instructions: the FP32
// hardware estimate y0 of the FP32 image of x (relative error below 4e-7), widened, then
// one third-order correction from the binomial series (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8
// + ..., e = 1 - x y0^2 (Householder's method of order two for 1/sqrt): y0 + e (y0/2 +
// e 3y0/8).  The narrowing and widening rebias the exponent on the integer pipe (every
// double<->float conversion is an FP64-pipe instruction), y0/2 is exact and 3y0/8 is
// formed in FP32 (it multiplies e^2 < 2e-13).  The omitted terms are below 2e-19, so the
// result is within one ulp of 1/sqrt(x).  x outside the FP32 normal range (including 0)
// takes the library's rsqrt.
__device__ __forceinline__ double rsqrt_refined(double x) {
  const long long xb = __double_as_longlong(x);
  const int ex = (int)(xb >> 52);   // biased exponent (x >= 0)
  if ((unsigned)(ex - 897) >= 252u) return rsqrt(x);
  const float yf = rsqrtf(__int_as_float((int)((xb >> 29) - (896LL << 23))));
  const double y0 = __longlong_as_double(((long long)__float_as_int(yf) << 29) + (896LL << 52));
  const double half = __longlong_as_double(__double_as_longlong(y0) - (1LL << 52));
  const double c = __longlong_as_double(((long long)__float_as_int(0.375f * yf) << 29) +
                                        (896LL << 52));
  const double e = fma(-(x * y0), y0, 1.0);
  return fma(e, fma(e, c, half), y0);
}

// What a row needs of its (sub-)scene's cell state: time step, diagonal of the cell
// H (image shift) and of W (velocity of a unit shift); all zero when aperiodic.
struct RowCell {
  double dt, H[3], W[3];
  int periodic, law, sheared;
};
__device__ __forceinline__ RowCell row_cell(const CellState &c) {
  RowCell r;
  r.dt = c.dt;
  r.periodic = c.periodic;
  r.law = c.law;
  r.sheared = c.sheared;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    r.H[i] = c.periodic ? c.H[4 * i] : 0.0;
    r.W[i] = c.periodic ? c.W[4 * i] : 0.0;
  }
  return r;
}

// One real row: Ip2 on creation, shear transport and increment, Law2, outputs.
// dx, dy, dz, l2 are the branch vector and its squared length from the exact test.
template <int kFeat>
__device__ __forceinline__ void real_row(const Table &t, const Bodies &b, const Mat *__restrict__ mats,
                                         long long k, double dx, double dy, double dz, double l2,
                                         double r1, double r2, const RowCell &rc,
                                         const CellState *__restrict__ cq) {
  const double dt = rc.dt;
  const int2 pr = t.pair[k];
  const double R = r1 + r2;
  double4_32a fs = t.hfs[k];
  double4_32a hn = t.hn[k];
  // 1/l from rsqrt_refined (instead of a square root and a division); l = l2 / l within
  // an ulp or two of the correctly rounded root
  const double il = rsqrt_refined(l2);
  const double l = l2 * il;
  const double nx = dx * il, ny = dy * il, nz = dz * il;   // eq. 2.7
  const double pen = R - l;                                  // penetrationDepth
  double kn = fs.w, ks = hn.w, tanphi;
  if (is_zero_bits(kn)) {   // kn == 0: a new contact
    const Mat &m1 = mats[b.mat[pr.x]], &m2 = mats[b.mat[pr.y]];
    if ((kFeat & 1) && rc.law) {   // Ip2_FrictMat_FrictMat_MindlinPhys: constants kno, kso
      mindlin_phys(m1, r1, m2, r2, kn, ks);
    } else {        // Ip2_FrictMat_FrictMat_FrictPhys (new contact)
      const double k1 = m1.young * (2 * r1), k2 = m2.young * (2 * r2);
      kn = k1 * k2 / (k1 + k2);
      const double s1 = m1.young * m1.poisson * (2 * r1), s2 = m2.young * m2.poisson * (2 * r2);
      ks = s1 * s2 / (s1 + s2);
    }
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
  const int cp = rc.periodic ? t.cpack[k] : 0;
  if (cp != 0) {   // velocity of the image of body 2 (the shift c moves with the cell;
                   // a row inside the cell has c = 0 and W c = 0 exactly)
    int i0, i1, i2;
    unpack_shift(cp, i0, i1, i2);
    const double c0 = i0, c1 = i1, c2 = i2;
    if ((kFeat & 2) && rc.sheared) {   // W c with the full image velocity matrix
      const double *W = cq->W;
      v2.x += W[0] * c0 + W[1] * c1 + W[2] * c2;
      v2.y += W[3] * c0 + W[4] * c1 + W[5] * c2;
      v2.z += W[6] * c0 + W[7] * c1 + W[8] * c2;
    } else {
      v2.x += rc.W[0] * c0;
      v2.y += rc.W[1] * c1;
      v2.z += rc.W[2] * c2;
    }
  }
  // 1. motion of the contact frame: -Fs x (n- x n) - Fs x (dt/2 n.(w1+w2) n)
  const double ax = hn.y * nz - hn.z * ny;
  const double ay = hn.z * nx - hn.x * nz;
  const double az = hn.x * ny - hn.y * nx;
  const double tw = 0.5 * dt * (nx * (w1.x + w2.x) + ny * (w1.y + w2.y) + nz * (w1.z + w2.z));
  const double bx = ax + tw * nx, by = ay + tw * ny, bz = az + tw * nz;
  double fx = fma(fs.z, by, fma(-fs.y, bz, fs.x));   // Fs - Fs x b, two fused steps
  double fy = fma(fs.x, bz, fma(-fs.z, bx, fs.y));
  double fz = fma(fs.y, bx, fma(-fs.x, by, fs.z));
  // 2. mutual motion: ratchet-free v12 (ScGeom), its part perpendicular to n
  const double rx = r2 * w2.x + r1 * w1.x, ry = r2 * w2.y + r1 * w1.y, rz = r2 * w2.z + r1 * w1.z;
  const double f = R * il;
  const double ux = f * (v2.x - v1.x) - (ry * nz - rz * ny);
  const double uy = f * (v2.y - v1.y) - (rz * nx - rx * nz);
  const double uz = f * (v2.z - v1.z) - (rx * ny - ry * nx);
  const double vn = nx * ux + ny * uy + nz * uz;
  // Hertz-Mindlin: shear stiffness kso pen^1/2 and normal force kno pen^3/2
  const double sq = ((kFeat & 1) && rc.law) ? sqrt(pen) : 1.0;
  const double kd = (ks * sq) * dt;
  fx -= kd * (ux - vn * nx);
  fy -= kd * (uy - vn * ny);
  fz -= kd * (uz - vn * nz);
  // Law2: normal force and Coulomb cap
  const double Fn = ((kFeat & 1) && rc.law) ? kn * pen * sq : kn * pen;
  const double maxFs = Fn * tanphi;
  const double fs2 = fx * fx + fy * fy + fz * fz;
  if (lt_nonneg(maxFs * maxFs, fs2)) {   // |Fs|^2 > (Fn tan phi)^2
    const double sc = maxFs * rsqrt_refined(fs2);
    fx *= sc; fy *= sc; fz *= sc;
  }
  const double Fx = Fn * nx + fx, Fy = Fn * ny + fy, Fz = Fn * nz + fz;
  // torques: T1 = (C - x1) x (-F) = d1 * M, T2 = (C - x2') x F = d2 * M, M = -(n x F)
  const double d1 = r1 - 0.5 * pen, d2 = r2 - 0.5 * pen;
  const double Mx = -(ny * Fz - nz * Fy), My = -(nz * Fx - nx * Fz), Mz = -(nx * Fy - ny * Fx);
  t.hfs[k] = make_double4_32a(fx, fy, fz, kn);
  t.hn[k] = make_double4_32a(nx, ny, nz, ks);
  t.oFM[2 * k] = make_double4_32a(Fx, Fy, Fz, d1);
  t.oFM[2 * k + 1] = make_double4_32a(Mx, My, Mz, d2);
}

// Queued real row: its index, branch vector, squared length, radii and sub-scene.
struct QRow {
  double dx, dy, dz, l2, r1, r2;
  long long k;
  int q;
};

// Each warp walks tiles of 32 consecutive rows (coalesced loads of the row and
// both bodies' positions).  The exact test runs on every row; rows that are not
// in contact are settled at once (reset when the contact was just lost), and the
// real ones are appended to a per-warp queue in shared memory.  Whenever the
// queue holds 32 rows every lane takes one, so the long FP64 law runs with all
// lanes busy instead of on the ~55% of lanes a plain row-per-thread pass leaves
// active.  Each row is still computed by one lane with the same arithmetic, so
// the results do not depend on which lane (or which pass) takes it.
// Sub-scenes (multi): each row takes its cell state from the sub-scene of body 1
// (both bodies of a row always belong to the same sub-scene).
// Register budget by block size (the autotuner picks): 128-thread blocks at six per SM
// (80 registers, a few spilled), 256-thread blocks at two per SM (no spills).
// kDesc: the table and bodies come from the device descriptor (a captured batch of
// steps stays valid across collider runs); otherwise from the launch parameters,
// which the kernel reads straight from the constant bank (fewer registers).
// kFeat: bit 0 some sub-scene uses the Hertz-Mindlin law, bit 1 some periodic cell is
// sheared; each variant carries only the branches it needs (they cost registers).
template <int kT, int kFeat, bool kDesc>
__global__ void __launch_bounds__(kT, kT == 128 ? 6 : 2) k_contact(const StepDesc *__restrict__ d,
                                                          Table tp, Bodies bp,
                                                          const CellState *__restrict__ cs,
                                                          const DevStatus *__restrict__ ds,
                                                          const Mat *__restrict__ mats, int multi) {
  constexpr int kWarps = kT / 32;
  const Table &t = kDesc ? d->t : tp;
  const Bodies &b = kDesc ? d->b : bp;
  if (ds->pending) return;
  __shared__ QRow q[kWarps][kQ];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  QRow *wq = q[wi];
  const RowCell rc0 = row_cell(cs[0]);
  const long long P = t.P;
  const long long stride = (long long)gridDim.x * kT;
  int cnt = 0;   // warp-uniform queue length
  for (long long base = (long long)blockIdx.x * kT + wi * 32; base < P; base += stride) {
    const long long k = base + lane;
    bool real = false;
    double dx = 0, dy = 0, dz = 0, l2 = 0, r1 = 0, r2 = 0;
    int sq = 0;
    // rows of neighbours inside the cell have no shift (c = 0, h = H c = 0 exactly): a
    // warp whose 32 rows all have none skips the conversions and products
    const int cp = k < P ? t.cpack[k] : 0;
    const bool any_shift = __any_sync(0xffffffffu, cp != 0);
    if (k < P) {
      const int2 pr = t.pair[k];
      const double4_32a p1 = b.pos[pr.x];
      const double4_32a p2 = b.pos[pr.y];
      if (multi) sq = b.sid[pr.x];
      const int periodic = multi ? cs[sq].periodic : rc0.periodic;
      if (periodic && any_shift) {
        double h0, h1, h2;
        int i0, i1, i2;
        unpack_shift(cp, i0, i1, i2);
        const double c0 = i0, c1 = i1, c2 = i2;
        if ((kFeat & 2) && (multi ? cs[sq].sheared : rc0.sheared)) {
          // H c of a sheared cell, each row summed left to right as the oracle writes it
          const double *H = cs[sq].H;
          h0 = __dadd_rn(__dadd_rn(__dmul_rn(H[0], c0), __dmul_rn(H[1], c1)), __dmul_rn(H[2], c2));
          h1 = __dadd_rn(__dadd_rn(__dmul_rn(H[3], c0), __dmul_rn(H[4], c1)), __dmul_rn(H[5], c2));
          h2 = __dadd_rn(__dadd_rn(__dmul_rn(H[6], c0), __dmul_rn(H[7], c1)), __dmul_rn(H[8], c2));
        } else {
          // diagonal cell: one term per axis, the same value the full product gives (the
          // off-diagonal terms are exact zeros)
          const double H0 = multi ? cs[sq].H[0] : rc0.H[0];
          const double H1 = multi ? cs[sq].H[4] : rc0.H[1];
          const double H2 = multi ? cs[sq].H[8] : rc0.H[2];
          h0 = __dmul_rn(H0, c0);
          h1 = __dmul_rn(H1, c1);
          h2 = __dmul_rn(H2, c2);
        }
        // branch vector x2 + H c - x1 (eq. 2.2, second pass; R1 of the oracle)
        dx = __dsub_rn(__dadd_rn(p2.x, h0), p1.x);
        dy = __dsub_rn(__dadd_rn(p2.y, h1), p1.y);
        dz = __dsub_rn(__dadd_rn(p2.z, h2), p1.z);
      } else {   // no shift in the warp: x2 + 0 - x1 is x2 - x1
        dx = __dsub_rn(p2.x, p1.x);
        dy = __dsub_rn(p2.y, p1.y);
        dz = __dsub_rn(p2.z, p1.z);
      }
      // the exact test
      l2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
      const double R = __dadd_rn(p1.w, p2.w);
      r1 = p1.w; r2 = p2.w;
      real = lt_nonneg(l2, __dmul_rn(R, R));   // l2 < R^2
      if (!real && !is_zero_bits(t.hfs[k].w)) {   // contact lost (u_N > 0): back to potential
        const double4_32a z = make_double4_32a(0, 0, 0, 0);
        t.hfs[k] = z; t.hn[k] = z; t.oFM[2 * k] = z; t.oFM[2 * k + 1] = z;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, real);
    if (real) {
      const int at = cnt + __popc(m & ((1u << lane) - 1u));
      wq[at] = QRow{dx, dy, dz, l2, r1, r2, k, sq};
    }
    cnt += __popc(m);
    __syncwarp();
    if (cnt >= 32) {
      const QRow e = wq[lane];
      real_row<kFeat>(t, b, mats, e.k, e.dx, e.dy, e.dz, e.l2, e.r1, e.r2,
                       multi ? row_cell(cs[e.q]) : rc0, cs + e.q);
      __syncwarp();
      if (lane < cnt - 32) wq[lane] = wq[lane + 32];
      cnt -= 32;
      __syncwarp();
    }
  }
  // Leftovers (< 32 per warp) are pooled over the block and taken one per thread, so
  // the block runs at most one partly filled pass of the law instead of one per warp.
  __shared__ int left[kWarps];
  if (lane == 0) left[wi] = cnt;
  __syncthreads();
  int from = 0, pos = threadIdx.x;
  for (; from < kWarps && pos >= left[from]; ++from) pos -= left[from];
  if (from < kWarps) {
    const QRow e = q[from][pos];
    real_row<kFeat>(t, b, mats, e.k, e.dx, e.dy, e.dz, e.l2, e.r1, e.r2,
                     multi ? row_cell(cs[e.q]) : rc0, cs + e.q);
  }
}
}  // namespace

void launch_contact(const StepDesc *d, const StepDesc &h, bool desc, long long rows,
                    const CellState *cs, const DevStatus *ds, const Mat *mats, int multi,
                    int feat, int nsm, int block, int per_sm, cudaStream_t st) {
  if (rows <= 0) return;
  long long need = (rows + block - 1) / block;
  long long cap = (long long)nsm * per_sm;   // persistent grid: per_sm blocks per SM
  unsigned grid = (unsigned)(need < cap ? need : cap);
#define DEM_C(B, F, D) k_contact<B, F, D><<<grid, B, 0, st>>>(d, h.t, h.b, cs, ds, mats, multi)
#define DEM_CB(F, D) if (block == 128) DEM_C(128, F, D); else DEM_C(256, F, D);
#define DEM_CF(D) switch (feat & 3) { case 0: DEM_CB(0, D) break; case 1: DEM_CB(1, D) break; \
                                      case 2: DEM_CB(2, D) break; default: DEM_CB(3, D) }
  if (desc) { DEM_CF(true) } else { DEM_CF(false) }
#undef DEM_CF
#undef DEM_CB
#undef DEM_C
}

}  // namespace dem
