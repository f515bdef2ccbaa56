// Internal declarations of the GB300 DEM library: device data layout, the
// per-scene cell state and the host-side launchers of every kernel.
//
// Layout in HBM (one scene):
//   bodies, in "slot" order (Morton order of the collider grid cell, ties by id),
//   struct-of-arrays of 32-byte records so that one body field is one sector:
//     pos    double4_32a (x, y, z, r)         vel    double4_32a (vx, vy, vz, 0)
//     angvel double4_32a (wx, wy, wz, 0)      ori    double4_32a (qw, qx, qy, qz)
//     xref   double4_32a (x at the last collider run, 0)
//     mprop  double4_32a (m, I, 1/m, 1/I)     id int, mat int, flags uint8
//     whist  double4_32a[6][N] wall-contact history (Fs xyz, signed Fn)
//   contact table (one row per potential interaction = collider candidate),
//   rows grouped by s1 in slot order:
//     pair int2, cpack int (cell shift of s2, 3 x 10-bit signed),
//     hfs double4_32a (Fs on body 2, kn)       kn == 0 <=> not in contact
//     hn  double4_32a (normal of the last step, ks), tanphi double,
//     oFM[2k] double4_32a (F on body 2, arm d1), oFM[2k+1] (-(n x F), arm d2): one
//     64-byte record per row, so a row's outputs are read with one access
//   so that the torques are T1 = d1*oM, T2 = d2*oM (section 2.1.4 with the
//   contact point of eq. 2.8: C - x1 = d1 n, C - x2' = -d2 n).
//   Row (s1, s2): s1 is the body with the smaller id (the canonical id1 < id2).
//   Per-body CSR over the table: row_start[s] (rows with s1 = s, contiguous, sorted
//   by the id of s2) and down_start/down (rows with s2 = s, sorted by the id of s1),
//   so the force sum of every body is a gather in increasing partner id (down list,
//   then own rows): one order that depends on the ids only, with no atomics on forces.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace dem {

constexpr int kMaxMat = 4096;
constexpr int kMaxGridSide = 256;   // cells per axis (Morton code of 24 bits)

// error bits set by kernels (DevStatus::error)
enum : int {
  kErrNonFinite = 1,
  kErrHistoryLost = 2,
  kErrShiftRange = 4,
};

struct Mat {
  double density, young, poisson, tanphi;
  // Hertz-Mindlin compliances of the material: (1 - nu^2) / E and (2 - nu) / G with
  // G = E / (2 (1 + nu)), so that a pair's E* and shear constant are 1 / (sum)
  double hz_e, hz_g;
};

// Ip2 of the Hertz-Mindlin law (Ip2_FrictMat_FrictMat_MindlinPhys): kno = 4/3 E* sqrt(R*)
// and kso = 8 sqrt(R*) / ((2 - nu1)/G1 + (2 - nu2)/G2) with 1/E* = sum (1 - nu^2)/E,
// G = E / (2 (1 + nu)); r2 < 0 stands for a wall (R* = r1).  Stored where the linear
// law keeps kn and ks; the law takes Fn = kno pen^3/2 and ks = kso pen^1/2.
__host__ __device__ inline void mindlin_phys(const Mat &m1, double r1, const Mat &m2, double r2,
                                             double &kno, double &kso) {
  const double Rs = r2 < 0 ? r1 : r1 * r2 / (r1 + r2);
  const double sR = sqrt(Rs);
  kno = 4.0 / 3.0 * sR / (m1.hz_e + m2.hz_e);
  kso = 8.0 * sR / (m1.hz_g + m2.hz_g);
}
inline void mindlin_compliances(Mat &m) {
  m.hz_e = (1 - m.poisson * m.poisson) / m.young;
  m.hz_g = (2 - m.poisson) / (m.young / (2 * (1 + m.poisson)));
}

// penetration of a wall contact from its stored normal force (linear: Fn = kn pen;
// Hertz: Fn = kno pen^3/2)
__host__ __device__ inline double wall_pen(double Fn, double k, int law) {
  return law ? cbrt((Fn / k) * (Fn / k)) : Fn / k;
}

struct Bodies {
  double4_32a *pos, *vel, *angvel, *ori, *xref, *mprop;
  int *id, *mat;
  int *sid;         // sub-scene of each body (read only when SceneConst::multi)
  uint8_t *flags;   // bit0 fixed; bit (1+w) in contact with wall w
  double4_32a *whist;   // [6 * cap] or null
  double *rdsc;     // 1 / density-scaling factor of each body (1: unscaled)
  // mixed precision mirrors (null in FP64 mode), written by the integrator:
  float4 *p32;      // (x - xref, r) in FP32
  float4 *vw32;     // [2 * cap]: (vx, vy, vz, wx), (wy, wz, 0, 0)
  float4 *xref32;   // xref in FP32 (collider trigger, fluctuation velocity)
  float4 *mprop32;  // (m, I, 1/m, 1/I) in FP32
  float4 *ori32;    // orientation quaternion (mixed mode keeps it in FP32)
};

struct Table {
  int2 *pair;
  int *cpack;
  double4_32a *hfs, *hn;   // FP64 mode; mixed mode uses hfs = (Fs, tan(phi))
  double4_32a *oFM;        // [2 * rows]: (F on body 2, d1), (-(n x F), d2) per row
  double *tanphi;
  // mixed precision rows (null in FP64 mode)
  float4 *g32;      // (reference branch vector xref2 + Href c - xref1, kn); kn == 0: not real
  float *s0;        // (r1 + r2)^2 - |reference branch vector|^2, formed in FP64 at the
                    // collider run and rounded once: the squared gap the FP32 geometry
                    // corrects by the offsets (contact_mixed.cu)
  float4 *hn32;     // (previous normal, ks)
  float4 *oFM32;    // [2 * rows]: (F on body 2, d1), (-(n x F), d2) per row (32 bytes)
  int *row_start;   // [nbody + 1]
  int *down_start;  // [nbody + 1]
  int *down;        // [cap]
  int *ord;         // [nbody]: bodies by decreasing number of incident rows (integration order)
  int *found;       // [cap]
  long long cap;    // rows
  long long nbody_cap;
  long long P;      // rows in use
};

// Cell and clock state of a scene, kept in device memory and advanced by a
// one-thread kernel after every step (so that a batch of steps needs no host
// round trip).  Matrices row-major.
struct CellState {
  double H[9], Hprev[9], L[9], Lprev[9];
  double W[9];      // image velocity matrix Lprev * Hprev (velocity of a cell shift)
  double dL[9];     // L - Lprev (homoDeform first term)
  double Hnext[9];  // (I + L dt) H
  double E[9];      // (Hnext - Href) Href^-1: affine strain since the collider run
  double Ep1[3];    // 1 + the diagonal of E (the displacement bound of a diagonal cell)
  double dtL[3];    // dt times the diagonal of L (homoDeform of a diagonal cell)
  int dl_zero;      // L == Lprev: the homoDeform term reduces to dt L v
  int pad_dl;
  double Href[9], Hrefinv[9];
  double dt, time;
  double dt_law;        // dt of this step's contact laws (the time stepper may change dt
                        // between the contact pass and the integration)
  double verlet, rmax;  // sweep margin dL and largest radius
  double thr2;          // squared displacement bound that triggers the collider
  long long iter;
  int periodic, pad;
  // FP32 diagonals used by the mixed-precision contact kernel for the current step
  float dHf[9];         // H - Href
  float Wf[9];          // image velocity matrix W
  float Ef[9];          // E
  int sheared;          // some off-diagonal entry of H, Hprev, Href, L or Lprev is nonzero
                        // (kernels then take full 3x3 products; diagonal cells keep the
                        // one-term-per-axis fast path, which gives the same values)
  // stress-controlled cell (PeriTriaxController): goal stress (stress_mask bit set)
  // or strain rate per axis, rate bound, growDamping, update period in steps
  double goal[3], max_rate[3], grow_damping;
  int triax, stress_mask, glob_update, pad3;
  // constants of the (sub-)scene: gravity, damping, walls of an aperiodic box
  double gravity[3], damping;
  double box_lo[3], box_hi[3];
  int wall_mask;    // walls present (bit w: wall w = 2 axis + side)
  int wall_mat;     // material of the walls
  int alive;        // 0: a removed sub-scene (its slot is skipped)
  int tstep;        // GlobalStiffnessTimeStepper on
  int tstep_interval;
  int law;          // contact law: 0 Cundall-Strack (linear), 1 Hertz-Mindlin
  double tstep_safety, tstep_default, tstep_max;   // default: dt when no contact exists
  // density scaling: on a stepper update the inertia of each body with contacts is
  // scaled so that its critical step (times the safety) is target_dt, the step used
  int dscale, pad_ds;
  double target_dt;
};

// Peri3dController of a scene without sub-scenes (device resident; the controller
// update runs in the cell advance of sub-scene 0).  Components in the order xx, yy,
// zz, yz, zx, xy; strains engineering (shear = 2 x the tensor entry).
struct P3d {
  int on, mask, first, done;
  long long nsteps, k;
  double goal[6], mod, max_rate, young, poisson, max_strain;
  int npath[6], pad;
  double path[6][16][2];        // (t, v) couples; the last stands for (nsteps, goal)
  double H0inv[9], T0[9];       // cell at the start (inverse) and Cell.trsf then
  double rate[6], err[6], stress[6], strain[6];
  double Lnext[9];              // gradient of the next step, picked up by the cell advance
  int has_next, pad2;
};

constexpr int kServoBlocks = 304;   // fixed partial count of the controller reductions
constexpr int kDegreeBuckets = 64;  // incident-row counts >= 63 share the last bucket

// Small status block read back by the host after a batch of steps.
struct DevStatus {
  int pending;    // collider run needed before the next step (steps are skipped)
  int request;    // set by the integrator when a displacement exceeds the bound
  int error;      // kErr* bits
  int arrive;     // blocks of the current cell-advance launch that have finished
  unsigned long long steps;   // steps completed (never reset)
};

struct Grid {
  int n[3];         // cells per axis
  int B;            // Morton side (power of two >= max n)
  double lo[3];     // aperiodic: origin of the grid
  double scale[3];  // aperiodic: cells per metre; periodic: 1 / L (fraction per metre)
  double L[3];      // periodic cell edges (diagonal H)
  int periodic;
  double reach;     // candidate margin: pair kept when |d| < r1 + r2 + reach
  float Lf[3];      // FP32 copies for the candidate test
  float reachf;
  float slack;      // FP32 rounding allowance of the candidate test (keeps it conservative)
  long long base;   // first global cell index of this grid (sub-scenes are consecutive)
  int morton;       // 1: cells indexed by Morton code (B^3), 0: row-major (n0 n1 n2)
  int sheared;      // periodic cell with off-diagonal terms: fractional coordinates
                    // s = Hinv x and image shifts H c use the full matrices below
  double H[9], Hinv[9];   // periodic cell at this collider run (row-major)
  float Hf[9];
};

struct SceneConst {
  long long N;
  int hertz;     // some sub-scene uses the Hertz-Mindlin law
  int sheared;   // some periodic sub-scene has a sheared cell
  int walls;     // some sub-scene has walls
  int periodic;  // some sub-scene is periodic
  int ordered;   // integrate bodies in Table::ord order (else slot order)
  int multi;     // more than one sub-scene: per-body constants from CellState[sid]
};

// What the step kernels read from device memory instead of their launch
// parameters, so that a captured batch of steps stays valid across collider runs
// (which swap the body buffers and the tables).
struct StepDesc {
  Table t;
  Bodies b;
  SceneConst sc;
  long long cap;   // body capacity (stride of the wall histories)
};

// Comparisons on the integer pipe (every FP64 instruction costs 1/58 of an FP32 one on
// GB300): non-negative doubles are ordered as their bit patterns read as signed 64-bit
// integers, and a double is zero when its bits other than the sign are zero.  Used
// where both sides are non-negative by construction (squared lengths, stiffnesses):
// the decisions are the FP64 comparisons' (a NaN, whose bits exceed every finite
// value's, compares as the FP64 comparison does for the positive NaNs arithmetic
// produces; a non-finite state fails the step in the integrator either way).
__device__ __forceinline__ bool lt_nonneg(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool is_zero_bits(double a) {
  return ((unsigned long long)__double_as_longlong(a) << 1) == 0ull;
}

// ---- cell shift packing: 3 x 10-bit two's complement in one int
__host__ __device__ inline int pack_shift(int c0, int c1, int c2) {
  return (c0 & 1023) | ((c1 & 1023) << 10) | ((c2 & 1023) << 20);
}
__host__ __device__ inline void unpack_shift(int p, int &c0, int &c1, int &c2) {
  c0 = (int)((unsigned)p << 22) >> 22;
  c1 = (int)((unsigned)p << 12) >> 22;
  c2 = (int)((unsigned)p << 2) >> 22;
}
constexpr int kShiftMax = 511;

// ---- launchers (each .cu file owns its kernels)
// scan.cu
size_t scan_workspace_bytes(long long n);
void exclusive_scan(const int *in, int *out, long long n, int *workspace, cudaStream_t st);

// collider.cu
void launch_bbox(const Bodies &b, long long N, double *partials, int nblk, cudaStream_t st);
int bbox_blocks(long long N);
// grids: device array, one per sub-scene (multi) or one; bodies whose grid has no
// cells take the key `dead`
void launch_bin(const Bodies &b, long long N, const Grid *grids, int multi, uint32_t dead,
                uint32_t *key, int *count, cudaStream_t st);
void launch_scatter(long long N, const uint32_t *key, const int *start, int *fill, int *tmp,
                    cudaStream_t st);
void launch_cellsort(const int *count, const int *start, long long ncell, const int *id,
                     int *tmp, cudaStream_t st);
// id_shift (nullable): per sub-scene amount subtracted from the ids (removals)
void launch_reorder(const Bodies &src, const Bodies &dst, long long N, long long cap,
                    const int *new_to_old, int *slot_of_id, int has_walls, int mixed,
                    const int *id_shift, cudaStream_t st);
// per-sub-scene bounding boxes as ordered keys (see collider.cu); keys preset
void launch_bbox_sub(const Bodies &b, long long N, int cap, unsigned long long *keys, int nsm,
                     cudaStream_t st);
void launch_cellrec(const Bodies &b, long long N, const Grid *grids, int multi, float4 *wpos,
                    int4 *info, cudaStream_t st);
// cnt_up / cnt_down: zeroed; counts of the rows of each body as body 1 / body 2 (body 1:
// the smaller id)
// The count pass keeps up to kCandKeep candidates per walker (partner slot and the
// wrap of its neighbour cell, packed in 32 bits) in a scratch list, and their number;
// the emit pass places those without walking the cells again (a walker with more, or
// slots beyond 2^26, walks again).
constexpr int kCandKeep = 32;
struct CandList {
  unsigned *list;   // kCandKeep entries per body: slot | wrap code << 26
  int *n;           // candidates the walker found (may exceed kCandKeep)
  int use;          // 0: slots too large to pack, emit walks
};
void launch_count(float4 *wpos, int4 *info, const int *sid, const int *id, long long N,
                  const Grid *grids, int multi, const int *count, const int *start, int *cnt_up,
                  int *cnt_down, int *err, CandList cl, cudaStream_t st);
// rows in body 1's range sorted by body 2's id, and the down lists filled (unsorted);
// ufill, dfill: zeroed; cl: the count pass's candidates
void launch_emit(float4 *wpos, int4 *info, const Bodies &b, long long N, const Grid *grids,
                 int multi, const int *count, const int *start, const Table &t, int *ufill,
                 int *dfill, CandList cl, cudaStream_t st);
// each down list sorted by body 1's id
void launch_downsort(const Table &t, const int *id, long long N, cudaStream_t st);
// t.ord = bodies in decreasing order of incident rows; ws: 2 * kDegreeBuckets zeroed ints
void launch_degree_order(const Table &t, long long N, int *ws, cudaStream_t st);
void launch_merge(const Table &nt, const Table &ot, long long N_old, const int *new_to_old,
                  int mixed, cudaStream_t st);
// mixed tables: reference branch vectors (g32.xyz) and squared reference gaps (s0) of
// every row, after the emit
void launch_ref_branch(const Table &t, const Bodies &b, const Grid *grids, int multi,
                       cudaStream_t st);
void launch_lost(const Table &ot, const Bodies &ob, const Grid *grids, int multi, int *err,
                 int mixed, cudaStream_t st);
// cell flip: rows of sub-scene `sub` (all rows unless multi) get c' = Minv c (apply = 1),
// or the largest out-of-range |c'| is recorded in *maxabs (apply = 0)
void launch_flip_shift(const Table &t, const int *sid, int multi, int sub, const int Minv[9],
                       int *maxabs, int apply, cudaStream_t st);

// contact.cu
// block: 128 or 256 threads; per_sm: blocks per SM of the persistent grid
// multi: cs is an array indexed by Bodies::sid (else cs[0] holds the one scene)
// rows: upper bound of the table rows (sizes the grid: the table capacity, so that the
// launch shape does not change between collider runs)
// hertz: some sub-scene uses the Hertz-Mindlin law (selects the variant with its branch)
// d / h: the device descriptor and its host copy; desc: read the table and bodies
// through d (captured batches) rather than from launch parameters
// feat: bit 0 some sub-scene uses the Hertz-Mindlin law, bit 1 some cell is sheared
void launch_contact(const StepDesc *d, const StepDesc &h, bool desc, long long rows,
                    const CellState *cs, const DevStatus *ds, const Mat *mats, int multi,
                    int feat, int nsm, int block, int per_sm, cudaStream_t st);
// contact_mixed.cu
void launch_contact_mixed(const StepDesc *d, const StepDesc &h, bool desc, long long rows,
                          const CellState *cs, const DevStatus *ds, const Mat *mats, int multi,
                          int feat, int nsm, int block, int per_sm, cudaStream_t st);

// integrate.cu
// block: 128, 256 or 512 threads
// h.sc.N and h.sc.walls size and select the launch (and must match *d when desc)
void launch_integrate(const StepDesc *d, const StepDesc &h, bool desc, const CellState *cs,
                      DevStatus *ds, const Mat *mats, int mixed, int block, cudaStream_t st);
// one thread per sub-scene (cs[0 .. nsub)); servo partials apply to sub-scene 0
void launch_cell_advance(CellState *cs, int nsub, DevStatus *ds, const double *servo_partials,
                         cudaStream_t st, P3d *p3d = nullptr, const double *p3d_partials = nullptr);
// Peri3dController stress sums of this step's real rows: kServoBlocks x 9 partials of
// sum F_a (-l n_b)
void launch_p3d_partials(const Table &t, const DevStatus *ds, int mixed, double *partials,
                         cudaStream_t st);
// GlobalStiffnessTimeStepper: per-sub-scene minimum critical step (keys: nsub entries
// preset to +inf bits, reset by the launch) applied to the due sub-scenes' dt
void launch_timestepper(const Bodies &b, const Table &t, CellState *cs, int nsub,
                        const DevStatus *ds, const Mat *mats, long long N, long long cap,
                        int mixed, int multi, int walls, unsigned long long *keys,
                        cudaStream_t st);
// servo: per-block sums of sigma_ii * V and K_i * V over the real rows (6 per block)
void launch_servo_partials(const Table &t, const Bodies &b, const DevStatus *ds, int mixed, int law,
                           double *partials, cudaStream_t st);
void launch_gather_forces(const Bodies &b, const Table &t, const Mat *mats, const CellState *cs,
                          const SceneConst &sc, long long cap, double4_32a *F, double4_32a *T,
                          int mixed, cudaStream_t st);
// dst[i] = src[slot_of_id[i]] for i < n (records of consecutive ids, in id order)
// density scaling switched off: factor 1 for the bodies of sub-scene `sub` (all unless multi)
void launch_dscale_reset(const Bodies &b, long long N, int multi, int sub, cudaStream_t st);
void launch_gather_ids(const int *slot_of_id, long long n, const double4_32a *src,
                       double4_32a *dst, cudaStream_t st);
void launch_gather_ids_f(const int *slot_of_id, long long n, const float4 *src, float4 *dst,
                         cudaStream_t st);
// micro.cu: fabric / normal-shear stress partials (28 per block, micro_blocks(P) blocks)
// and per-body stress tensors (9 per slot)
int micro_blocks(long long P);
void launch_micro_rows(const Table &t, int mixed, double *partials, cudaStream_t st);
void launch_body_stress(const Bodies &b, const Table &t, long long N, long long cap, int mixed,
                        int walls, int multi, const CellState *cs, const Mat *mats, double *out,
                        cudaStream_t st);
// stats: per-block partial sums (deterministic tree), summed on the host in block order
int stats_blocks(long long n);
void launch_body_stats(const Bodies &b, const double4_32a *F, long long N, double *partials,
                       cudaStream_t st);
void launch_row_stats(const Table &t, const Bodies &b, double *partials, int mixed,
                      cudaStream_t st);
void launch_wall_stats(const Bodies &b, const SceneConst &sc, const Mat *mats, long long cap,
                       double *partials, cudaStream_t st);

}  // namespace dem
