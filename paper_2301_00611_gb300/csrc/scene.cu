// Host side of the library: scene lifetime, device arenas, the step driver
// and the extern "C" entry points declared in include/dem.h.
//
// Step driver.  A step is: contact kernel (rows) -> integrate kernel (bodies)
// -> one-thread cell/clock advance.  Steps are queued in batches with no host
// round trip: the integrator raises a request when some body has moved more
// than the sweep margin since the last collider run (eq. 2.3-2.4, corrected for
// the affine strain of a deforming cell), the cell advance turns it into
// "pending", and every kernel of a later step returns immediately while
// pending is set.  After each batch the host reads a small status block; if a
// collider run is pending it runs the collider (collider.cu) and continues.
#include <algorithm>
#include <chrono>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dem_internal.cuh"
#include "dem.h"

using namespace dem;

namespace {
thread_local std::string g_create_error;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

double timeout_s() {
  const char *e = std::getenv("DEM_TIMEOUT_S");
  double t = e ? std::atof(e) : 120.0;
  return t > 0 ? t : 120.0;
}

// host twin of the device cell derivations (same operation order as the oracle)
void m_mul(const double *A, const double *B, double *O) {
  double T[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      T[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
  std::memcpy(O, T, sizeof T);
}
double m_det(const double *M) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}
bool m_inv(const double *M, double *O) {
  double d = m_det(M);
  if (d == 0 || !std::isfinite(d)) return false;
  double T[9];
  T[0] = (M[4] * M[8] - M[5] * M[7]) / d;
  T[1] = (M[2] * M[7] - M[1] * M[8]) / d;
  T[2] = (M[1] * M[5] - M[2] * M[4]) / d;
  T[3] = (M[5] * M[6] - M[3] * M[8]) / d;
  T[4] = (M[0] * M[8] - M[2] * M[6]) / d;
  T[5] = (M[2] * M[3] - M[0] * M[5]) / d;
  T[6] = (M[3] * M[7] - M[4] * M[6]) / d;
  T[7] = (M[1] * M[6] - M[0] * M[7]) / d;
  T[8] = (M[0] * M[4] - M[1] * M[3]) / d;
  std::memcpy(O, T, sizeof T);
  return true;
}
bool is_diag(const double *M) {
  return M[1] == 0 && M[2] == 0 && M[3] == 0 && M[5] == 0 && M[6] == 0 && M[7] == 0;
}

// Quantities of the next step that follow from (H, L, Lprev, Hprev, dt, Href).
void cell_derive(CellState &c) {
  if (!c.periodic) {
    for (int q = 0; q < 9; ++q) {
      c.E[q] = 0; c.W[q] = 0; c.dL[q] = 0;
      c.dHf[q] = 0; c.Wf[q] = 0; c.Ef[q] = 0;
    }
    for (int k = 0; k < 3; ++k) { c.Ep1[k] = 1.0; c.dtL[k] = 0.0; }
    c.dl_zero = 1;
    c.sheared = 0;
    c.thr2 = c.verlet * c.verlet;
    return;
  }
  c.sheared = !(is_diag(c.H) && is_diag(c.Hprev) && is_diag(c.Href) && is_diag(c.L) &&
                is_diag(c.Lprev));
  m_mul(c.Lprev, c.Hprev, c.W);
  for (int q = 0; q < 9; ++q) c.dL[q] = c.L[q] - c.Lprev[q];
  double A[9];
  for (int q = 0; q < 9; ++q) A[q] = ((q % 4 == 0) ? 1.0 : 0.0) + c.L[q] * c.dt;
  m_mul(A, c.H, c.Hnext);
  double D[9];
  for (int q = 0; q < 9; ++q) D[q] = c.Hnext[q] - c.Href[q];
  m_mul(D, c.Hrefinv, c.E);
  double e2 = 0;
  for (int q = 0; q < 9; ++q) e2 += c.E[q] * c.E[q];
  double eff = c.verlet - std::sqrt(e2) * (c.rmax + c.verlet);
  c.thr2 = eff > 0 ? eff * eff : -1.0;
  for (int q = 0; q < 9; ++q) {
    c.dHf[q] = (float)(c.H[q] - c.Href[q]);
    c.Wf[q] = (float)c.W[q];
    c.Ef[q] = (float)c.E[q];
  }
  for (int k = 0; k < 3; ++k) {
    c.Ep1[k] = 1.0 + c.E[4 * k];
    c.dtL[k] = c.dt * c.L[4 * k];
  }
  bool dlz = true;
  for (int q = 0; q < 9; ++q) dlz &= c.dL[q] == 0.0;
  c.dl_zero = dlz ? 1 : 0;
}

// Cell state of a new (sub-)scene: periodic cell H (identity otherwise), walls of an
// aperiodic box, wall material, gravity, damping; clock at zero.
void init_cell(CellState &c, int periodic, const double *cell_h, const double *lo,
               const double *hi, int wall_mask, int wall_mat, const double *gravity,
               double damping) {
  std::memset(&c, 0, sizeof c);
  c.periodic = periodic ? 1 : 0;
  for (int q = 0; q < 9; ++q) {
    c.H[q] = periodic ? cell_h[q] : ((q % 4 == 0) ? 1.0 : 0.0);
    c.Hprev[q] = c.H[q];
    c.Href[q] = c.H[q];
  }
  m_inv(c.Href, c.Hrefinv);
  for (int k = 0; k < 3; ++k) {
    c.box_lo[k] = lo[k];
    c.box_hi[k] = hi[k];
    c.gravity[k] = gravity[k];
  }
  c.damping = damping;
  c.wall_mask = periodic ? 0 : (wall_mask & 0x3F);
  c.wall_mat = wall_mat;
  c.alive = 1;
}

unsigned next_pow2(unsigned v) {
  unsigned p = 1;
  while (p < v) p <<= 1;
  return p;
}
}  // namespace

// automatic step graphs below this many bodies (launch overhead matters there; larger
// scenes keep the leaner parameter-fed kernels)
constexpr long long kGraphAutoBodies = 1 << 18;

struct Readback {
  DevStatus ds;
  int totals[4];
};

// What a captured batch of steps depends on besides its step count.
struct GraphKey {
  long long N = -1, rows = -1;
  int contact_block = 0, contact_per_sm = 0, integrate_block = 0, multi = 0, walls = 0, nsub = 0,
      mixed = 0;
  const void *cs = nullptr;
  bool operator==(const GraphKey &o) const {
    return N == o.N && rows == o.rows && contact_block == o.contact_block &&
           contact_per_sm == o.contact_per_sm && integrate_block == o.integrate_block &&
           multi == o.multi && walls == o.walls && nsub == o.nsub && mixed == o.mixed && cs == o.cs;
  }
};

// A sub-scene: an independent scene sharing the library's arrays with the others
// (its own cell or box, walls, gravity, damping, time step and clock; its bodies
// carry its index in Bodies::sid).  Sub-scene 0 is the scene of the descriptor.
struct Sub {
  bool used = false;
  CellState cs{};                 // host copy (refreshed after every batch of steps)
  long long n = 0, id0 = 0;       // bodies and first id (ids of a sub-scene are consecutive)
  double rmin = INFINITY, rmax = 0, vsolid = 0;
  double verlet_rule = -0.5;      // > 0 absolute sweep margin, < 0 fraction of r_min
  bool dt_set = false;
  Grid grid{};                    // grid of the last collider run
  long long slot0 = 0;            // first slot (valid after a collider run)
  bool removing = false;          // removed; its bodies go at the next collider run
  bool velgrad_pending = false;   // velocity gradient for the next step (Cell.velGrad)
  double velgrad_next[9]{};
  double tstep_default_rule = -1; // time stepper's defaultDt as set (< 0: from the p-wave step)
  long long tstep_default_n = -1; // body count the derived default was computed for
};

struct dem_scene {
  dem_scene_desc desc{};
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int nsm = 152;
  std::string err;

  Mat mats_h[kMaxMat]{};
  bool mat_set[kMaxMat]{};
  Mat *mats_d = nullptr;

  long long N = 0, cap = 0;
  std::vector<double> radius_h;  // by id
  std::vector<int> mat_h;        // by id
  std::vector<unsigned char> fixed_h;

  Bodies cur{}, alt{};
  int *slot_of_id = nullptr, *new_to_old = nullptr, *cnt_up = nullptr, *cnt_down = nullptr;
  uint32_t *key = nullptr;
  double4_32a *gF = nullptr, *gT = nullptr;
  float4 *wpos = nullptr;
  int4 *cinfo = nullptr;
  unsigned *cand_list = nullptr;   // the count pass's candidates (kCandKeep per body)
  int *cand_n = nullptr;

  Table tab[2]{};
  long long tab_nbody[2]{0, 0};
  int tc = 0;

  int *cell_count = nullptr, *cell_start = nullptr, *cell_fill = nullptr;
  long long cell_cap = 0;
  int *scan_ws = nullptr;
  size_t scan_ws_bytes = 0;
  double *partials = nullptr;  // 1024 blocks x 32 doubles
  double *servo = nullptr;     // kServoBlocks x 6 doubles
  // Peri3dController (scene without sub-scenes): device state, stress partials, host copy
  P3d *p3d_d = nullptr;
  double *p3d_part = nullptr;   // kServoBlocks x 9 doubles
  P3d p3d_h{};
  bool p3d_on = false;
  int *deg_ws = nullptr;       // 2 x kDegreeBuckets ints (integration order)
  // launch shapes of the step kernels (none changes a result)
  int contact_block = 256, contact_per_sm = 8, integrate_block = 256, degree_order = 1;
  int step_graphs = -1;          // replay captured batches: 1 yes, 0 no, -1 small scenes
  StepDesc *step_d = nullptr;    // device step descriptor
  StepDesc *step_h = nullptr;    // pinned staging copy
  GraphKey graph_key{};
  std::map<long long, cudaGraphExec_t> graphs;   // captured batches by step count
  double *partials_h = nullptr;

  std::vector<Sub> subs;         // sub-scene 0 always exists
  CellState *cs_d = nullptr;     // [subs_cap]
  CellState *cs_rb = nullptr;    // pinned [subs_cap]: read back after each batch
  Grid *grids_d = nullptr;       // [subs_cap]
  int *id_shift_d = nullptr;     // [subs_cap]: id renumbering at a collider run
  Grid *grids_h = nullptr;       // pinned [subs_cap]
  int *shift_h = nullptr;        // pinned [subs_cap]
  unsigned long long *bbox_keys = nullptr;   // [6 * subs_cap]
  unsigned long long *dt_keys = nullptr;     // [subs_cap] time-stepper minima (+inf bits)
  unsigned long long *bbox_h = nullptr;      // pinned [6 * subs_cap]
  int subs_cap = 0;
  unsigned long long steps_seen = 0;   // DevStatus::steps at the last read
  CellState &cs0() { return subs[0].cs; }
  int nsub() const { return (int)subs.size(); }
  DevStatus *ds_d = nullptr;
  Readback *rb_h = nullptr;  // pinned
  cudaEvent_t ev = nullptr;

  bool need_rebuild = true;
  bool table_fresh = false;   // table rows hold the contacts of the last completed step
  bool check_lost = false;
  bool cs_dirty = true;
  bool layout_dirty = true;      // bodies added or removed since the last collider run
  bool has_walls = false;        // some sub-scene has walls
  bool mixed = false;
  long long n_rebuilds = 0;
  bool broken = false;
  long long batch = 16;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> tev;   // event pool: 6 per step of a batch + 2 for the collider
  dem_timing tm{};
  long long launches = 0;
  // device memory held (stream-ordered allocations of dalloc, by pointer)
  std::unordered_map<void *, size_t> alloc_bytes;
  long long dev_bytes = 0;
};

namespace {

dem_status fail(dem_scene *s, dem_status code, const std::string &msg) {
  if (s) s->err = msg;
  return code;
}

dem_status cuda_fail(dem_scene *s, cudaError_t e, const char *what) {
  if (s) s->broken = true;
  return fail(s, DEM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                       \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return cuda_fail(s, e_, #call);             \
  } while (0)

template <class T>
dem_status dalloc(dem_scene *s, T **p, long long count) {
  *p = nullptr;
  if (count <= 0) return DEM_OK;
  cudaError_t e = cudaMallocAsync((void **)p, sizeof(T) * (size_t)count, s->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(s, DEM_ERR_OOM, std::string("device allocation failed: ") + cudaGetErrorString(e));
  }
  s->alloc_bytes[(void *)*p] = sizeof(T) * (size_t)count;
  s->dev_bytes += (long long)(sizeof(T) * (size_t)count);
  return DEM_OK;
}

template <class T>
void dfree(dem_scene *s, T *&p) {
  if (p) {
    auto it = s->alloc_bytes.find((void *)p);
    if (it != s->alloc_bytes.end()) {
      s->dev_bytes -= (long long)it->second;
      s->alloc_bytes.erase(it);
    }
    cudaFreeAsync(p, s->st);
  }
  p = nullptr;
}

dem_status wait(dem_scene *s) {
  CK(cudaEventRecord(s->ev, s->st));
  const double deadline = now_s() + timeout_s();
  int spins = 0;
  while (true) {
    cudaError_t e = cudaEventQuery(s->ev);
    if (e == cudaSuccess) return DEM_OK;
    if (e != cudaErrorNotReady) return cuda_fail(s, e, "stream wait");
    if (now_s() > deadline) {
      s->broken = true;
      return fail(s, DEM_ERR_TIMEOUT, "timed out waiting for the GPU");
    }
    if (++spins > 2000) std::this_thread::sleep_for(std::chrono::microseconds(50));
    else std::this_thread::yield();
  }
}

void drop_graphs(dem_scene *s) {
  for (auto &kv : s->graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
}

void free_bodies(dem_scene *s, Bodies &b) {
  dfree(s, b.pos); dfree(s, b.vel); dfree(s, b.angvel); dfree(s, b.ori); dfree(s, b.xref);
  dfree(s, b.mprop); dfree(s, b.id); dfree(s, b.sid); dfree(s, b.mat); dfree(s, b.flags);
  dfree(s, b.whist); dfree(s, b.rdsc);
  dfree(s, b.p32); dfree(s, b.vw32); dfree(s, b.xref32); dfree(s, b.mprop32); dfree(s, b.ori32);
}

dem_status alloc_bodies(dem_scene *s, Bodies &b, long long cap) {
  dem_status r;
  if ((r = dalloc(s, &b.pos, cap)) || (r = dalloc(s, &b.vel, cap)) ||
      (r = dalloc(s, &b.angvel, cap)) || (r = dalloc(s, &b.ori, cap)) ||
      (r = dalloc(s, &b.xref, cap)) || (r = dalloc(s, &b.mprop, cap)) ||
      (r = dalloc(s, &b.id, cap)) || (r = dalloc(s, &b.sid, cap)) ||
      (r = dalloc(s, &b.mat, cap)) || (r = dalloc(s, &b.flags, cap)) ||
      (r = dalloc(s, &b.rdsc, cap)))
    return r;
  // wall histories exist for every body (a sub-scene with walls may join later)
  if ((r = dalloc(s, &b.whist, 6 * cap))) return r;
  if (s->mixed && ((r = dalloc(s, &b.p32, cap)) || (r = dalloc(s, &b.vw32, 2 * cap)) ||
                   (r = dalloc(s, &b.xref32, cap)) || (r = dalloc(s, &b.mprop32, cap)) ||
                   (r = dalloc(s, &b.ori32, cap))))
    return r;
  return DEM_OK;
}

void free_rows(dem_scene *s, Table &t) {
  dfree(s, t.pair); dfree(s, t.cpack); dfree(s, t.hfs); dfree(s, t.hn); dfree(s, t.oFM);
  dfree(s, t.tanphi); dfree(s, t.down); dfree(s, t.found);
  dfree(s, t.g32); dfree(s, t.hn32); dfree(s, t.oFM32); dfree(s, t.s0);
}

void free_table(dem_scene *s, Table &t) {
  free_rows(s, t);
  dfree(s, t.row_start); dfree(s, t.down_start); dfree(s, t.ord);
  t.cap = 0; t.nbody_cap = 0; t.P = 0;
}

// capacity for `rows` rows and `nbody` bodies; keeps nothing (callers rebuild)
dem_status ensure_table(dem_scene *s, Table &t, long long rows, long long nbody) {
  dem_status r;
  if (rows > t.cap) {
    long long P = t.P;
    long long nc = std::max<long long>(rows + rows / 4, 1024);
    free_rows(s, t);
    if ((r = dalloc(s, &t.pair, nc)) || (r = dalloc(s, &t.cpack, nc)) ||
        (r = dalloc(s, &t.hfs, nc)) || (r = dalloc(s, &t.down, nc)) ||
        (r = dalloc(s, &t.found, nc)))
      return r;
    if (s->mixed) {
      if ((r = dalloc(s, &t.g32, nc)) || (r = dalloc(s, &t.hn32, nc)) || (r = dalloc(s, &t.s0, nc)) ||
          (r = dalloc(s, &t.oFM32, 2 * nc)))
        return r;
    } else if ((r = dalloc(s, &t.hn, nc)) || (r = dalloc(s, &t.oFM, 2 * nc)) ||
               (r = dalloc(s, &t.tanphi, nc))) {
      return r;
    }
    t.cap = nc;
    t.P = std::min(P, nc);
  }
  if (nbody + 1 > t.nbody_cap) {
    long long nb = std::max<long long>(nbody + 1, 64);
    dfree(s, t.row_start); dfree(s, t.down_start); dfree(s, t.ord);
    if ((r = dalloc(s, &t.row_start, nb)) || (r = dalloc(s, &t.down_start, nb)) ||
        (r = dalloc(s, &t.ord, nb)))
      return r;
    t.nbody_cap = nb;
  }
  return DEM_OK;
}

// capacity of the per-sub-scene arrays (device cell states, grids, staging)
dem_status ensure_subs(dem_scene *s, int need) {
  if (need <= s->subs_cap) return DEM_OK;
  const int nc = std::max(need, std::max(8, 2 * s->subs_cap));
  CellState *cs = nullptr;
  dem_status r;
  if ((r = dalloc(s, &cs, nc))) return r;
  if (s->cs_d && s->subs_cap > 0)
    CK(cudaMemcpyAsync(cs, s->cs_d, sizeof(CellState) * s->subs_cap, cudaMemcpyDeviceToDevice, s->st));
  if ((r = wait(s))) return r;
  dfree(s, s->cs_d);
  s->cs_d = cs;
  dfree(s, s->grids_d); dfree(s, s->id_shift_d); dfree(s, s->bbox_keys); dfree(s, s->dt_keys);
  if ((r = dalloc(s, &s->grids_d, nc)) || (r = dalloc(s, &s->id_shift_d, nc)) ||
      (r = dalloc(s, &s->bbox_keys, 6LL * nc)) || (r = dalloc(s, &s->dt_keys, nc)))
    return r;
  {
    std::vector<unsigned long long> inf(nc, 0x7ff0000000000000ull);
    CK(cudaMemcpyAsync(s->dt_keys, inf.data(), sizeof(unsigned long long) * nc,
                       cudaMemcpyHostToDevice, s->st));
    if ((r = wait(s))) return r;
  }
  if (s->cs_rb) cudaFreeHost(s->cs_rb);
  if (s->grids_h) cudaFreeHost(s->grids_h);
  if (s->shift_h) cudaFreeHost(s->shift_h);
  if (s->bbox_h) cudaFreeHost(s->bbox_h);
  s->cs_rb = nullptr; s->grids_h = nullptr; s->shift_h = nullptr; s->bbox_h = nullptr;
  CK(cudaMallocHost((void **)&s->cs_rb, sizeof(CellState) * nc));
  CK(cudaMallocHost((void **)&s->grids_h, sizeof(Grid) * nc));
  CK(cudaMallocHost((void **)&s->shift_h, sizeof(int) * nc));
  CK(cudaMallocHost((void **)&s->bbox_h, sizeof(unsigned long long) * 6 * nc));
  s->subs_cap = nc;
  return DEM_OK;
}

dem_status ensure_bodies(dem_scene *s, long long need) {
  if (need <= s->cap) return DEM_OK;
  long long nc = std::max<long long>(need, std::max<long long>(s->cap * 2, 1024));
  Bodies nb{}, na{};
  dem_status r;
  if ((r = alloc_bodies(s, nb, nc)) || (r = alloc_bodies(s, na, nc))) return r;
  const long long N = s->N;
  if (N > 0) {
    size_t d4 = sizeof(double4_32a) * N;
    CK(cudaMemcpyAsync(nb.pos, s->cur.pos, d4, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.vel, s->cur.vel, d4, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.angvel, s->cur.angvel, d4, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.ori, s->cur.ori, d4, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.xref, s->cur.xref, d4, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.mprop, s->cur.mprop, d4, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.id, s->cur.id, sizeof(int) * N, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.sid, s->cur.sid, sizeof(int) * N, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.mat, s->cur.mat, sizeof(int) * N, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.flags, s->cur.flags, N, cudaMemcpyDeviceToDevice, s->st));
    CK(cudaMemcpyAsync(nb.rdsc, s->cur.rdsc, sizeof(double) * N, cudaMemcpyDeviceToDevice, s->st));
    if (s->has_walls)
      for (int w = 0; w < 6; ++w)
        CK(cudaMemcpyAsync(nb.whist + w * nc, s->cur.whist + w * s->cap, d4,
                           cudaMemcpyDeviceToDevice, s->st));
    if (s->mixed) {
      const size_t f4 = sizeof(float4) * N;
      CK(cudaMemcpyAsync(nb.p32, s->cur.p32, f4, cudaMemcpyDeviceToDevice, s->st));
      CK(cudaMemcpyAsync(nb.vw32, s->cur.vw32, 2 * f4, cudaMemcpyDeviceToDevice, s->st));
      CK(cudaMemcpyAsync(nb.xref32, s->cur.xref32, f4, cudaMemcpyDeviceToDevice, s->st));
      CK(cudaMemcpyAsync(nb.mprop32, s->cur.mprop32, f4, cudaMemcpyDeviceToDevice, s->st));
      CK(cudaMemcpyAsync(nb.ori32, s->cur.ori32, f4, cudaMemcpyDeviceToDevice, s->st));
    }
  }
  free_bodies(s, s->cur);
  free_bodies(s, s->alt);
  s->cur = nb;
  s->alt = na;
  int *sid = nullptr;
  if ((r = dalloc(s, &sid, nc))) return r;
  if (N > 0) CK(cudaMemcpyAsync(sid, s->slot_of_id, sizeof(int) * N, cudaMemcpyDeviceToDevice, s->st));
  dfree(s, s->slot_of_id);
  s->slot_of_id = sid;
  dfree(s, s->new_to_old); dfree(s, s->cnt_up); dfree(s, s->cnt_down); dfree(s, s->key);
  dfree(s, s->gF); dfree(s, s->gT); dfree(s, s->wpos); dfree(s, s->cinfo);
  dfree(s, s->cand_list); dfree(s, s->cand_n);
  if ((r = dalloc(s, &s->new_to_old, nc)) || (r = dalloc(s, &s->cnt_up, nc)) ||
      (r = dalloc(s, &s->cnt_down, nc)) || (r = dalloc(s, &s->key, nc)) ||
      (r = dalloc(s, &s->gF, nc)) || (r = dalloc(s, &s->gT, nc)) ||
      (r = dalloc(s, &s->wpos, nc)) || (r = dalloc(s, &s->cinfo, nc)) ||
      (r = dalloc(s, &s->cand_list, nc * kCandKeep)) || (r = dalloc(s, &s->cand_n, nc)))
    return r;
  s->cap = nc;
  size_t ws = scan_workspace_bytes(nc + 1);
  if (ws > s->scan_ws_bytes) {
    dfree(s, s->scan_ws);
    if ((r = dalloc(s, &s->scan_ws, (long long)(ws / sizeof(int) + 1)))) return r;
    s->scan_ws_bytes = ws;
  }
  return DEM_OK;
}

SceneConst scene_const(const dem_scene *s) {
  SceneConst c{};
  c.N = s->N;
  c.walls = 0;
  c.periodic = 0;
  for (const Sub &u : s->subs)
    if (u.used) {
      c.walls |= u.cs.wall_mask ? 1 : 0;
      c.periodic |= u.cs.periodic;
      c.hertz |= u.cs.law;
      c.sheared |= u.cs.sheared;
    }
  c.ordered = s->degree_order;
  c.multi = s->nsub() > 1;
  return c;
}

// 0.5 * utils.PWaveTimeStep: min over the sub-scene's spheres of SpherePWaveTimeStep
// = r / sqrt(E / rho)
double default_dt(const dem_scene *s, const Sub &u) {
  double dt = INFINITY;
  for (long long i = u.id0; i < u.id0 + u.n; ++i) {
    const Mat &m = s->mats_h[s->mat_h[i]];
    double d = s->radius_h[i] / std::sqrt(m.young / m.density);
    if (d < dt) dt = d;
  }
  return 0.5 * dt;
}

// every used sub-scene with bodies needs a time step; sub-scene 0 without bodies
// and without an explicit dt is an error only when nothing else can step
dem_status ensure_dt(dem_scene *s) {
  for (Sub &u : s->subs) {
    if (!u.used || u.n == 0) continue;
    if (!u.dt_set) {
      u.cs.dt = default_dt(s, u);
      u.dt_set = true;
      s->cs_dirty = true;
    }
    // time stepper without contacts: safety x p-wave step of the current spheres
    if (u.cs.tstep && u.tstep_default_rule <= 0 && u.tstep_default_n != u.n) {
      u.cs.tstep_default = u.cs.tstep_safety * 2.0 * default_dt(s, u);
      u.tstep_default_n = u.n;
      s->cs_dirty = true;
    }
  }
  if (s->N == 0) return fail(s, DEM_ERR_STATE, "no time step: the scene has no bodies");
  return DEM_OK;
}

dem_status upload_cell(dem_scene *s) {
  for (Sub &u : s->subs) {
    cell_derive(u.cs);
    u.cs.dt_law = u.cs.dt;
  }
  for (int q = 0; q < s->nsub(); ++q) s->cs_rb[q] = s->subs[q].cs;
  CK(cudaMemcpyAsync(s->cs_d, s->cs_rb, sizeof(CellState) * s->nsub(), cudaMemcpyHostToDevice,
                     s->st));
  s->cs_dirty = false;
  return wait(s);   // the pinned staging buffer is read again after each batch
}

dem_status status_error(dem_scene *s, int e) {
  if (e & kErrNonFinite) return fail(s, DEM_ERR_NONFINITE, "a body state became NaN or Inf");
  if (e & kErrShiftRange)
    return fail(s, DEM_ERR_CAPACITY, "a periodic cell shift exceeds +-511 cells");
  if (e & kErrHistoryLost)
    return fail(s, DEM_ERR_STATE,
                "a real contact was missing from the collider candidates (sweep margin violated)");
  return fail(s, DEM_ERR_STATE, "device error");
}

// ------------------------------------------------------------------ collider
dem_status rebuild_core(dem_scene *s);

// kernels the collider launches (bin, scan x2-3, scatter, cellsort, reorder, count,
// scans, emit, down sort, degree order x3, merge, lost): counted approximately from
// its phases
dem_status rebuild(dem_scene *s) {
  if (s->timing) CK(cudaEventRecord(s->tev[0], s->st));
  dem_status r = rebuild_core(s);
  if (r) return r;
  s->launches += 17 + (s->mixed ? 1 : 0);
  if (s->timing) {
    CK(cudaEventRecord(s->tev[1], s->st));
    CK(cudaEventSynchronize(s->tev[1]));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, s->tev[0], s->tev[1]));
    s->tm.collider_ms += ms;
    s->tm.collider_runs += 1;
  }
  return DEM_OK;
}

double key_value(unsigned long long k) {   // inverse of the device's ord_key
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
}

// Grid of one sub-scene: cell edge >= 2 r_max + 2 dL; periodic: the cell divided
// into n >= 3 cells per axis; aperiodic: the bounding box [lo, hi] of its spheres.
dem_status sub_grid(dem_scene *s, Sub &u, const double lo[3], const double hi[3], bool morton,
                    Grid &g) {
  const double verlet = u.cs.verlet;
  const double reach = 2 * verlet;
  const double hmin = 2 * u.rmax + reach;
  g = Grid{};
  g.periodic = u.cs.periodic;
  g.reach = reach;
  if (g.periodic) {
    const double *H = u.cs.H;
    g.sheared = !is_diag(H);
    // perpendicular width of the cell across each pair of faces: |det H| / |a_i x a_j|,
    // a_k the cell vectors (columns of H); cells are slabs of fractional coordinates
    double w[3];
    const double V = std::fabs(m_det(H));
    for (int k = 0; k < 3; ++k) {
      const int i = (k + 1) % 3, j = (k + 2) % 3;
      const double a[3] = {H[i], H[3 + i], H[6 + i]}, b[3] = {H[j], H[3 + j], H[6 + j]};
      const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2],
                   cz = a[0] * b[1] - a[1] * b[0];
      w[k] = g.sheared ? V / std::sqrt(cx * cx + cy * cy + cz * cz) : H[4 * k];
    }
    if (!m_inv(H, g.Hinv)) return fail(s, DEM_ERR_INVALID_ARG, "singular periodic cell");
    for (int q = 0; q < 9; ++q) {
      g.H[q] = H[q];
      g.Hf[q] = (float)H[q];
    }
    for (int k = 0; k < 3; ++k) {
      double L = H[4 * k];
      int n = (int)std::floor(w[k] / hmin);
      if (n < 3)
        return fail(s, DEM_ERR_GEOMETRY,
                    "periodic cell width shorter than 3 * (2 r_max + 2 verlet_dist): a sphere "
                    "spans too large a part of the cell");
      g.n[k] = std::min(n, kMaxGridSide);
      g.L[k] = L;
      g.scale[k] = 1.0 / L;
      g.lo[k] = 0;
    }
  } else {
    for (int k = 0; k < 3; ++k) {
      if (!std::isfinite(lo[k]) || !std::isfinite(hi[k]))
        return fail(s, DEM_ERR_NONFINITE, "non-finite body position");
      double ext = std::max(hi[k] - lo[k], hmin);
      int n = (int)std::floor(ext / hmin);
      n = std::max(1, std::min(n, kMaxGridSide));
      g.n[k] = n;
      g.lo[k] = lo[k];
      g.scale[k] = n / ext;
      g.L[k] = 0;
    }
  }
  double ext = 0;
  for (int k = 0; k < 3; ++k) {
    double e = g.periodic ? std::fabs(g.H[3 * k]) + std::fabs(g.H[3 * k + 1]) + std::fabs(g.H[3 * k + 2])
                          : g.n[k] / g.scale[k];
    ext = std::max(ext, e);
    g.Lf[k] = (float)g.L[k];
  }
  g.reachf = (float)reach;
  // FP32 coordinates are bounded by ext: a few ulps of ext plus a relative allowance
  g.slack = (float)(8.0 * ext * std::ldexp(1.0, -23) + 1e-5 * hmin);
  g.B = (int)next_pow2((unsigned)std::max(g.n[0], std::max(g.n[1], g.n[2])));
  g.morton = morton ? 1 : 0;
  return DEM_OK;
}

dem_status rebuild_core(dem_scene *s) {
  const long long N = s->N;   // slots in use: live bodies and those of removed sub-scenes
  const int nsub = s->nsub();
  const bool multi = nsub > 1;
  dem_status r;
  // 0. bounding boxes of the aperiodic sub-scenes
  std::vector<double> lo(3 * nsub, INFINITY), hi(3 * nsub, -INFINITY);
  bool need_box = false;
  for (const Sub &u : s->subs) need_box |= u.used && !u.removing && u.n > 0 && !u.cs.periodic;
  if (need_box && !multi) {
    int nblk = bbox_blocks(N);
    launch_bbox(s->cur, N, s->partials, nblk, s->st);
    CK(cudaMemcpyAsync(s->partials_h, s->partials, sizeof(double) * 6 * nblk,
                       cudaMemcpyDeviceToHost, s->st));
    if ((r = wait(s))) return r;
    for (int b = 0; b < nblk; ++b)
      for (int k = 0; k < 3; ++k) {
        lo[k] = std::min(lo[k], s->partials_h[6 * b + k]);
        hi[k] = std::max(hi[k], s->partials_h[6 * b + 3 + k]);
      }
  } else if (need_box) {
    const long long cap = s->subs_cap;
    CK(cudaMemsetAsync(s->bbox_keys, 0xff, sizeof(unsigned long long) * 3 * cap, s->st));
    CK(cudaMemsetAsync(s->bbox_keys + 3 * cap, 0, sizeof(unsigned long long) * 3 * cap, s->st));
    launch_bbox_sub(s->cur, N, (int)cap, s->bbox_keys, s->nsm, s->st);
    CK(cudaMemcpyAsync(s->bbox_h, s->bbox_keys, sizeof(unsigned long long) * 6 * cap,
                       cudaMemcpyDeviceToHost, s->st));
    if ((r = wait(s))) return r;
    for (int q = 0; q < nsub; ++q)
      for (int k = 0; k < 3; ++k) {
        lo[3 * q + k] = key_value(s->bbox_h[k * cap + q]);
        hi[3 * q + k] = key_value(s->bbox_h[(3 + k) * cap + q]);
      }
  }
  // 1. grids, one block of cells per live sub-scene (Morton order for a single scene,
  //    row-major for sub-scenes), consecutive in sub-scene order; bodies of removed
  //    sub-scenes take the sentinel cell after the last one
  long long total = 0, n_live = 0;
  bool removal = false;
  for (int q = 0; q < nsub; ++q) {
    Sub &u = s->subs[q];
    Grid &g = u.grid;
    removal |= u.removing;
    if (!u.used || u.removing || u.n == 0) {
      g = Grid{};
      g.base = total;
      continue;
    }
    if ((r = sub_grid(s, u, &lo[3 * q], &hi[3 * q], !multi, g))) return r;
    g.base = total;
    total += multi ? (long long)g.n[0] * g.n[1] * g.n[2] : (long long)g.B * g.B * g.B;
    u.slot0 = n_live;
    n_live += u.n;
  }
  if (total + 1 > 0x7fffffffLL) return fail(s, DEM_ERR_CAPACITY, "collider grid exceeds 2^31 cells");
  const uint32_t dead = (uint32_t)total;
  const long long ncell = total + 1;
  for (int q = 0; q < nsub; ++q) s->grids_h[q] = s->subs[q].grid;
  CK(cudaMemcpyAsync(s->grids_d, s->grids_h, sizeof(Grid) * nsub, cudaMemcpyHostToDevice, s->st));
  if (ncell > s->cell_cap) {
    dfree(s, s->cell_count); dfree(s, s->cell_start); dfree(s, s->cell_fill);
    if ((r = dalloc(s, &s->cell_count, ncell)) || (r = dalloc(s, &s->cell_start, ncell + 1)) ||
        (r = dalloc(s, &s->cell_fill, ncell)))
      return r;
    s->cell_cap = ncell;
    size_t ws = scan_workspace_bytes(ncell + 1);
    if (ws > s->scan_ws_bytes) {
      dfree(s, s->scan_ws);
      if ((r = dalloc(s, &s->scan_ws, (long long)(ws / sizeof(int) + 1)))) return r;
      s->scan_ws_bytes = ws;
    }
  }
  CK(cudaMemsetAsync(s->cell_count, 0, sizeof(int) * ncell, s->st));
  CK(cudaMemsetAsync(s->cell_fill, 0, sizeof(int) * ncell, s->st));
  CK(cudaMemsetAsync(&s->ds_d->error, 0, sizeof(int), s->st));
  // ids close up over removed sub-scenes: each live sub-scene's ids move down by the
  // bodies of removed sub-scenes with smaller ids
  const int *id_shift = nullptr;
  if (removal) {
    for (int q = 0; q < nsub; ++q) {
      long long sh = 0;
      for (const Sub &v : s->subs)
        if (v.removing && v.id0 < s->subs[q].id0) sh += v.n;
      s->shift_h[q] = (int)sh;
    }
    CK(cudaMemcpyAsync(s->id_shift_d, s->shift_h, sizeof(int) * nsub, cudaMemcpyHostToDevice,
                       s->st));
    id_shift = s->id_shift_d;
  }
  // 2-3: bin, counting sort (cell order, then id within a cell), permute the bodies
  launch_bin(s->cur, N, s->grids_d, multi, dead, s->key, s->cell_count, s->st);
  exclusive_scan(s->cell_count, s->cell_start, ncell, s->scan_ws, s->st);
  launch_scatter(N, s->key, s->cell_start, s->cell_fill, s->new_to_old, s->st);
  // the sentinel cell of removed bodies is left unsorted: its order is never used (and
  // it can hold every body of a large removed sub-scene)
  launch_cellsort(s->cell_count, s->cell_start, total, s->cur.id, s->new_to_old, s->st);
  launch_reorder(s->cur, s->alt, n_live, s->cap, s->new_to_old, s->slot_of_id, s->has_walls,
                 s->mixed, id_shift, s->st);
  std::swap(s->cur, s->alt);
  const long long N_old = N;
  s->N = n_live;
  const long long NL = n_live;
  // 4: candidates (count, prefix sums, emit)
  Table &ot = s->tab[s->tc];
  Table &nt = s->tab[1 - s->tc];
  if ((r = ensure_table(s, nt, 0, NL))) return r;
  launch_cellrec(s->cur, NL, s->grids_d, multi, s->wpos, s->cinfo, s->st);
  CK(cudaMemsetAsync(s->cnt_up, 0, sizeof(int) * std::max<long long>(NL, 1), s->st));
  CK(cudaMemsetAsync(s->cnt_down, 0, sizeof(int) * std::max<long long>(NL, 1), s->st));
  // slots are packed in 26 bits of a candidate entry
  const CandList cl{s->cand_list, s->cand_n, s->cap < (1LL << 26) ? 1 : 0};
  launch_count(s->wpos, s->cinfo, s->cur.sid, s->cur.id, NL, s->grids_d, multi, s->cell_count,
               s->cell_start, s->cnt_up, s->cnt_down, &s->ds_d->error, cl, s->st);
  exclusive_scan(s->cnt_up, nt.row_start, NL, s->scan_ws, s->st);
  exclusive_scan(s->cnt_down, nt.down_start, NL, s->scan_ws, s->st);
  CK(cudaMemcpyAsync(&s->rb_h->totals[0], nt.row_start + NL, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(&s->rb_h->totals[1], nt.down_start + NL, sizeof(int), cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(&s->rb_h->ds, s->ds_d, sizeof(DevStatus), cudaMemcpyDeviceToHost, s->st));
  if ((r = wait(s))) return r;
  if (s->rb_h->ds.error) return status_error(s, s->rb_h->ds.error);
  const long long P = s->rb_h->totals[0];
  if (P != s->rb_h->totals[1]) return fail(s, DEM_ERR_STATE, "internal: candidate count mismatch");
  if ((r = ensure_table(s, nt, P, NL))) return r;
  nt.P = P;
  // fill counters: the bin keys and the up counts (scanned already) are no longer needed
  int *dfill = reinterpret_cast<int *>(s->key);
  int *ufill = s->cnt_up;
  CK(cudaMemsetAsync(dfill, 0, sizeof(int) * std::max<long long>(NL, 1), s->st));
  CK(cudaMemsetAsync(ufill, 0, sizeof(int) * std::max<long long>(NL, 1), s->st));
  launch_emit(s->wpos, s->cinfo, s->cur, NL, s->grids_d, multi, s->cell_count, s->cell_start, nt,
              ufill, dfill, cl, s->st);
  if (s->mixed) launch_ref_branch(nt, s->cur, s->grids_d, multi, s->st);
  launch_downsort(nt, s->cur.id, NL, s->st);
  CK(cudaMemsetAsync(s->deg_ws, 0, sizeof(int) * 2 * kDegreeBuckets, s->st));
  launch_degree_order(nt, NL, s->deg_ws, s->st);
  // 5: carry the contact history of the previous table
  ot.P = std::min(ot.P, ot.cap);
  if (ot.P > 0) CK(cudaMemsetAsync(ot.found, 0, sizeof(int) * ot.P, s->st));
  Table otv = ot;
  if (ot.P == 0 || ot.row_start == nullptr) otv.P = 0;
  launch_merge(nt, otv, s->tab_nbody[s->tc], s->new_to_old, s->mixed, s->st);
  // a removed sub-scene's contacts vanish by design: no history check on that run
  if (s->check_lost && !removal)
    launch_lost(otv, s->alt, s->grids_d, multi, &s->ds_d->error, s->mixed, s->st);
  (void)N_old;
  s->tab_nbody[1 - s->tc] = NL;
  s->tc = 1 - s->tc;
  // host bookkeeping of removals: ids and per-id host arrays close up
  if (removal) {
    std::vector<const Sub *> gone;   // erase id ranges from the highest down
    for (const Sub &u : s->subs)
      if (u.removing) gone.push_back(&u);
    std::sort(gone.begin(), gone.end(), [](const Sub *a, const Sub *b) { return a->id0 > b->id0; });
    for (const Sub *u : gone) {
      s->radius_h.erase(s->radius_h.begin() + u->id0, s->radius_h.begin() + u->id0 + u->n);
      s->mat_h.erase(s->mat_h.begin() + u->id0, s->mat_h.begin() + u->id0 + u->n);
      s->fixed_h.erase(s->fixed_h.begin() + u->id0, s->fixed_h.begin() + u->id0 + u->n);
    }
    for (int q = 0; q < nsub; ++q) s->subs[q].id0 -= s->shift_h[q];
    for (Sub &u : s->subs)
      if (u.removing) u = Sub{};   // free slot (used = false, cs.alive = 0)
  }
  // reference configuration of this collider run
  for (Sub &u : s->subs) {
    if (!u.used) continue;
    std::memcpy(u.cs.Href, u.cs.H, sizeof u.cs.H);
    if (!m_inv(u.cs.Href, u.cs.Hrefinv)) return fail(s, DEM_ERR_INVALID_ARG, "singular periodic cell");
  }
  if ((r = upload_cell(s))) return r;
  // clear pending/request; the error word keeps the history check of this run,
  // which the host reads with the next status block
  CK(cudaMemsetAsync(s->ds_d, 0, 2 * sizeof(int), s->st));
  s->need_rebuild = false;
  s->layout_dirty = false;
  s->check_lost = true;
  s->n_rebuilds += 1;
  CK(cudaGetLastError());
  return DEM_OK;
}

// status block and every sub-scene's cell state (clock, cell, servo gradient)
dem_status read_status(dem_scene *s) {
  CK(cudaMemcpyAsync(s->cs_rb, s->cs_d, sizeof(CellState) * s->nsub(), cudaMemcpyDeviceToHost,
                     s->st));
  CK(cudaMemcpyAsync(&s->rb_h->ds, s->ds_d, sizeof(DevStatus), cudaMemcpyDeviceToHost, s->st));
  dem_status r = wait(s);
  if (r) return r;
  for (int q = 0; q < s->nsub(); ++q) s->subs[q].cs = s->cs_rb[q];
  return DEM_OK;
}

dem_status sync_host(dem_scene *s) {
  if (s->broken) return fail(s, DEM_ERR_STATE, "scene unusable after an earlier CUDA error");
  return wait(s);
}

// Bring pending host-side changes (velGrad, dt) into the device cell states.
dem_status prepare_step(dem_scene *s) {
  for (Sub &u : s->subs)
    if (u.velgrad_pending) {
      std::memcpy(u.cs.L, u.velgrad_next, sizeof u.velgrad_next);
      u.velgrad_pending = false;
      s->cs_dirty = true;
    }
  if (s->cs_dirty) return upload_cell(s);
  return DEM_OK;
}

}  // namespace

namespace dem {
void set_global_error(const std::string &msg) { g_create_error = msg; }

// Used by the server (same thread as the scene's other calls).
long long scene_device_bytes(const dem_scene *s) { return s ? s->dev_bytes : 0; }
long long scene_table_rows(const dem_scene *s) { return s ? s->tab[s->tc].P : 0; }

// Device bytes of one body and of one table row, as alloc_bodies, ensure_bodies and
// ensure_table allocate them: two body buffers (current and permuted) with the wall
// histories and, in mixed precision, the FP32 mirrors; the per-body collider scratch
// and force buffers; the per-body arrays of both tables.  A row: its record in both
// tables (current and the one the next collider run fills), with the 25% headroom
// ensure_table adds.
double scene_bytes_per_body(int mixed) {
  const double d4 = sizeof(double4_32a), f4 = sizeof(float4);
  double buf = 6 * d4 + 3 * sizeof(int) + sizeof(uint8_t) + sizeof(double) + 6 * d4;
  if (mixed) buf += 6 * f4;
  const double scratch = 5 * sizeof(int) + 2 * d4 + f4 + sizeof(int4) +
                        kCandKeep * sizeof(unsigned) + sizeof(int);
  const double tables = 2 * 3 * sizeof(int);
  return 2 * buf + scratch + tables;
}
double scene_bytes_per_row(int mixed) {
  double row = sizeof(int2) + sizeof(int) + sizeof(double4_32a) + 2 * sizeof(int);
  if (mixed) row += 2 * sizeof(float4) + 2 * sizeof(float4) + sizeof(float);
  else row += sizeof(double4_32a) + 2 * sizeof(double4_32a) + sizeof(double);
  return 2 * 1.25 * row;
}
}  // namespace dem

// =================================================================== C ABI
extern "C" {

void dem_scene_desc_init(dem_scene_desc *d) {
  if (!d) return;
  std::memset(d, 0, sizeof *d);
  d->periodic = 0;
  for (int q = 0; q < 9; ++q) d->cell_h[q] = (q % 4 == 0) ? 1.0 : 0.0;
  for (int k = 0; k < 3; ++k) { d->box_lo[k] = 0; d->box_hi[k] = 1; d->gravity[k] = 0; }
  d->wall_mask = 0;
  d->damping = 0.2;
  d->dt = 0;
  d->verlet_dist = -0.5;
  d->precision = DEM_FP64;
  d->capacity_bodies = 0;
  d->capacity_contacts = 0;
  d->cuda_stream = nullptr;
  d->device = -1;
}

const char *dem_version(void) { return "gb300-dem 0.2 (sm_103a, fp64 + mixed)"; }

const char *dem_last_error(const dem_scene *s) {
  return s ? s->err.c_str() : g_create_error.c_str();
}

dem_status dem_scene_create(const dem_scene_desc *desc, dem_scene **out) {
  g_create_error.clear();
  if (!desc || !out) {
    g_create_error = "null argument";
    return DEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (desc->precision != DEM_FP64 && desc->precision != DEM_MIXED) {
    g_create_error = "precision must be DEM_FP64 or DEM_MIXED";
    return DEM_ERR_UNSUPPORTED;
  }
  if (!(desc->damping >= 0) || !(desc->damping < 1)) {
    g_create_error = "damping must be in [0, 1)";
    return DEM_ERR_INVALID_ARG;
  }
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(desc->gravity[k]) || !std::isfinite(desc->box_lo[k]) ||
        !std::isfinite(desc->box_hi[k])) {
      g_create_error = "non-finite gravity or box";
      return DEM_ERR_INVALID_ARG;
    }
  if (desc->periodic) {
    if (!(m_det(desc->cell_h) > 0) || !(desc->cell_h[0] > 0) || !(desc->cell_h[4] > 0) ||
        !(desc->cell_h[8] > 0)) {
      g_create_error = "the periodic cell needs a positive determinant and positive diagonal";
      return DEM_ERR_INVALID_ARG;
    }
  } else if (desc->wall_mask) {
    for (int k = 0; k < 3; ++k)
      if (!(desc->box_hi[k] > desc->box_lo[k])) {
        g_create_error = "box_hi must exceed box_lo";
        return DEM_ERR_INVALID_ARG;
      }
  }
  dem_scene *s = new (std::nothrow) dem_scene();
  if (!s) {
    g_create_error = "out of host memory";
    return DEM_ERR_OOM;
  }
  s->desc = *desc;
  s->has_walls = !desc->periodic && (desc->wall_mask & 0x3F);
  s->mixed = desc->precision == DEM_MIXED;
  if (!s->has_walls) s->desc.wall_mask = 0;
  auto bad = [&](cudaError_t e, const char *what) {
    g_create_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
  };
  cudaError_t e;
  if (desc->device >= 0) {
    if ((e = cudaSetDevice(desc->device)) != cudaSuccess) { bad(e, "cudaSetDevice"); delete s; return DEM_ERR_CUDA; }
    s->device = desc->device;
  } else if ((e = cudaGetDevice(&s->device)) != cudaSuccess) {
    bad(e, "cudaGetDevice");
    delete s;
    return DEM_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device);
  if (desc->cuda_stream) {
    s->st = (cudaStream_t)desc->cuda_stream;
  } else {
    if ((e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking)) != cudaSuccess) {
      bad(e, "cudaStreamCreate");
      delete s;
      return DEM_ERR_CUDA;
    }
    s->own_stream = true;
  }
  if ((e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMallocHost((void **)&s->rb_h, sizeof(Readback))) != cudaSuccess ||
      (e = cudaMallocHost((void **)&s->partials_h, sizeof(double) * 1024 * 32)) != cudaSuccess ||
      (e = cudaMallocHost((void **)&s->step_h, sizeof(StepDesc))) != cudaSuccess) {
    bad(e, "scene setup");
    dem_scene_destroy(s);
    return DEM_ERR_CUDA;
  }
  if (dalloc(s, &s->mats_d, kMaxMat) || dalloc(s, &s->ds_d, 1) ||
      dalloc(s, &s->partials, 1024 * 32) || dalloc(s, &s->servo, kServoBlocks * 6) ||
      dalloc(s, &s->deg_ws, 2 * kDegreeBuckets) || dalloc(s, &s->step_d, 1) || ensure_subs(s, 1)) {
    g_create_error = s->err;
    dem_scene_destroy(s);
    return DEM_ERR_OOM;
  }
  // sub-scene 0: the scene of the descriptor
  s->subs.resize(1);
  Sub &u0 = s->subs[0];
  u0.used = true;
  u0.verlet_rule = desc->verlet_dist;
  CellState &c = u0.cs;
  std::memset(&c, 0, sizeof c);
  init_cell(c, s->desc.periodic, s->desc.cell_h, s->desc.box_lo, s->desc.box_hi,
            s->has_walls ? s->desc.wall_mask : 0, 0, s->desc.gravity, s->desc.damping);
  DevStatus z{};
  if ((e = cudaMemcpyAsync(s->ds_d, &z, sizeof z, cudaMemcpyHostToDevice, s->st)) != cudaSuccess) {
    bad(e, "status init");
    dem_scene_destroy(s);
    return DEM_ERR_CUDA;
  }
  if (desc->capacity_bodies > 0 && ensure_bodies(s, desc->capacity_bodies)) {
    g_create_error = s->err;
    dem_scene_destroy(s);
    return DEM_ERR_OOM;
  }
  if (desc->capacity_contacts > 0 &&
      (ensure_table(s, s->tab[0], desc->capacity_contacts, std::max<long long>(s->cap, 1)) ||
       ensure_table(s, s->tab[1], desc->capacity_contacts, std::max<long long>(s->cap, 1)))) {
    g_create_error = s->err;
    dem_scene_destroy(s);
    return DEM_ERR_OOM;
  }
  u0.dt_set = desc->dt > 0;
  c.dt = u0.dt_set ? desc->dt : 0;
  *out = s;
  return DEM_OK;
}

void dem_scene_destroy(dem_scene *s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  drop_graphs(s);
  dfree(s, s->step_d);
  if (s->step_h) cudaFreeHost(s->step_h);
  free_bodies(s, s->cur);
  free_bodies(s, s->alt);
  free_table(s, s->tab[0]);
  free_table(s, s->tab[1]);
  dfree(s, s->slot_of_id); dfree(s, s->new_to_old); dfree(s, s->cnt_up); dfree(s, s->cnt_down);
  dfree(s, s->key); dfree(s, s->gF); dfree(s, s->gT); dfree(s, s->wpos); dfree(s, s->cinfo);
  dfree(s, s->cand_list); dfree(s, s->cand_n);
  dfree(s, s->cell_count); dfree(s, s->cell_start); dfree(s, s->cell_fill);
  dfree(s, s->scan_ws); dfree(s, s->partials); dfree(s, s->servo); dfree(s, s->p3d_d); dfree(s, s->p3d_part); dfree(s, s->deg_ws);
  dfree(s, s->mats_d); dfree(s, s->cs_d); dfree(s, s->ds_d);
  dfree(s, s->grids_d); dfree(s, s->id_shift_d); dfree(s, s->bbox_keys); dfree(s, s->dt_keys);
  if (s->st) cudaStreamSynchronize(s->st);
  if (s->cs_rb) cudaFreeHost(s->cs_rb);
  if (s->grids_h) cudaFreeHost(s->grids_h);
  if (s->shift_h) cudaFreeHost(s->shift_h);
  if (s->bbox_h) cudaFreeHost(s->bbox_h);
  if (s->rb_h) cudaFreeHost(s->rb_h);
  if (s->partials_h) cudaFreeHost(s->partials_h);
  if (s->ev) cudaEventDestroy(s->ev);
  for (auto &e : s->tev) cudaEventDestroy(e);
  if (s->own_stream && s->st) cudaStreamDestroy(s->st);
  delete s;
}

dem_status dem_set_material(dem_scene *s, int mat, double density, double young, double poisson,
                            double friction) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (mat < 0 || mat >= kMaxMat) return fail(s, DEM_ERR_INVALID_ARG, "material id out of [0, 4095]");
  if (!(density > 0) || !(young > 0) || !(poisson >= 0) || !(friction >= 0) ||
      !(friction < 1.5707963267948966) || !std::isfinite(density) || !std::isfinite(young) ||
      !std::isfinite(poisson))
    return fail(s, DEM_ERR_INVALID_ARG, "bad material parameters");
  Mat m{density, young, poisson, std::tan(friction), 0.0, 0.0};
  mindlin_compliances(m);
  s->mats_h[mat] = m;
  s->mat_set[mat] = true;
  CK(cudaMemcpyAsync(s->mats_d + mat, &s->mats_h[mat], sizeof(Mat), cudaMemcpyHostToDevice, s->st));
  return sync_host(s);
}

namespace {
dem_status add_spheres_sub(dem_scene *s, int q, long long n, const double *pos,
                           const double *radius, const int *mat, const double *vel,
                           const double *angvel, const unsigned char *fixed, long long *first_id) {
  if (n < 0) return fail(s, DEM_ERR_INVALID_ARG, "negative count");
  if (q < 0 || q >= s->nsub() || !s->subs[q].used || s->subs[q].removing)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  Sub &u = s->subs[q];
  if (n == 0) {
    if (first_id) *first_id = u.n ? u.id0 : s->N;
    return DEM_OK;
  }
  // the ids of a sub-scene are consecutive: only the sub-scene holding the last ids
  // (or an empty one) can grow
  if (u.n > 0 && u.id0 + u.n != s->N)
    return fail(s, DEM_ERR_UNSUPPORTED,
                "spheres can be added only to the sub-scene that received the last ones");
  if (!pos || !radius) return fail(s, DEM_ERR_INVALID_ARG, "null pos or radius");
  if (s->N + n > 0x7fffffffLL) return fail(s, DEM_ERR_CAPACITY, "more than 2^31-1 bodies");
  for (long long i = 0; i < n; ++i) {
    int m = mat ? mat[i] : 0;
    if (m < 0 || m >= kMaxMat || !s->mat_set[m])
      return fail(s, DEM_ERR_INVALID_ARG, "unknown material id (set_material first)");
    if (!(radius[i] > 0) || !std::isfinite(radius[i]))
      return fail(s, DEM_ERR_INVALID_ARG, "radius must be positive and finite");
    for (int k = 0; k < 3; ++k) {
      if (!std::isfinite(pos[3 * i + k]) || (vel && !std::isfinite(vel[3 * i + k])) ||
          (angvel && !std::isfinite(angvel[3 * i + k])))
        return fail(s, DEM_ERR_NONFINITE, "non-finite position or velocity");
    }
  }
  dem_status r;
  if ((r = sync_host(s))) return r;
  if ((r = ensure_bodies(s, s->N + n))) return r;
  std::vector<double4_32a> P(n), V(n), A(n), O(n), M(n);
  std::vector<int> ID(n), MT(n), SU(n, q);
  std::vector<uint8_t> FL(n);
  std::vector<int> SL(n);
  const double pi = 3.14159265358979323846;
  for (long long t = 0; t < n; ++t) {
    int m = mat ? mat[t] : 0;
    double rr = radius[t];
    P[t] = make_double4_32a(pos[3 * t], pos[3 * t + 1], pos[3 * t + 2], rr);
    V[t] = vel ? make_double4_32a(vel[3 * t], vel[3 * t + 1], vel[3 * t + 2], 0) : make_double4_32a(0, 0, 0, 0);
    A[t] = angvel ? make_double4_32a(angvel[3 * t], angvel[3 * t + 1], angvel[3 * t + 2], 0)
                  : make_double4_32a(0, 0, 0, 0);
    O[t] = make_double4_32a(1, 0, 0, 0);
    // utils.sphere: m = density 4/3 pi r^3, I = 2/5 m r^2
    double mass = s->mats_h[m].density * (4.0 / 3.0) * pi * rr * rr * rr;
    double I = 0.4 * mass * rr * rr;
    M[t] = make_double4_32a(mass, I, 1.0 / mass, 1.0 / I);
    ID[t] = (int)(s->N + t);
    MT[t] = m;
    FL[t] = (fixed && fixed[t]) ? 1 : 0;
    SL[t] = (int)(s->N + t);
    u.rmin = std::min(u.rmin, rr);
    u.rmax = std::max(u.rmax, rr);
    u.vsolid += (4.0 / 3.0) * pi * rr * rr * rr;
    s->radius_h.push_back(rr);
    s->mat_h.push_back(m);
    s->fixed_h.push_back(FL[t]);
  }
  const long long o = s->N;
  const size_t d4 = sizeof(double4_32a) * n;
  CK(cudaMemcpyAsync(s->cur.pos + o, P.data(), d4, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.vel + o, V.data(), d4, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.angvel + o, A.data(), d4, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.ori + o, O.data(), d4, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.xref + o, P.data(), d4, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.mprop + o, M.data(), d4, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.id + o, ID.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.sid + o, SU.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.mat + o, MT.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->cur.flags + o, FL.data(), n, cudaMemcpyHostToDevice, s->st));
  const std::vector<double> ones(n, 1.0);   // no density scaling yet
  CK(cudaMemcpyAsync(s->cur.rdsc + o, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->slot_of_id + o, SL.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s->st));
  for (int w = 0; w < 6; ++w) CK(cudaMemsetAsync(s->cur.whist + w * s->cap + o, 0, d4, s->st));
  if (s->mixed) {   // FP32 mirrors of the new bodies (the collider run refreshes p32, vw32)
    std::vector<float4> M32(n), O32(n, make_float4(1, 0, 0, 0));
    for (long long t = 0; t < n; ++t)
      M32[t] = make_float4((float)M[t].x, (float)M[t].y, (float)M[t].z, (float)M[t].w);
    CK(cudaMemcpyAsync(s->cur.mprop32 + o, M32.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->cur.ori32 + o, O32.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, s->st));
  }
  if (first_id) *first_id = s->N;
  if (u.n == 0) u.id0 = s->N;
  u.n += n;
  s->N += n;
  s->need_rebuild = true;
  s->layout_dirty = true;
  s->table_fresh = false;
  s->check_lost = false;
  // sweep margin: > 0 absolute, < 0 fraction of the smallest radius
  const double vd = u.verlet_rule;
  u.cs.verlet = vd > 0 ? vd : (vd < 0 ? -vd * u.rmin : 0.5 * u.rmin);
  u.cs.rmax = u.rmax;
  s->cs_dirty = true;
  return sync_host(s);
}
}  // namespace

dem_status dem_add_spheres(dem_scene *s, long long n, const double *pos, const double *radius,
                           const int *mat, const double *vel, const double *angvel,
                           const unsigned char *fixed, long long *first_id) {
  if (!s) return DEM_ERR_INVALID_ARG;
  return add_spheres_sub(s, 0, n, pos, radius, mat, vel, angvel, fixed, first_id);
}


dem_status dem_set_dt(dem_scene *s, double dt) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (!(dt > 0) || !std::isfinite(dt)) return fail(s, DEM_ERR_INVALID_ARG, "dt must be positive");
  s->cs0().dt = dt;
  s->subs[0].dt_set = true;
  s->cs_dirty = true;
  return DEM_OK;
}

dem_status dem_get_dt(dem_scene *s, double *dt) {
  if (!s || !dt) return DEM_ERR_INVALID_ARG;
  dem_status r = ensure_dt(s);
  if (r) return r;
  *dt = s->cs0().dt;
  return DEM_OK;
}

dem_status dem_set_triax(dem_scene *s, const double *goal, int stress_mask,
                         const double *max_rate, double grow_damping, int glob_update) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (!s->desc.periodic) return fail(s, DEM_ERR_STATE, "the stress servo needs a periodic scene");
  if (s->nsub() > 1)
    return fail(s, DEM_ERR_UNSUPPORTED, "the stress servo runs on a scene without sub-scenes");
  if (!goal || !max_rate || glob_update < 1 || !(grow_damping >= 0) || !(grow_damping < 1))
    return fail(s, DEM_ERR_INVALID_ARG, "bad servo parameters");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(goal[a]) || !(max_rate[a] >= 0) || !std::isfinite(max_rate[a]))
      return fail(s, DEM_ERR_INVALID_ARG, "bad servo goal or rate bound");
  dem_status r;
  if ((r = sync_host(s))) return r;
  for (int a = 0; a < 3; ++a) {
    s->cs0().goal[a] = goal[a];
    s->cs0().max_rate[a] = max_rate[a];
  }
  s->cs0().stress_mask = stress_mask & 7;
  s->cs0().grow_damping = grow_damping;
  s->cs0().glob_update = glob_update;
  s->cs0().triax = 1;
  s->p3d_on = false;   // one cell controller at a time
  s->cs_dirty = true;
  return DEM_OK;
}

dem_status dem_set_peri3d(dem_scene *s, const double *goal, int stress_mask, long long n_steps,
                          double mod, double max_strain_rate, double young_est, double poisson_est,
                          double max_strain, const int *npath, const double *path,
                          const double *trsf0) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (!s->desc.periodic) return fail(s, DEM_ERR_STATE, "Peri3dController needs a periodic scene");
  if (s->nsub() > 1)
    return fail(s, DEM_ERR_UNSUPPORTED, "Peri3dController runs on a scene without sub-scenes");
  if (!goal || n_steps < 1 || !(max_strain_rate > 0) || !std::isfinite(max_strain_rate) ||
      !(young_est > 0) || !(poisson_est > -1 && poisson_est < 0.5) || !(max_strain > 0) ||
      !(mod >= 0) || !std::isfinite(mod))
    return fail(s, DEM_ERR_INVALID_ARG, "bad Peri3dController parameters");
  P3d P{};
  for (int i = 0; i < 6; ++i) {
    if (!std::isfinite(goal[i])) return fail(s, DEM_ERR_INVALID_ARG, "non-finite goal");
    P.goal[i] = goal[i];
    const int n = npath ? npath[i] : 0;
    if (n < 0 || n > 16 || (n > 0 && !path)) return fail(s, DEM_ERR_INVALID_ARG, "bad path size");
    if (n == 0) {   // default: linear from 0 to the goal
      P.npath[i] = 1;
      P.path[i][0][0] = 1.0;
      P.path[i][0][1] = 1.0;
      continue;
    }
    P.npath[i] = n;
    for (int j = 0; j < n; ++j) {
      P.path[i][j][0] = path[(16 * i + j) * 2];
      P.path[i][j][1] = path[(16 * i + j) * 2 + 1];
      if (!std::isfinite(P.path[i][j][0]) || !std::isfinite(P.path[i][j][1]) ||
          !(P.path[i][j][0] > (j ? P.path[i][j - 1][0] : 0.0)))
        return fail(s, DEM_ERR_INVALID_ARG, "path times must increase from a positive first one");
    }
    if (P.path[i][n - 1][1] == 0.0)
      return fail(s, DEM_ERR_INVALID_ARG, "the last couple of a path stands for the goal: nonzero value");
  }
  for (int q = 0; q < 9; ++q) P.T0[q] = trsf0 ? trsf0[q] : ((q % 4 == 0) ? 1.0 : 0.0);
  if (trsf0 && !(m_det(P.T0) > 0)) return fail(s, DEM_ERR_INVALID_ARG, "trsf0 needs det > 0");
  dem_status r;
  if ((r = sync_host(s))) return r;
  if (!m_inv(s->cs0().H, P.H0inv)) return fail(s, DEM_ERR_INVALID_ARG, "singular cell");
  P.on = 1;
  P.mask = stress_mask & 63;
  P.first = 1;
  P.nsteps = n_steps;
  P.mod = mod;
  P.max_rate = max_strain_rate;
  P.young = young_est;
  P.poisson = poisson_est;
  P.max_strain = max_strain;
  if (!s->p3d_d && ((r = dalloc(s, &s->p3d_d, 1)) || (r = dalloc(s, &s->p3d_part, kServoBlocks * 9))))
    return r;
  s->p3d_h = P;
  CK(cudaMemcpyAsync(s->p3d_d, &s->p3d_h, sizeof(P3d), cudaMemcpyHostToDevice, s->st));
  if ((r = wait(s))) return r;
  s->p3d_on = true;
  s->cs0().triax = 0;   // one cell controller at a time
  s->cs_dirty = true;
  return DEM_OK;
}

dem_status dem_get_peri3d(dem_scene *s, double *stress, double *strain, double *rate, int *done) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (!s->p3d_on) return fail(s, DEM_ERR_STATE, "no Peri3dController on this scene");
  dem_status r;
  if ((r = sync_host(s))) return r;
  CK(cudaMemcpyAsync(&s->p3d_h, s->p3d_d, sizeof(P3d), cudaMemcpyDeviceToHost, s->st));
  if ((r = wait(s))) return r;
  for (int i = 0; i < 6; ++i) {
    if (stress) stress[i] = s->p3d_h.stress[i];
    if (strain) strain[i] = s->p3d_h.strain[i];
    if (rate) rate[i] = s->p3d_h.rate[i];
  }
  if (done) *done = s->p3d_h.done;
  return DEM_OK;
}

dem_status dem_set_cell_velgrad(dem_scene *s, const double *L) {
  if (!s || !L) return DEM_ERR_INVALID_ARG;
  if (!s->desc.periodic) return fail(s, DEM_ERR_STATE, "velGrad needs a periodic scene");
  for (int q = 0; q < 9; ++q)
    if (!std::isfinite(L[q])) return fail(s, DEM_ERR_INVALID_ARG, "non-finite velGrad");
  std::memcpy(s->subs[0].velgrad_next, L, sizeof s->subs[0].velgrad_next);
  s->subs[0].velgrad_pending = true;
  return DEM_OK;
}


dem_status dem_step(dem_scene *s, long long nsteps) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (nsteps < 0) return fail(s, DEM_ERR_INVALID_ARG, "negative step count");
  if (s->broken) return fail(s, DEM_ERR_STATE, "scene unusable after an earlier CUDA error");
  if (nsteps == 0) return DEM_OK;
  dem_status r;
  if (s->N == 0) {
    bool any = false;
    for (Sub &u : s->subs) {
      if (!u.used || !u.dt_set) continue;
      for (long long k = 0; k < nsteps; ++k) u.cs.time += u.cs.dt;
      u.cs.iter += nsteps;
      any = true;
    }
    if (!any) return fail(s, DEM_ERR_STATE, "no bodies and no time step");
    s->cs_dirty = true;
    return DEM_OK;
  }
  if ((r = ensure_dt(s))) return r;
  if ((r = prepare_step(s))) return r;
  long long remaining = nsteps;
  while (remaining > 0) {
    if (s->need_rebuild && (r = rebuild(s))) return r;
    const SceneConst sc = scene_const(s);
    const long long B = std::min<long long>(remaining, s->batch);
    const long long it0 = s->cs0().iter;
    const Table &t = s->tab[s->tc];
    cudaEvent_t *ev = s->timing ? s->tev.data() + 2 : nullptr;
    // the step kernels read tables and bodies through the step descriptor
    *s->step_h = StepDesc{t, s->cur, sc, s->cap};
    CK(cudaMemcpyAsync(s->step_d, s->step_h, sizeof(StepDesc), cudaMemcpyHostToDevice, s->st));
    const long long rows = std::max(s->tab[0].cap, s->tab[1].cap);
    const bool servo = !sc.multi && s->cs0().triax;
    const bool p3d = !sc.multi && s->p3d_on;
    bool tstep = false;
    for (const Sub &u : s->subs) tstep |= u.used && u.cs.tstep;
    auto tstep_due = [&](long long i) {
      for (const Sub &u : s->subs)
        if (u.used && u.cs.tstep && (u.cs.iter + i) % u.cs.tstep_interval == 0) return true;
      return false;
    };
    // captured batches read the descriptor; launched ones take the arrays as parameters
    const bool use_graph = (s->step_graphs > 0 || (s->step_graphs < 0 && sc.N < kGraphAutoBodies)) &&
                           !ev && !servo && !tstep && !p3d;
    bool desc = use_graph;
    auto launch_steps = [&](bool record) -> dem_status {
      for (long long i = 0; i < B; ++i) {
        if (record) CK(cudaEventRecord(ev[6 * i], s->st));
        if (s->mixed)
          launch_contact_mixed(s->step_d, *s->step_h, desc, rows, s->cs_d, s->ds_d, s->mats_d,
                               sc.multi, sc.hertz | (sc.sheared << 1), s->nsm,
                               s->contact_block, s->contact_per_sm, s->st);
        else
          launch_contact(s->step_d, *s->step_h, desc, rows, s->cs_d, s->ds_d, s->mats_d,
                         sc.multi, sc.hertz | (sc.sheared << 1), s->nsm, s->contact_block,
                         s->contact_per_sm, s->st);
        if (record) CK(cudaEventRecord(ev[6 * i + 1], s->st));
        if (tstep && tstep_due(i)) {   // GlobalStiffnessTimeStepper: after the contacts
          launch_timestepper(s->cur, t, s->cs_d, s->nsub(), s->ds_d, s->mats_d, sc.N, s->cap,
                             s->mixed, sc.multi, sc.walls, s->dt_keys, s->st);
          s->launches += 2;
        }
        if (record) CK(cudaEventRecord(ev[6 * i + 2], s->st));
        launch_integrate(s->step_d, *s->step_h, desc, s->cs_d, s->ds_d, s->mats_d, s->mixed,
                         s->integrate_block, s->st);
        if (record) { CK(cudaEventRecord(ev[6 * i + 3], s->st)); CK(cudaEventRecord(ev[6 * i + 4], s->st)); }
        // servo update steps (PeriTriaxController every glob_update steps)
        const bool upd = servo && ((it0 + i + 1) % s->cs0().glob_update == 0);
        if (upd) {
          launch_servo_partials(t, s->cur, s->ds_d, s->mixed, s->cs0().law, s->servo, s->st);
          s->launches += 1;
        }
        if (p3d) {   // Peri3dController: every step, from this step's contacts
          launch_p3d_partials(t, s->ds_d, s->mixed, s->p3d_part, s->st);
          s->launches += 2;
        }
        launch_cell_advance(s->cs_d, s->nsub(), s->ds_d, upd ? s->servo : nullptr, s->st,
                            p3d ? s->p3d_d : nullptr, s->p3d_part);
        if (record) CK(cudaEventRecord(ev[6 * i + 5], s->st));
      }
      return DEM_OK;
    };
    if (use_graph) {
      // replay a captured batch of B steps (one graph launch instead of 3B launches);
      // captures are kept while nothing that shapes the launches changes
      const GraphKey key{sc.N, rows, s->contact_block, s->contact_per_sm, s->integrate_block,
                         sc.multi, sc.walls | (sc.hertz << 1) | (sc.sheared << 2), s->nsub(),
                         s->mixed ? 1 : 0,
                         s->cs_d};
      if (!(key == s->graph_key)) {
        drop_graphs(s);
        s->graph_key = key;
      }
      cudaGraphExec_t &ex = s->graphs[B];
      if (!ex) {
        CK(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
        const long long keep = s->launches;
        dem_status q = launch_steps(false);
        s->launches = keep;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s->st, &g);
        if (q) return q;
        if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          ex = nullptr;
          return cuda_fail(s, e, "cudaGraphInstantiate");
        }
      }
      CK(cudaGraphLaunch(ex, s->st));
    } else {
      desc = false;
      if ((r = launch_steps(ev != nullptr))) return r;
    }
    s->launches += B * ((rows > 0 ? 1 : 0) + 2);
    CK(cudaGetLastError());
    if ((r = read_status(s))) return r;
    s->table_fresh = true;
    const long long done_b = (long long)(s->rb_h->ds.steps - s->steps_seen);
    if (ev) {
      // all B launches are timed (the ones skipped after a collider request return at
      // once); they are counted as the steps actually done, so a per-launch average is
      // the time of a working launch, slightly over-estimated
      for (long long i = 0; i < B; ++i) {
        float a = 0, b = 0, c = 0;
        CK(cudaEventElapsedTime(&a, ev[6 * i], ev[6 * i + 1]));
        CK(cudaEventElapsedTime(&b, ev[6 * i + 2], ev[6 * i + 3]));
        CK(cudaEventElapsedTime(&c, ev[6 * i + 4], ev[6 * i + 5]));
        s->tm.contact_ms += a;
        s->tm.integrate_ms += b;
        s->tm.cell_ms += c;
      }
      s->tm.contact_launches += t.P > 0 ? done_b : 0;
      s->tm.integrate_launches += done_b;
      s->tm.cell_launches += done_b;
      s->tm.rows_processed += done_b * t.P;
    }
    const DevStatus ds = s->rb_h->ds;
    const long long done = done_b;
    s->steps_seen = ds.steps;
    if (ds.error) return status_error(s, ds.error);
    remaining -= done;
    if (ds.pending) {
      s->need_rebuild = true;
      // aim the next batch at the observed interval between collider runs
      s->batch = std::max<long long>(4, std::min<long long>(64, done + 1));
    } else if (done != B) {
      return fail(s, DEM_ERR_STATE, "internal: steps were skipped without a collider request");
    } else {
      s->batch = std::min<long long>(64, s->batch + 4);
    }
  }
  return DEM_OK;
}

static dem_status fetch4(dem_scene *s, const double4_32a *src, const std::vector<int> &sid, double *out,
                         int comps) {
  const long long N = s->N;
  std::vector<double4_32a> h(N);
  CK(cudaMemcpyAsync(h.data(), src, sizeof(double4_32a) * N, cudaMemcpyDeviceToHost, s->st));
  dem_status r = wait(s);
  if (r) return r;
  for (long long i = 0; i < N; ++i) {
    const double4_32a &v = h[sid[i]];
    const double c[4] = {v.x, v.y, v.z, v.w};
    for (int k = 0; k < comps; ++k) out[comps * i + k] = c[k];
  }
  return DEM_OK;
}

static dem_status fetch_sid(dem_scene *s, std::vector<int> &sid) {
  sid.resize(s->N);
  if (s->N == 0) return DEM_OK;
  CK(cudaMemcpyAsync(sid.data(), s->slot_of_id, sizeof(int) * s->N, cudaMemcpyDeviceToHost, s->st));
  return wait(s);
}

dem_status dem_get_state(dem_scene *s, double *pos, double *vel, double *angvel, double *ori,
                         double *force, double *torque) {
  if (!s) return DEM_ERR_INVALID_ARG;
  dem_status r;
  if ((r = sync_host(s))) return r;
  if (s->N == 0) return DEM_OK;
  std::vector<int> sid;
  if ((r = fetch_sid(s, sid))) return r;
  if (pos && (r = fetch4(s, s->cur.pos, sid, pos, 3))) return r;
  if (vel && (r = fetch4(s, s->cur.vel, sid, vel, 3))) return r;
  if (angvel && (r = fetch4(s, s->cur.angvel, sid, angvel, 3))) return r;
  if (ori) {
    if (s->mixed) {
      std::vector<float4> h(s->N);
      CK(cudaMemcpyAsync(h.data(), s->cur.ori32, sizeof(float4) * s->N, cudaMemcpyDeviceToHost, s->st));
      if ((r = wait(s))) return r;
      for (long long i = 0; i < s->N; ++i) {
        const float4 &q = h[sid[i]];
        ori[4 * i] = q.x; ori[4 * i + 1] = q.y; ori[4 * i + 2] = q.z; ori[4 * i + 3] = q.w;
      }
    } else if ((r = fetch4(s, s->cur.ori, sid, ori, 4))) {
      return r;
    }
  }
  if (force || torque) {
    if (!s->table_fresh) {
      // no contact table matches the current body order yet: no contact forces
      if (force) std::memset(force, 0, sizeof(double) * 3 * s->N);
      if (torque) std::memset(torque, 0, sizeof(double) * 3 * s->N);
      return DEM_OK;
    }
    launch_gather_forces(s->cur, s->tab[s->tc], s->mats_d, s->cs_d, scene_const(s), s->cap,
                         s->gF, s->gT, s->mixed, s->st);
    CK(cudaGetLastError());
    if (force && (r = fetch4(s, s->gF, sid, force, 3))) return r;
    if (torque && (r = fetch4(s, s->gT, sid, torque, 3))) return r;
  }
  return DEM_OK;
}

dem_status dem_set_state(dem_scene *s, const double *pos, const double *vel, const double *angvel,
                         const double *ori) {
  if (!s) return DEM_ERR_INVALID_ARG;
  dem_status r;
  if ((r = sync_host(s))) return r;
  const long long N = s->N;
  if (N == 0) return DEM_OK;
  for (long long i = 0; i < 3 * N; ++i)
    if ((pos && !std::isfinite(pos[i])) || (vel && !std::isfinite(vel[i])) ||
        (angvel && !std::isfinite(angvel[i])))
      return fail(s, DEM_ERR_NONFINITE, "non-finite state");
  std::vector<int> sid;
  if ((r = fetch_sid(s, sid))) return r;
  std::vector<double4_32a> h(N);
  auto put = [&](const double *src, double4_32a *dst, int comps, bool radius_w) -> dem_status {
    for (long long i = 0; i < N; ++i) {
      const double *p = src + comps * i;
      double w = radius_w ? s->radius_h[i] : (comps == 4 ? p[3] : 0.0);
      h[sid[i]] = make_double4_32a(p[0], p[1], p[2], w);
    }
    CK(cudaMemcpyAsync(dst, h.data(), sizeof(double4_32a) * N, cudaMemcpyHostToDevice, s->st));
    return wait(s);
  };
  if (pos && (r = put(pos, s->cur.pos, 3, true))) return r;
  if (vel && (r = put(vel, s->cur.vel, 3, false))) return r;
  if (angvel && (r = put(angvel, s->cur.angvel, 3, false))) return r;
  if (ori && (r = put(ori, s->cur.ori, 4, false))) return r;
  if (ori && s->mixed) {
    std::vector<float4> h32(N);
    for (long long i = 0; i < N; ++i)
      h32[sid[i]] = make_float4((float)ori[4 * i], (float)ori[4 * i + 1], (float)ori[4 * i + 2],
                                (float)ori[4 * i + 3]);
    CK(cudaMemcpyAsync(s->cur.ori32, h32.data(), sizeof(float4) * N, cudaMemcpyHostToDevice, s->st));
    if ((r = wait(s))) return r;
  }
  if (pos) {
    s->need_rebuild = true;
    s->table_fresh = false;
    s->check_lost = false;
  }
  if (s->mixed && (vel || angvel)) s->need_rebuild = true;   // refresh the FP32 mirrors
  return DEM_OK;
}

dem_status dem_get_cell(dem_scene *s, double *H, double *velgrad, double *prev_velgrad,
                        double *prev_H) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (!s->desc.periodic) return fail(s, DEM_ERR_STATE, "the scene is not periodic");
  dem_status r;
  if ((r = sync_host(s))) return r;
  if (H) std::memcpy(H, s->cs0().H, sizeof s->cs0().H);
  if (velgrad)
    std::memcpy(velgrad, s->subs[0].velgrad_pending ? s->subs[0].velgrad_next : s->cs0().L,
                sizeof s->cs0().L);
  if (prev_velgrad) std::memcpy(prev_velgrad, s->cs0().Lprev, sizeof s->cs0().Lprev);
  if (prev_H) std::memcpy(prev_H, s->cs0().Hprev, sizeof s->cs0().Hprev);
  return DEM_OK;
}

dem_status dem_set_cell(dem_scene *s, const double *H, const double *velgrad,
                        const double *prev_velgrad, const double *prev_H) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (!s->desc.periodic) return fail(s, DEM_ERR_STATE, "the scene is not periodic");
  for (const double *M : {H, velgrad, prev_velgrad, prev_H})
    if (M) {
      for (int q = 0; q < 9; ++q)
        if (!std::isfinite(M[q])) return fail(s, DEM_ERR_INVALID_ARG, "non-finite cell matrix");
    }
  if (H && !(H[0] > 0 && H[4] > 0 && H[8] > 0 && m_det(H) > 0))
    return fail(s, DEM_ERR_INVALID_ARG, "cell needs a positive determinant and positive diagonal");
  dem_status r;
  if ((r = sync_host(s))) return r;
  if (H) {
    std::memcpy(s->cs0().H, H, sizeof s->cs0().H);
    s->need_rebuild = true;
    s->table_fresh = false;
    s->check_lost = false;
  }
  if (velgrad) {
    std::memcpy(s->cs0().L, velgrad, sizeof s->cs0().L);
    s->subs[0].velgrad_pending = false;
  }
  if (prev_velgrad) std::memcpy(s->cs0().Lprev, prev_velgrad, sizeof s->cs0().Lprev);
  if (prev_H) std::memcpy(s->cs0().Hprev, prev_H, sizeof s->cs0().Hprev);
  s->cs_dirty = true;
  return DEM_OK;
}

dem_status dem_get_clock(dem_scene *s, long long *iter, double *time) {
  if (!s) return DEM_ERR_INVALID_ARG;
  dem_status r;
  if ((r = sync_host(s))) return r;
  if (iter) *iter = s->cs0().iter;
  if (time) *time = s->cs0().time;
  return DEM_OK;
}

dem_status dem_set_clock(dem_scene *s, long long iter, double time) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (iter < 0 || !std::isfinite(time)) return fail(s, DEM_ERR_INVALID_ARG, "bad clock");
  dem_status r;
  if ((r = sync_host(s))) return r;
  s->cs0().iter = iter;
  s->cs0().time = time;
  s->cs_dirty = true;
  return DEM_OK;
}

namespace {
struct HostContact {
  int id1, id2, c[3];
  double fn[3], fs[3], n[3], cp[3], phys[3], pen;
};

void wall_phys_h(const dem_scene *s, int wmat, int mat, double r, double &kn, double &ks,
                 double &tp, int law) {
  const Mat &mw = s->mats_h[wmat], &ms = s->mats_h[mat];
  tp = std::min(mw.tanphi, ms.tanphi);
  if (law) {   // Hertz-Mindlin constants kno, kso with an infinite wall radius
    mindlin_phys(ms, r, mw, -1.0, kn, ks);
    return;
  }
  double k1 = mw.young * (2 * r), k2 = ms.young * (2 * r);
  kn = k1 * k2 / (k1 + k2);
  double s1 = mw.young * mw.poisson * (2 * r), s2 = ms.young * ms.poisson * (2 * r);
  ks = s1 * s2 / (s1 + s2);
}

dem_status collect_contacts(dem_scene *s, std::vector<HostContact> &out) {
  out.clear();
  dem_status r;
  if ((r = sync_host(s))) return r;
  const long long N = s->N;
  if (N == 0 || !s->table_fresh) return DEM_OK;
  const Table &t = s->tab[s->tc];
  const long long P = t.P;
  std::vector<int2> pair(P);
  std::vector<int> cp(P), id(N);
  std::vector<double4_32a> hfs(P), hn(P), oF(P), oM(P), oFM, pos(N);
  std::vector<double> tp(P);
  std::vector<float4> g32, hn32, oFM32;
  if (P > 0) {
    CK(cudaMemcpyAsync(pair.data(), t.pair, sizeof(int2) * P, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(cp.data(), t.cpack, sizeof(int) * P, cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(hfs.data(), t.hfs, sizeof(double4_32a) * P, cudaMemcpyDeviceToHost, s->st));
    if (s->mixed) {
      g32.resize(P); hn32.resize(P); oFM32.resize(2 * P);
      CK(cudaMemcpyAsync(g32.data(), t.g32, sizeof(float4) * P, cudaMemcpyDeviceToHost, s->st));
      CK(cudaMemcpyAsync(hn32.data(), t.hn32, sizeof(float4) * P, cudaMemcpyDeviceToHost, s->st));
      CK(cudaMemcpyAsync(oFM32.data(), t.oFM32, sizeof(float4) * 2 * P, cudaMemcpyDeviceToHost, s->st));
    } else {
      CK(cudaMemcpyAsync(hn.data(), t.hn, sizeof(double4_32a) * P, cudaMemcpyDeviceToHost, s->st));
      oFM.resize(2 * P);
      CK(cudaMemcpyAsync(oFM.data(), t.oFM, sizeof(double4_32a) * 2 * P, cudaMemcpyDeviceToHost, s->st));
      CK(cudaMemcpyAsync(tp.data(), t.tanphi, sizeof(double) * P, cudaMemcpyDeviceToHost, s->st));
    }
  }
  CK(cudaMemcpyAsync(id.data(), s->cur.id, sizeof(int) * N, cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(pos.data(), s->cur.pos, sizeof(double4_32a) * N, cudaMemcpyDeviceToHost, s->st));
  std::vector<uint8_t> flags(N);
  std::vector<double4_32a> wh;
  CK(cudaMemcpyAsync(flags.data(), s->cur.flags, N, cudaMemcpyDeviceToHost, s->st));
  if (s->has_walls) {
    wh.resize(6 * N);
    for (int w = 0; w < 6; ++w)
      CK(cudaMemcpyAsync(wh.data() + w * N, s->cur.whist + w * s->cap, sizeof(double4_32a) * N,
                         cudaMemcpyDeviceToHost, s->st));
  }
  if ((r = wait(s))) return r;
  if (s->mixed) {   // one view of both layouts: hfs = (Fs, kn), hn = (n, ks), tp = tan(phi)
    for (long long k = 0; k < P; ++k) {
      tp[k] = hfs[k].w;
      hfs[k].w = g32[k].w;
      hn[k] = make_double4_32a(hn32[k].x, hn32[k].y, hn32[k].z, hn32[k].w);
      const float4 f = oFM32[2 * k], m = oFM32[2 * k + 1];
      oF[k] = make_double4_32a(f.x, f.y, f.z, f.w);
      oM[k] = make_double4_32a(m.x, m.y, m.z, m.w);
    }
  } else {
    for (long long k = 0; k < P; ++k) {
      oF[k] = oFM[2 * k];
      oM[k] = oFM[2 * k + 1];
    }
  }
  for (long long k = 0; k < P; ++k) {
    if (hfs[k].w == 0.0) continue;
    HostContact h{};
    int a = pair[k].x, b = pair[k].y;
    int c0, c1, c2;
    unpack_shift(cp[k], c0, c1, c2);
    double sg = 1.0;
    const double F[3] = {oF[k].x, oF[k].y, oF[k].z};
    const double fs[3] = {hfs[k].x, hfs[k].y, hfs[k].z};
    const double n[3] = {hn[k].x, hn[k].y, hn[k].z};
    const double d1 = oF[k].w;
    const double r1 = pos[a].w;
    const double pen = 2.0 * (r1 - d1);
    if (id[a] < id[b]) {
      h.id1 = id[a]; h.id2 = id[b]; h.c[0] = c0; h.c[1] = c1; h.c[2] = c2;
    } else {
      h.id1 = id[b]; h.id2 = id[a]; h.c[0] = -c0; h.c[1] = -c1; h.c[2] = -c2; sg = -1.0;
    }
    for (int q = 0; q < 3; ++q) {
      h.fs[q] = sg * fs[q];
      h.fn[q] = sg * (F[q] - fs[q]);
      h.n[q] = sg * n[q];
    }
    // contact point x1 + (r1 - pen/2) n from the current position of the slot-first body
    const double pa[3] = {pos[a].x, pos[a].y, pos[a].z};
    for (int q = 0; q < 3; ++q) h.cp[q] = pa[q] + d1 * n[q];
    h.phys[0] = hfs[k].w; h.phys[1] = hn[k].w; h.phys[2] = tp[k];
    h.pen = pen;
    out.push_back(h);
  }
  if (s->has_walls) {
    std::vector<int> wmat(N, 0), wlaw(N, 0);   // wall material and law of each id's sub-scene
    for (const Sub &u : s->subs)
      if (u.used || u.removing)
        for (long long i = u.id0; i < u.id0 + u.n && i < N; ++i) {
          wmat[i] = u.cs.wall_mat;
          wlaw[i] = u.cs.law;
        }
    for (long long sl = 0; sl < N; ++sl) {
      if (!(flags[sl] & 0x7e)) continue;
      for (int w = 0; w < 6; ++w) {
        if (!(flags[sl] & (2 << w))) continue;
        const double4_32a hw = wh[w * N + sl];
        HostContact h{};
        int ax = w >> 1;
        double sn = hw.w >= 0 ? 1.0 : -1.0, Fn = std::fabs(hw.w);
        h.id1 = -(w + 1);
        h.id2 = id[sl];
        double kn, ks, tanp;
        const double rr = pos[sl].w;
        const int law = wlaw[id[sl]];
        wall_phys_h(s, wmat[id[sl]], s->mat_h[id[sl]], rr, kn, ks, tanp, law);
        h.n[ax] = sn;
        h.fn[ax] = sn * Fn;
        h.fs[0] = hw.x; h.fs[1] = hw.y; h.fs[2] = hw.z;
        h.pen = wall_pen(Fn, kn, law);
        const double pp[3] = {pos[sl].x, pos[sl].y, pos[sl].z};
        for (int q = 0; q < 3; ++q) h.cp[q] = pp[q] - (rr - 0.5 * h.pen) * h.n[q];
        h.phys[0] = kn; h.phys[1] = ks; h.phys[2] = tanp;
        out.push_back(h);
      }
    }
  }
  std::sort(out.begin(), out.end(), [](const HostContact &x, const HostContact &y) {
    return x.id1 != y.id1 ? x.id1 < y.id1 : x.id2 < y.id2;
  });
  return DEM_OK;
}
}  // namespace

dem_status dem_count_contacts(dem_scene *s, long long *count) {
  if (!s || !count) return DEM_ERR_INVALID_ARG;
  std::vector<HostContact> v;
  dem_status r = collect_contacts(s, v);
  if (r) return r;
  *count = (long long)v.size();
  return DEM_OK;
}

dem_status dem_get_contacts(dem_scene *s, long long cap, long long *count, int *id1, int *id2,
                            int *cell_dist, double *normal_force, double *shear_force,
                            double *normal, double *contact_point, double *phys, double *pen) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (cap < 0) return fail(s, DEM_ERR_INVALID_ARG, "negative capacity");
  std::vector<HostContact> v;
  dem_status r = collect_contacts(s, v);
  if (r) return r;
  if (count) *count = (long long)v.size();
  long long m = std::min<long long>(cap, (long long)v.size());
  for (long long k = 0; k < m; ++k) {
    const HostContact &h = v[k];
    if (id1) id1[k] = h.id1;
    if (id2) id2[k] = h.id2;
    for (int q = 0; q < 3; ++q) {
      if (cell_dist) cell_dist[3 * k + q] = h.c[q];
      if (normal_force) normal_force[3 * k + q] = h.fn[q];
      if (shear_force) shear_force[3 * k + q] = h.fs[q];
      if (normal) normal[3 * k + q] = h.n[q];
      if (contact_point) contact_point[3 * k + q] = h.cp[q];
      if (phys) phys[3 * k + q] = h.phys[q];
    }
    if (pen) pen[k] = h.pen;
  }
  return DEM_OK;
}

dem_status dem_set_contacts(dem_scene *s, long long n, const int *id1, const int *id2,
                            const int *cell_dist, const double *shear_force,
                            const double *normal_prev, const double *phys) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!id1 || !id2 || !shear_force || !normal_prev || !phys)))
    return fail(s, DEM_ERR_INVALID_ARG, "null contact arrays");
  const long long N = s->N;
  for (long long k = 0; k < n; ++k) {
    if (id2[k] < 0 || id2[k] >= N || id1[k] >= id2[k] || id1[k] < -6)
      return fail(s, DEM_ERR_OUT_OF_RANGE, "contact id out of range or not canonical");
    if (id1[k] < 0 && (!s->has_walls || !(s->desc.wall_mask & (1 << (-id1[k] - 1)))))
      return fail(s, DEM_ERR_INVALID_ARG, "wall contact with a wall the scene does not have");
    if (k > 0 && (id1[k - 1] > id1[k] || (id1[k - 1] == id1[k] && id2[k - 1] >= id2[k])))
      return fail(s, DEM_ERR_INVALID_ARG, "contacts must be sorted by (id1, id2) without repeats");
    for (int q = 0; q < 3; ++q)
      if (!std::isfinite(shear_force[3 * k + q]) || !std::isfinite(normal_prev[3 * k + q]) ||
          !std::isfinite(phys[3 * k + q]))
        return fail(s, DEM_ERR_NONFINITE, "non-finite contact history");
    if (cell_dist)
      for (int q = 0; q < 3; ++q)
        if (std::abs(cell_dist[3 * k + q]) > kShiftMax)
          return fail(s, DEM_ERR_CAPACITY, "cell shift beyond +-511");
  }
  dem_status r;
  if ((r = sync_host(s))) return r;
  std::vector<int> sid;
  if ((r = fetch_sid(s, sid))) return r;
  struct Row { int a, b, cp; double4_32a fs, hn; double tp; };
  std::vector<Row> rows;
  std::vector<uint8_t> flags(N);
  std::vector<double4_32a> wh;
  if (N > 0) CK(cudaMemcpyAsync(flags.data(), s->cur.flags, N, cudaMemcpyDeviceToHost, s->st));
  if ((r = wait(s))) return r;
  if (s->has_walls) wh.assign(6 * N, make_double4_32a(0, 0, 0, 0));
  for (long long sl = 0; sl < N; ++sl) flags[sl] &= 1;
  for (long long k = 0; k < n; ++k) {
    const double *f = shear_force + 3 * k, *nn = normal_prev + 3 * k, *ph = phys + 3 * k;
    if (id1[k] < 0) {
      int w = -id1[k] - 1, ax = w >> 1;
      int sl = sid[id2[k]];
      double sn = nn[ax] >= 0 ? 1.0 : -1.0;
      wh[w * N + sl] = make_double4_32a(f[0], f[1], f[2], sn);
      flags[sl] |= (2 << w);
      continue;
    }
    // rows are oriented by id (body 1 = id1 < id2), as the collider orients them
    const int a = sid[id1[k]], b = sid[id2[k]];
    int c[3] = {0, 0, 0};
    if (cell_dist) for (int q = 0; q < 3; ++q) c[q] = cell_dist[3 * k + q];
    const double sg = 1.0;
    rows.push_back(Row{a, b, pack_shift(c[0], c[1], c[2]),
                       make_double4_32a(sg * f[0], sg * f[1], sg * f[2], ph[0]),
                       make_double4_32a(sg * nn[0], sg * nn[1], sg * nn[2], ph[1]), ph[2]});
  }
  std::sort(rows.begin(), rows.end(), [](const Row &x, const Row &y) {
    return x.a != y.a ? x.a < y.a : x.b < y.b;
  });
  const long long P = (long long)rows.size();
  Table &t = s->tab[s->tc];
  if ((r = ensure_table(s, t, std::max<long long>(P, 1), N))) return r;
  std::vector<int2> pair(P);
  std::vector<int> cp(P), rs(N + 1, 0);
  std::vector<double4_32a> hfs(P), hn(P);
  std::vector<double> tp(P);
  for (long long k = 0; k < P; ++k) {
    pair[k] = make_int2(rows[k].a, rows[k].b);
    cp[k] = rows[k].cp;
    hfs[k] = rows[k].fs;
    hn[k] = rows[k].hn;
    tp[k] = rows[k].tp;
    rs[rows[k].a + 1] += 1;
  }
  for (long long i = 0; i < N; ++i) rs[i + 1] += rs[i];
  std::vector<float4> g32, hn32;
  if (s->mixed) {   // history layout of the mixed table: hfs = (Fs, tan(phi)), hn32, g32.w = kn
    g32.resize(P);
    hn32.resize(P);
    for (long long k = 0; k < P; ++k) {
      g32[k] = make_float4(0, 0, 0, (float)hfs[k].w);
      hn32[k] = make_float4((float)hn[k].x, (float)hn[k].y, (float)hn[k].z, (float)hn[k].w);
      hfs[k].w = tp[k];
    }
  }
  if (P > 0) {
    CK(cudaMemcpyAsync(t.pair, pair.data(), sizeof(int2) * P, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(t.cpack, cp.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(t.hfs, hfs.data(), sizeof(double4_32a) * P, cudaMemcpyHostToDevice, s->st));
    if (s->mixed) {
      CK(cudaMemcpyAsync(t.g32, g32.data(), sizeof(float4) * P, cudaMemcpyHostToDevice, s->st));
      CK(cudaMemcpyAsync(t.hn32, hn32.data(), sizeof(float4) * P, cudaMemcpyHostToDevice, s->st));
    } else {
      CK(cudaMemcpyAsync(t.hn, hn.data(), sizeof(double4_32a) * P, cudaMemcpyHostToDevice, s->st));
      CK(cudaMemcpyAsync(t.tanphi, tp.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s->st));
    }
  }
  CK(cudaMemcpyAsync(t.row_start, rs.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, s->st));
  t.P = P;
  s->tab_nbody[s->tc] = N;
  s->table_fresh = false;
  if (N > 0) CK(cudaMemcpyAsync(s->cur.flags, flags.data(), N, cudaMemcpyHostToDevice, s->st));
  if (s->has_walls)
    for (int w = 0; w < 6; ++w)
      CK(cudaMemcpyAsync(s->cur.whist + w * s->cap, wh.data() + w * N, sizeof(double4_32a) * N,
                         cudaMemcpyHostToDevice, s->st));
  s->need_rebuild = true;
  s->check_lost = false;
  return wait(s);
}

dem_status dem_set_timing(dem_scene *s, int enable) {
  if (!s) return DEM_ERR_INVALID_ARG;
  dem_status r;
  if ((r = sync_host(s))) return r;
  if (enable && s->tev.empty()) {
    s->tev.resize(2 + 6 * 64);
    for (auto &e : s->tev) CK(cudaEventCreate(&e));
  }
  s->timing = enable != 0;
  long long keep = s->launches;
  s->tm = dem_timing{};
  s->tm.kernel_launches = keep;
  return DEM_OK;
}

dem_status dem_get_timing(dem_scene *s, dem_timing *out) {
  if (!s || !out) return DEM_ERR_INVALID_ARG;
  dem_status r;
  if ((r = sync_host(s))) return r;
  *out = s->tm;
  out->kernel_launches = s->launches;
  return DEM_OK;
}

namespace {
Bodies body_view(const Bodies &b, long long o) {
  Bodies v = b;
  auto sh = [o](auto *&p, long long k = 1) { if (p) p += k * o; };
  sh(v.pos); sh(v.vel); sh(v.angvel); sh(v.ori); sh(v.xref); sh(v.mprop);
  sh(v.id); sh(v.sid); sh(v.mat); sh(v.flags); sh(v.whist); sh(v.rdsc);
  sh(v.p32); sh(v.vw32, 2); sh(v.xref32); sh(v.mprop32); sh(v.ori32);
  return v;
}
Table row_view(const Table &t, long long o, long long P) {
  Table v = t;
  auto sh = [o](auto *&p) { if (p) p += o; };
  sh(v.pair); sh(v.cpack); sh(v.hfs); sh(v.hn); sh(v.tanphi);
  if (v.oFM) v.oFM += 2 * o;
  if (v.oFM32) v.oFM32 += 2 * o;
  sh(v.g32); sh(v.hn32); sh(v.found); sh(v.s0);
  v.P = P;
  return v;
}

// Statistics of sub-scene q (q < 0: of the whole scene, geometry of sub-scene 0).
dem_status stats_of(dem_scene *s, int q, dem_stats *o) {
  dem_status r;
  if ((r = sync_host(s))) return r;
  std::memset(o, 0, sizeof *o);
  const Sub &u = s->subs[q < 0 ? 0 : q];
  o->iter = u.cs.iter;
  o->time = u.cs.time;
  o->dt = u.cs.dt;
  o->n_rebuilds = s->n_rebuilds;
  long long b0 = 0, nb_ = s->N;
  double vsolid = 0;
  for (const Sub &v : s->subs) vsolid += v.used ? v.vsolid : 0;
  if (q >= 0) { b0 = u.slot0; nb_ = u.n; vsolid = u.vsolid; }
  o->n_bodies = nb_;
  double V;
  if (u.cs.periodic) V = std::fabs(m_det(u.cs.H));
  else V = (u.cs.box_hi[0] - u.cs.box_lo[0]) * (u.cs.box_hi[1] - u.cs.box_lo[1]) *
           (u.cs.box_hi[2] - u.cs.box_lo[2]);
  o->packing_fraction = V > 0 ? vsolid / V : 0;
  if (nb_ == 0) return DEM_OK;
  const bool have_table = s->table_fresh;
  const Table &t = s->tab[s->tc];
  const SceneConst sc = scene_const(s);
  long long r0 = 0, r1 = have_table ? t.P : 0;
  if (q >= 0 && have_table) {   // rows whose first body is in the sub-scene
    CK(cudaMemcpyAsync(&s->rb_h->totals[0], t.row_start + b0, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    CK(cudaMemcpyAsync(&s->rb_h->totals[1], t.row_start + b0 + nb_, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    if ((r = wait(s))) return r;
    r0 = s->rb_h->totals[0];
    r1 = s->rb_h->totals[1];
  }
  o->n_candidates = r1 - r0;
  double *ph = s->partials_h;
  // bodies: kinetic energy, |F| of free bodies
  if (have_table)
    launch_gather_forces(s->cur, t, s->mats_d, s->cs_d, sc, s->cap, s->gF, s->gT, s->mixed, s->st);
  else CK(cudaMemsetAsync(s->gF, 0, sizeof(double4_32a) * s->N, s->st));
  const Bodies bv = body_view(s->cur, b0);
  int nb = stats_blocks(nb_);
  launch_body_stats(bv, s->gF + b0, nb_, s->partials, s->st);
  CK(cudaMemcpyAsync(ph, s->partials, sizeof(double) * 3 * nb, cudaMemcpyDeviceToHost, s->st));
  if ((r = wait(s))) return r;
  double ke = 0, sumF = 0, ndyn = 0;
  for (int b = 0; b < nb; ++b) { ke += ph[3 * b]; sumF += ph[3 * b + 1]; ndyn += ph[3 * b + 2]; }
  double nc = 0, sumC = 0, sig[9] = {0};
  if (have_table && r1 > r0) {
    const Table tv = row_view(t, r0, r1 - r0);
    int nr = stats_blocks(tv.P);
    launch_row_stats(tv, bv, s->partials, s->mixed, s->st);
    CK(cudaMemcpyAsync(ph, s->partials, sizeof(double) * 11 * nr, cudaMemcpyDeviceToHost, s->st));
    if ((r = wait(s))) return r;
    for (int b = 0; b < nr; ++b) {
      nc += ph[11 * b];
      sumC += ph[11 * b + 1];
      for (int k = 0; k < 9; ++k) sig[k] += ph[11 * b + 2 + k];
    }
  }
  double nw = 0, sumW = 0;
  if (s->has_walls) {
    SceneConst sv = sc;
    sv.N = nb_;
    launch_wall_stats(bv, sv, s->mats_d, s->cap, s->partials, s->st);
    CK(cudaMemcpyAsync(ph, s->partials, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, s->st));
    if ((r = wait(s))) return r;
    for (int b = 0; b < nb; ++b) { nw += ph[2 * b]; sumW += ph[2 * b + 1]; }
  }
  o->kinetic_energy = ke;
  o->n_contacts = (long long)nc;
  o->n_wall_contacts = (long long)nw;
  const double call = nc + nw;
  o->unbalanced_force = (call > 0 && ndyn > 0) ? (sumF / ndyn) / ((sumC + sumW) / call) : NAN;
  o->coordination = 2.0 * nc / nb_;
  for (int k = 0; k < 9; ++k) o->stress[k] = V > 0 ? sig[k] / V : 0;
  return DEM_OK;
}
}  // namespace

dem_status dem_get_stats(dem_scene *s, dem_stats *o) {
  if (!s || !o) return DEM_ERR_INVALID_ARG;
  return stats_of(s, -1, o);
}

}  // extern "C"

// ------------------------------------------------------------------ launch shapes
namespace {
bool valid_tuning(const dem_tuning &t) {
  return (t.contact_block == 128 || t.contact_block == 256) && t.contact_blocks_per_sm >= 1 &&
         t.contact_blocks_per_sm <= 64 &&
         (t.integrate_block == 128 || t.integrate_block == 256 || t.integrate_block == 512) &&
         (t.degree_order == 0 || t.degree_order == 1) && t.step_graphs >= -1 && t.step_graphs <= 1;
}
void apply_tuning(dem_scene *s, const dem_tuning &t) {
  s->contact_block = t.contact_block;
  s->contact_per_sm = t.contact_blocks_per_sm;
  s->integrate_block = t.integrate_block;
  s->degree_order = t.degree_order;
  s->step_graphs = t.step_graphs;
}
dem_tuning current_tuning(const dem_scene *s) {
  dem_tuning t{};
  t.contact_block = s->contact_block;
  t.contact_blocks_per_sm = s->contact_per_sm;
  t.integrate_block = s->integrate_block;
  t.degree_order = s->degree_order;
  t.step_graphs = s->step_graphs;
  return t;
}
}  // namespace

dem_status dem_set_tuning(dem_scene *s, const dem_tuning *t) {
  if (!s || !t) return DEM_ERR_INVALID_ARG;
  if (!valid_tuning(*t)) return fail(s, DEM_ERR_INVALID_ARG, "launch shape out of range");
  apply_tuning(s, *t);
  return DEM_OK;
}

dem_status dem_get_tuning(const dem_scene *s, dem_tuning *t) {
  if (!s || !t) return DEM_ERR_INVALID_ARG;
  *t = current_tuning(s);
  return DEM_OK;
}

// Coordinate search over the launch shapes, timed on the scene's own steps: first
// the contact kernel's (block, persistent grid) with the integrator fixed, then the
// integrator's (block, body order) with the best contact shape.  Each trial runs
// one untimed step, then `steps` timed steps; its cost is the contact plus
// integrator kernel time per completed step (collider runs excluded).
dem_status dem_autotune(dem_scene *s, long long steps, dem_tuning *chosen) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (steps < 1) return fail(s, DEM_ERR_INVALID_ARG, "autotune needs at least one step per trial");
  dem_status r;
  const bool was_timing = s->timing;
  const dem_timing keep_tm = s->tm;
  // The scene keeps evolving while the trials run (a compaction gains rows from one
  // trial to the next), so the contact time is taken per row processed and scaled to
  // the rows of the first trial, and each contact shape is timed twice, in two passes
  // over the list, keeping its better time.
  double rows_ref = 0;
  auto trial = [&](const dem_tuning &t, double &cost) -> dem_status {
    apply_tuning(s, t);
    dem_status q;
    if ((q = dem_step(s, 1))) return q;
    if ((q = dem_set_timing(s, 1))) return q;
    const long long it0 = s->cs0().iter;
    if ((q = dem_step(s, steps))) return q;
    const long long done = std::max<long long>(s->cs0().iter - it0, 1);
    const double rows = (double)s->tm.rows_processed;
    if (rows_ref == 0) rows_ref = rows / (double)done;
    const double contact = rows > 0 ? s->tm.contact_ms / rows * rows_ref : 0.0;
    cost = contact + s->tm.integrate_ms / (double)done;
    return DEM_OK;
  };
  dem_tuning best = current_tuning(s);
  double best_cost = INFINITY;
  const int cblocks[2] = {128, 256};
  const int per_sm[3] = {4, 8, 16};
  double shape_cost[2][3];
  for (int pass = 0; pass < 2; ++pass)
    for (int ib = 0; ib < 2; ++ib)
      for (int ip = 0; ip < 3; ++ip) {
        dem_tuning t = current_tuning(s);
        t.contact_block = cblocks[ib];
        t.contact_blocks_per_sm = per_sm[ip] * (256 / cblocks[ib]);
        double c;
        if ((r = trial(t, c))) return r;
        shape_cost[ib][ip] = pass ? std::min(shape_cost[ib][ip], c) : c;
        if (pass && shape_cost[ib][ip] < best_cost) { best_cost = shape_cost[ib][ip]; best = t; }
      }
  const int iblocks[3] = {128, 256, 512};
  const dem_tuning base = best;
  for (int b : iblocks)
    for (int o = 0; o < 2; ++o) {
      dem_tuning t = base;
      t.integrate_block = b;
      t.degree_order = o;
      if (t.integrate_block == base.integrate_block && t.degree_order == base.degree_order) continue;
      double c;
      if ((r = trial(t, c))) return r;
      if (c < best_cost) { best_cost = c; best = t; }
    }
  apply_tuning(s, best);
  if ((r = dem_set_timing(s, was_timing ? 1 : 0))) return r;
  if (was_timing) {
    const long long kl = s->tm.kernel_launches;
    s->tm = keep_tm;
    s->tm.kernel_launches = kl;
  }
  if (chosen) *chosen = best;
  return DEM_OK;
}

// ------------------------------------------------------------------ sub-scenes
void dem_subscene_desc_init(dem_subscene_desc *d) {
  if (!d) return;
  std::memset(d, 0, sizeof *d);
  for (int q = 0; q < 9; ++q) d->cell_h[q] = (q % 4 == 0) ? 1.0 : 0.0;
  for (int k = 0; k < 3; ++k) { d->box_lo[k] = 0; d->box_hi[k] = 1; }
  d->damping = 0.2;
  d->verlet_dist = -0.5;
}

dem_status dem_add_subscene(dem_scene *s, const dem_subscene_desc *d, int *sub) {
  if (!s || !d || !sub) return DEM_ERR_INVALID_ARG;
  if (!(d->damping >= 0) || !(d->damping < 1) || !(d->dt >= 0) || !std::isfinite(d->dt) ||
      !std::isfinite(d->verlet_dist))
    return fail(s, DEM_ERR_INVALID_ARG, "bad damping, dt or verlet_dist");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(d->gravity[k]) || !std::isfinite(d->box_lo[k]) || !std::isfinite(d->box_hi[k]))
      return fail(s, DEM_ERR_INVALID_ARG, "non-finite gravity or box");
  if (d->periodic) {
    if (!(m_det(d->cell_h) > 0) || !(d->cell_h[0] > 0) || !(d->cell_h[4] > 0) || !(d->cell_h[8] > 0))
      return fail(s, DEM_ERR_INVALID_ARG,
                  "the periodic cell needs a positive determinant and positive diagonal");
  } else if (d->wall_mask & 0x3F) {
    for (int k = 0; k < 3; ++k)
      if (!(d->box_hi[k] > d->box_lo[k])) return fail(s, DEM_ERR_INVALID_ARG, "box_hi must exceed box_lo");
  }
  const int wm = d->periodic ? 0 : (d->wall_mask & 0x3F);
  if (wm && (d->wall_material < 0 || d->wall_material >= kMaxMat || !s->mat_set[d->wall_material]))
    return fail(s, DEM_ERR_INVALID_ARG, "unknown wall material (set_material first)");
  if (s->cs0().triax || s->p3d_on)
    return fail(s, DEM_ERR_UNSUPPORTED, "a scene running a cell controller takes no sub-scenes");
  dem_status r;
  if ((r = sync_host(s))) return r;
  int q = -1;
  for (int i = 0; i < s->nsub(); ++i)
    if (!s->subs[i].used && !s->subs[i].removing) { q = i; break; }
  if (q < 0) {
    if ((r = ensure_subs(s, s->nsub() + 1))) return r;
    s->subs.emplace_back();
    q = s->nsub() - 1;
  }
  Sub &u = s->subs[q];
  u = Sub{};
  u.used = true;
  u.verlet_rule = d->verlet_dist;
  init_cell(u.cs, d->periodic, d->cell_h, d->box_lo, d->box_hi, wm, d->wall_material, d->gravity,
            d->damping);
  u.dt_set = d->dt > 0;
  u.cs.dt = d->dt;
  u.id0 = s->N;
  if (wm) s->has_walls = true;
  s->cs_dirty = true;
  s->need_rebuild = true;
  *sub = q;
  return DEM_OK;
}

dem_status dem_add_spheres_to(dem_scene *s, int sub, long long n, const double *pos,
                              const double *radius, const int *mat, const double *vel,
                              const double *angvel, const unsigned char *fixed, long long *first_id) {
  if (!s) return DEM_ERR_INVALID_ARG;
  return add_spheres_sub(s, sub, n, pos, radius, mat, vel, angvel, fixed, first_id);
}

dem_status dem_remove_subscene(dem_scene *s, int sub) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (sub < 0 || sub >= s->nsub() || !s->subs[sub].used || s->subs[sub].removing)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  dem_status r;
  if ((r = sync_host(s))) return r;
  Sub &u = s->subs[sub];
  u.removing = true;
  u.used = false;
  u.cs.alive = 0;
  s->cs_dirty = true;
  s->need_rebuild = true;
  s->layout_dirty = true;
  s->table_fresh = false;
  return DEM_OK;
}

dem_status dem_get_subscene(dem_scene *s, int sub, long long *first_id, long long *n,
                            long long *iter, double *time, double *dt) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (sub < 0 || sub >= s->nsub() || !s->subs[sub].used)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  dem_status r;
  if ((r = sync_host(s))) return r;
  if ((r = ensure_dt(s)) && s->N > 0) return r;
  const Sub &u = s->subs[sub];
  if (first_id) *first_id = u.id0;
  if (n) *n = u.n;
  if (iter) *iter = u.cs.iter;
  if (time) *time = u.cs.time;
  if (dt) *dt = u.cs.dt;
  return DEM_OK;
}

dem_status dem_get_subscene_stats(dem_scene *s, int sub, dem_stats *out) {
  if (!s || !out) return DEM_ERR_INVALID_ARG;
  if (sub < 0 || sub >= s->nsub() || !s->subs[sub].used)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  if (s->layout_dirty && s->subs[sub].n > 0)
    return fail(s, DEM_ERR_STATE, "sub-scene layout changed since the last step: step first");
  return stats_of(s, sub, out);
}

dem_status dem_set_subscene_velgrad(dem_scene *s, int sub, const double *L) {
  if (!s || !L) return DEM_ERR_INVALID_ARG;
  if (sub < 0 || sub >= s->nsub() || !s->subs[sub].used)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  Sub &u = s->subs[sub];
  if (!u.cs.periodic) return fail(s, DEM_ERR_STATE, "velGrad needs a periodic sub-scene");
  for (int q = 0; q < 9; ++q)
    if (!std::isfinite(L[q])) return fail(s, DEM_ERR_INVALID_ARG, "non-finite velGrad");
  std::memcpy(u.velgrad_next, L, sizeof u.velgrad_next);
  u.velgrad_pending = true;
  return DEM_OK;
}

dem_status dem_flip_cell(dem_scene *s, int sub, const int *flip, int *applied) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (sub < 0 || sub >= s->nsub() || !s->subs[sub].used)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  dem_status r;
  if ((r = sync_host(s))) return r;
  Sub &u = s->subs[sub];
  CellState &c = u.cs;
  if (!c.periodic) return fail(s, DEM_ERR_STATE, "a cell flip needs a periodic (sub-)scene");
  // M = I + K: the caller's K, or column reductions of the current H
  long long M[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  if (flip) {
    for (int q = 0; q < 9; ++q) {
      if (flip[q] < -1000 || flip[q] > 1000) return fail(s, DEM_ERR_INVALID_ARG, "flip entries beyond +-1000");
      M[q] += flip[q];
    }
  } else {
    double h[9];
    std::memcpy(h, c.H, sizeof h);
    const int pairs[6][2] = {{1, 2}, {0, 2}, {0, 1}, {1, 0}, {2, 0}, {2, 1}};
    for (const auto &pr : pairs) {
      const int i = pr[0], j = pr[1];   // column j against column i, on row i
      const double k = std::floor(h[3 * i + j] / h[3 * i + i] + 0.5);
      if (k == 0.0 || !(h[3 * j + j] - k * h[3 * j + i] > 0.0)) continue;
      for (int row = 0; row < 3; ++row) {
        h[3 * row + j] -= k * h[3 * row + i];
        M[3 * row + j] -= (long long)k * M[3 * row + i];
      }
    }
  }
  const long long det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                        M[2] * (M[3] * M[7] - M[4] * M[6]);
  if (det != 1) return fail(s, DEM_ERR_INVALID_ARG, "a cell flip needs det(I + flip) = 1");
  // adjugate = inverse (det 1)
  const long long Ai[9] = {M[4] * M[8] - M[5] * M[7], M[2] * M[7] - M[1] * M[8], M[1] * M[5] - M[2] * M[4],
                           M[5] * M[6] - M[3] * M[8], M[0] * M[8] - M[2] * M[6], M[2] * M[3] - M[0] * M[5],
                           M[3] * M[7] - M[4] * M[6], M[1] * M[6] - M[0] * M[7], M[0] * M[4] - M[1] * M[3]};
  double Md[9], Hn[9];
  int Mi[9];
  bool ident = true;
  for (int q = 0; q < 9; ++q) {
    Md[q] = (double)M[q];
    if (Ai[q] < -(1 << 20) || Ai[q] > (1 << 20))
      return fail(s, DEM_ERR_INVALID_ARG, "flip inverse entries too large");
    Mi[q] = (int)Ai[q];
    ident &= M[q] == ((q % 4 == 0) ? 1 : 0);
  }
  m_mul(c.H, Md, Hn);
  if (!(Hn[0] > 0 && Hn[4] > 0 && Hn[8] > 0))
    return fail(s, DEM_ERR_INVALID_ARG, "the flipped cell needs a positive diagonal");
  if (!ident) {
    // rows keep their images: c' = M^-1 c (checked for range before any is changed)
    const Table &t = s->tab[s->tc];
    if (t.P > 0 && t.row_start != nullptr && s->N > 0) {
      const int multi = s->nsub() > 1;
      int *maxabs = s->deg_ws;
      CK(cudaMemsetAsync(maxabs, 0, sizeof(int), s->st));
      launch_flip_shift(t, s->cur.sid, multi, sub, Mi, maxabs, 0, s->st);
      int worst = 0;
      CK(cudaMemcpyAsync(&s->rb_h->totals[0], maxabs, sizeof(int), cudaMemcpyDeviceToHost, s->st));
      if ((r = wait(s))) return r;
      worst = s->rb_h->totals[0];
      if (worst > kShiftMax)
        return fail(s, DEM_ERR_GEOMETRY, "a cell flip would move an image shift out of range");
      launch_flip_shift(t, s->cur.sid, multi, sub, Mi, maxabs, 1, s->st);
      CK(cudaGetLastError());
    }
    double Hp[9], Hr[9], Hri[9];
    m_mul(c.Hprev, Md, Hp);
    m_mul(c.Href, Md, Hr);
    double Mid[9];
    for (int q = 0; q < 9; ++q) Mid[q] = (double)Mi[q];
    m_mul(Mid, c.Hrefinv, Hri);
    std::memcpy(c.H, Hn, sizeof Hn);
    std::memcpy(c.Hprev, Hp, sizeof Hp);
    std::memcpy(c.Href, Hr, sizeof Hr);
    std::memcpy(c.Hrefinv, Hri, sizeof Hri);
    cell_derive(c);
    s->need_rebuild = true;   // the collider re-initialises on the new cell
    s->cs_dirty = true;
  }
  if (applied)
    for (int q = 0; q < 9; ++q) applied[q] = (int)(M[q] - ((q % 4 == 0) ? 1 : 0));
  return DEM_OK;
}

dem_status dem_num_bodies(dem_scene *s, long long *n) {
  if (!s || !n) return DEM_ERR_INVALID_ARG;
  *n = s->N;
  return DEM_OK;
}

dem_status dem_get_state_range(dem_scene *s, long long first_id, long long n, double *pos,
                               double *vel, double *angvel, double *ori) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (first_id < 0 || n < 0 || first_id + n > s->N)
    return fail(s, DEM_ERR_OUT_OF_RANGE, "id range outside [0, number of bodies)");
  dem_status r;
  if ((r = sync_host(s))) return r;
  if (n == 0) return DEM_OK;
  std::vector<double4_32a> h(n);
  auto get = [&](const double4_32a *src, double *out, int comps) -> dem_status {
    launch_gather_ids(s->slot_of_id + first_id, n, src, s->gT, s->st);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h.data(), s->gT, sizeof(double4_32a) * n, cudaMemcpyDeviceToHost, s->st));
    dem_status q = wait(s);
    if (q) return q;
    for (long long i = 0; i < n; ++i) {
      const double c[4] = {h[i].x, h[i].y, h[i].z, h[i].w};
      for (int k = 0; k < comps; ++k) out[comps * i + k] = c[k];
    }
    return DEM_OK;
  };
  if (pos && (r = get(s->cur.pos, pos, 3))) return r;
  if (vel && (r = get(s->cur.vel, vel, 3))) return r;
  if (angvel && (r = get(s->cur.angvel, angvel, 3))) return r;
  if (ori) {
    if (s->mixed) {
      std::vector<float4> f(n);
      launch_gather_ids_f(s->slot_of_id + first_id, n, s->cur.ori32, reinterpret_cast<float4 *>(s->gT),
                          s->st);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(f.data(), s->gT, sizeof(float4) * n, cudaMemcpyDeviceToHost, s->st));
      if ((r = wait(s))) return r;
      for (long long i = 0; i < n; ++i) {
        ori[4 * i] = f[i].x; ori[4 * i + 1] = f[i].y; ori[4 * i + 2] = f[i].z; ori[4 * i + 3] = f[i].w;
      }
    } else if ((r = get(s->cur.ori, ori, 4))) {
      return r;
    }
  }
  return DEM_OK;
}

// ------------------------------------------------------------------ micromechanics
dem_status dem_get_micro(dem_scene *s, int sub, double *fabric, double *normal_stress,
                         double *shear_stress, long long *n_contacts) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (sub >= s->nsub() || (sub >= 0 && !s->subs[sub].used))
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  if (sub >= 0 && s->layout_dirty && s->subs[sub].n > 0)
    return fail(s, DEM_ERR_STATE, "sub-scene layout changed since the last step: step first");
  dem_status r;
  if ((r = sync_host(s))) return r;
  const Sub &u = s->subs[sub < 0 ? 0 : sub];
  double V;
  if (u.cs.periodic) V = std::fabs(m_det(u.cs.H));
  else V = (u.cs.box_hi[0] - u.cs.box_lo[0]) * (u.cs.box_hi[1] - u.cs.box_lo[1]) *
           (u.cs.box_hi[2] - u.cs.box_lo[2]);
  double acc[28] = {0};
  if (s->table_fresh && s->N > 0) {
    const Table &t = s->tab[s->tc];
    long long r0 = 0, r1 = t.P;
    if (sub >= 0) {
      CK(cudaMemcpyAsync(&s->rb_h->totals[0], t.row_start + u.slot0, sizeof(int), cudaMemcpyDeviceToHost, s->st));
      CK(cudaMemcpyAsync(&s->rb_h->totals[1], t.row_start + u.slot0 + u.n, sizeof(int), cudaMemcpyDeviceToHost, s->st));
      if ((r = wait(s))) return r;
      r0 = s->rb_h->totals[0];
      r1 = s->rb_h->totals[1];
    }
    if (r1 > r0) {
      const Table tv = row_view(t, r0, r1 - r0);
      const int nb = micro_blocks(tv.P);
      launch_micro_rows(tv, s->mixed, s->partials, s->st);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(s->partials_h, s->partials, sizeof(double) * 28 * nb, cudaMemcpyDeviceToHost, s->st));
      if ((r = wait(s))) return r;
      for (int b = 0; b < nb; ++b)
        for (int q = 0; q < 28; ++q) acc[q] += s->partials_h[28 * b + q];
    }
  }
  const double nc = acc[0];
  for (int q = 0; q < 9; ++q) {
    if (fabric) fabric[q] = nc > 0 ? acc[1 + q] / nc : 0.0;
    if (normal_stress) normal_stress[q] = V > 0 ? -acc[10 + q] / V : 0.0;
    if (shear_stress) shear_stress[q] = V > 0 ? -acc[19 + q] / V : 0.0;
  }
  if (n_contacts) *n_contacts = (long long)nc;
  return DEM_OK;
}

dem_status dem_get_body_stress(dem_scene *s, double *out) {
  if (!s || !out) return DEM_ERR_INVALID_ARG;
  dem_status r;
  if ((r = sync_host(s))) return r;
  const long long N = s->N;
  if (N == 0) return DEM_OK;
  if (!s->table_fresh) {   // no contacts computed for the current layout yet
    std::memset(out, 0, sizeof(double) * 9 * N);
    return DEM_OK;
  }
  double *dev = nullptr;
  if ((r = dalloc(s, &dev, 9 * N))) return r;
  const SceneConst sc = scene_const(s);
  launch_body_stress(s->cur, s->tab[s->tc], N, s->cap, s->mixed, sc.walls, sc.multi, s->cs_d,
                     s->mats_d, dev, s->st);
  CK(cudaGetLastError());
  std::vector<double> h(9 * N);
  std::vector<int> slot(N);
  CK(cudaMemcpyAsync(h.data(), dev, sizeof(double) * 9 * N, cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemcpyAsync(slot.data(), s->slot_of_id, sizeof(int) * N, cudaMemcpyDeviceToHost, s->st));
  dfree(s, dev);
  if ((r = wait(s))) return r;
  for (long long i = 0; i < N; ++i)
    std::memcpy(out + 9 * i, h.data() + 9 * (long long)slot[i], sizeof(double) * 9);
  return DEM_OK;
}

// ------------------------------------------------------------------ time stepper
dem_status dem_set_timestepper(dem_scene *s, int sub, double safety, int interval,
                               double default_dt, double max_dt) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (sub < 0 || sub >= s->nsub() || !s->subs[sub].used)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  if (!(safety > 0) || !(safety <= 1) || interval < 1 || !std::isfinite(default_dt) ||
      !std::isfinite(max_dt))
    return fail(s, DEM_ERR_INVALID_ARG, "bad time-stepper parameters");
  dem_status r;
  if ((r = sync_host(s))) return r;
  Sub &u = s->subs[sub];
  u.cs.tstep = 1;
  u.cs.tstep_safety = safety;
  u.cs.tstep_interval = interval;
  u.cs.tstep_max = max_dt;
  u.tstep_default_rule = default_dt;
  u.tstep_default_n = -1;
  if (default_dt > 0) u.cs.tstep_default = default_dt;
  s->cs_dirty = true;
  return DEM_OK;
}

dem_status dem_set_density_scaling(dem_scene *s, int sub, int enable, double target_dt) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (sub < 0 || sub >= s->nsub() || !s->subs[sub].used)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  if (enable && !(std::isfinite(target_dt) && target_dt > 0))
    return fail(s, DEM_ERR_INVALID_ARG, "density scaling needs a finite target_dt > 0");
  dem_status r;
  if ((r = sync_host(s))) return r;
  Sub &u = s->subs[sub];
  if (enable && !u.cs.tstep)
    return fail(s, DEM_ERR_STATE, "density scaling needs the time stepper (dem_set_timestepper)");
  if (!enable && u.cs.dscale) {
    launch_dscale_reset(s->cur, s->N, s->nsub() > 1, sub, s->st);
    CK(cudaGetLastError());
  }
  u.cs.dscale = enable ? 1 : 0;
  u.cs.target_dt = enable ? target_dt : 0.0;
  s->cs_dirty = true;
  return DEM_OK;
}

dem_status dem_get_density_scaling(dem_scene *s, double *f) {
  if (!s || !f) return DEM_ERR_INVALID_ARG;
  dem_status r;
  if ((r = sync_host(s))) return r;
  const long long N = s->N;
  if (N == 0) return DEM_OK;
  std::vector<int> sid;
  if ((r = fetch_sid(s, sid))) return r;
  std::vector<double> h(N);
  CK(cudaMemcpyAsync(h.data(), s->cur.rdsc, sizeof(double) * N, cudaMemcpyDeviceToHost, s->st));
  if ((r = wait(s))) return r;
  for (long long i = 0; i < N; ++i) f[i] = 1.0 / h[sid[i]];
  return DEM_OK;
}

// ------------------------------------------------------------------ contact law
dem_status dem_set_law(dem_scene *s, int sub, int law) {
  if (!s) return DEM_ERR_INVALID_ARG;
  if (sub < 0 || sub >= s->nsub() || !s->subs[sub].used)
    return fail(s, DEM_ERR_INVALID_ARG, "no such sub-scene");
  if (law != DEM_LAW_LINEAR && law != DEM_LAW_HERTZ_MINDLIN)
    return fail(s, DEM_ERR_INVALID_ARG, "unknown contact law");
  dem_status r;
  if ((r = sync_host(s))) return r;
  Sub &u = s->subs[sub];
  if (u.cs.iter != 0 && u.cs.law != law)
    return fail(s, DEM_ERR_STATE, "the contact law is chosen before the sub-scene's first step");
  u.cs.law = law;
  s->cs_dirty = true;
  return DEM_OK;
}
