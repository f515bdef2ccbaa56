// Continuous-batching server of the C ABI (dem_server_*): the scheduling core
// of server_sched.h driving one device scene through the scene API, each
// request a sub-scene.  Host code only; every step runs in the library's
// kernels.  The paper has no counterpart (it runs one scene per process): this
// is the serving pattern applied to the method's hot path.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <future>
#include <string>

#include "dem.h"
#include "dem_internal.cuh"
#include "server_sched.h"

namespace dem {
long long scene_device_bytes(const dem_scene *s);
long long scene_table_rows(const dem_scene *s);
double scene_bytes_per_body(int mixed);
double scene_bytes_per_row(int mixed);
void set_global_error(const std::string &msg);
}  // namespace dem

namespace {

using dem_sched::Req;

constexpr int kMatSlots = dem::kMaxMat;   // material ids 1 .. kMatSlots-1 go to requests
constexpr int kMaxReqMaterials = 64;

// The device side: one scene whose sub-scene 0 stays empty; a request is a
// sub-scene with its own material id range.
struct SceneBackend {
  dem_scene *scene = nullptr;
  int device = 0;
  std::vector<std::pair<int, int>> free_mats;   // (first id, count), sorted

  int alloc_mats(int k) {
    for (auto &f : free_mats)
      if (f.second >= k) {
        const int a = f.first;
        f.first += k;
        f.second -= k;
        return a;
      }
    return -1;
  }
  void free_mat_range(int a, int k) {
    free_mats.emplace_back(a, k);
    std::sort(free_mats.begin(), free_mats.end());
    std::vector<std::pair<int, int>> m;
    for (auto &f : free_mats) {
      if (!m.empty() && m.back().first + m.back().second == f.first) m.back().second += f.second;
      else if (f.second > 0) m.push_back(f);
    }
    free_mats.swap(m);
  }
  int err(int rc, std::string &msg) {
    msg = dem_last_error(scene);
    return rc;
  }

  // The collider's rule for a periodic cell (its grid needs three slabs of edge
  // 2 r_max + 2 verlet_dist across each pair of faces), checked before admission so
  // that such a request fails alone instead of failing the step of every scene.
  static int check_cell(const Req &r, const dem_subscene_desc &d, std::string &msg) {
    if (!d.periodic) return 0;
    double rmin = r.radius[0], rmax = r.radius[0];
    for (double x : r.radius) { rmin = std::min(rmin, x); rmax = std::max(rmax, x); }
    const double dl = d.verlet_dist > 0 ? d.verlet_dist : -d.verlet_dist * rmin;
    const double *H = d.cell_h;
    const double V = std::fabs(H[0] * (H[4] * H[8] - H[5] * H[7]) -
                               H[1] * (H[3] * H[8] - H[5] * H[6]) +
                               H[2] * (H[3] * H[7] - H[4] * H[6]));
    for (int k = 0; k < 3; ++k) {
      const int i = (k + 1) % 3, j = (k + 2) % 3;
      const double a[3] = {H[i], H[3 + i], H[6 + i]}, b[3] = {H[j], H[3 + j], H[6 + j]};
      const double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2],
                   cz = a[0] * b[1] - a[1] * b[0];
      const double w = V / std::sqrt(cx * cx + cy * cy + cz * cz);
      if (!(w >= 3 * (2 * rmax + 2 * dl))) {
        msg = "periodic cell width shorter than 3 * (2 r_max + 2 verlet_dist)";
        return DEM_ERR_GEOMETRY;
      }
    }
    return 0;
  }

  int admit(Req &r, std::string &msg) {
    {
      dem_subscene_desc d;
      std::memcpy(&d, r.desc.data(), sizeof d);
      if (const int rc = check_cell(r, d, msg)) return rc;
    }
    const int base = alloc_mats(r.nmat);
    if (base < 0) { msg = "material table full"; return DEM_ERR_CAPACITY; }
    int rc;
    for (int k = 0; k < r.nmat; ++k) {
      const double *m = &r.mats[4 * k];
      if ((rc = dem_set_material(scene, base + k, m[0], m[1], m[2], m[3]))) {
        free_mat_range(base, r.nmat);
        return err(rc, msg);
      }
    }
    dem_subscene_desc d;
    std::memcpy(&d, r.desc.data(), sizeof d);
    d.wall_material += base;
    int sub = -1;
    if ((rc = dem_add_subscene(scene, &d, &sub))) {
      free_mat_range(base, r.nmat);
      return err(rc, msg);
    }
    std::vector<int> mat(r.n);
    for (long long i = 0; i < r.n; ++i) mat[i] = base + r.mat[i];
    long long first = 0;
    rc = dem_add_spheres_to(scene, sub, r.n, r.pos.data(), r.radius.data(), mat.data(),
                            r.vel.empty() ? nullptr : r.vel.data(),
                            r.angvel.empty() ? nullptr : r.angvel.data(), nullptr, &first);
    if (!rc && r.has_velgrad) rc = dem_set_subscene_velgrad(scene, sub, r.velgrad);
    if (rc) {
      const int code = err(rc, msg);
      dem_remove_subscene(scene, sub);
      free_mat_range(base, r.nmat);
      return code;
    }
    r.sub = sub;
    r.mat_base = base;
    return 0;
  }
  int step(long long k, std::string &msg) {
    const int rc = dem_step(scene, k);
    return rc ? err(rc, msg) : 0;
  }
  int collect(Req &r, std::string &msg) {
    dem_stats st;
    long long first = 0, n = 0;
    int rc = dem_get_subscene_stats(scene, r.sub, &st);
    if (!rc) rc = dem_get_subscene(scene, r.sub, &first, &n, &r.iter, &r.time, &r.dt);
    if (rc) return err(rc, msg);
    r.stats.assign((sizeof st + sizeof(double) - 1) / sizeof(double), 0.0);
    std::memcpy(r.stats.data(), &st, sizeof st);
    if (r.keep_state) {
      r.out_pos.resize(3 * n);
      r.out_vel.resize(3 * n);
      r.out_angvel.resize(3 * n);
      r.out_ori.resize(4 * n);
      rc = dem_get_state_range(scene, first, n, r.out_pos.data(), r.out_vel.data(),
                               r.out_angvel.data(), r.out_ori.data());
      if (rc) return err(rc, msg);
    }
    return 0;
  }
  void remove(Req &r) {
    if (r.sub >= 0) dem_remove_subscene(scene, r.sub);
    if (r.mat_base >= 0) free_mat_range(r.mat_base, r.nmat);
    r.sub = -1;
    r.mat_base = -1;
  }
  double rows_per_body() {
    long long n = 0;
    if (dem_num_bodies(scene, &n) || n <= 0) return 0;
    return (double)dem::scene_table_rows(scene) / (double)n;
  }
  long long device_bytes() { return dem::scene_device_bytes(scene); }
  void thread_init() { cudaSetDevice(device); }
};

using Sched = dem_sched::Scheduler<SceneBackend>;

}  // namespace

struct dem_server {
  dem_server_desc desc{};
  SceneBackend be;
  std::unique_ptr<Sched> sched;
  cudaStream_t own_stream = nullptr;
  std::string err;
  std::mutex err_mu;
};

namespace {
dem_status server_fail(dem_server *s, dem_status code, const std::string &msg) {
  if (s) {
    std::lock_guard<std::mutex> lk(s->err_mu);
    s->err = msg;
  } else {
    dem::set_global_error(msg);
  }
  return code;
}
}  // namespace

extern "C" {

void dem_server_desc_init(dem_server_desc *d) {
  if (!d) return;
  std::memset(d, 0, sizeof *d);
  d->precision = DEM_MIXED;
  d->budget_bytes = 0;
  d->tick_steps = 200;
  d->rows_per_body = 8.0;
  d->cuda_stream = nullptr;
  d->device = -1;
}

dem_status dem_server_create(const dem_server_desc *desc, dem_server **out) {
  if (!desc || !out) return server_fail(nullptr, DEM_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if ((desc->precision != DEM_FP64 && desc->precision != DEM_MIXED) || desc->tick_steps < 1 ||
      desc->budget_bytes < 0 || !(desc->rows_per_body >= 0))
    return server_fail(nullptr, DEM_ERR_INVALID_ARG, "bad server descriptor");
  int dev = desc->device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return server_fail(nullptr, DEM_ERR_CUDA, "no CUDA device");
  }
  auto *s = new dem_server;
  s->desc = *desc;
  s->desc.device = dev;
  // the worker thread owns the device scene: create it there and wait for the result
  std::promise<std::pair<int, std::string>> ready;
  auto fut = ready.get_future();
  // set-up on a temporary thread with the device current (the caller's current device
  // is left alone)
  std::thread init([&] {
    std::string msg;
    if (cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      ready.set_value({DEM_ERR_CUDA, "cudaSetDevice failed"});
      return;
    }
    cudaStream_t st = (cudaStream_t)desc->cuda_stream;
    if (!st) {
      if (cudaStreamCreateWithFlags(&s->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ready.set_value({DEM_ERR_CUDA, "stream creation failed"});
        return;
      }
      st = s->own_stream;
    }
    long long budget = desc->budget_bytes;
    if (budget <= 0) {   // default: half of the device memory free now
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        ready.set_value({DEM_ERR_CUDA, "cudaMemGetInfo failed"});
        return;
      }
      budget = (long long)(fr / 2);
    }
    s->desc.budget_bytes = budget;
    dem_scene_desc sd;
    dem_scene_desc_init(&sd);
    sd.precision = desc->precision;
    sd.dt = 1.0;   // sub-scene 0 stays empty
    sd.cuda_stream = st;
    sd.device = dev;
    dem_scene *sc = nullptr;
    int rc = dem_scene_create(&sd, &sc);
    if (rc) {
      ready.set_value({rc, dem_last_error(nullptr)});
      return;
    }
    rc = dem_set_material(sc, 0, 1000.0, 1e6, 0.25, 0.5);
    if (rc) {
      std::string m = dem_last_error(sc);
      dem_scene_destroy(sc);
      ready.set_value({rc, m});
      return;
    }
    s->be.scene = sc;
    s->be.device = dev;
    s->be.free_mats = {{1, kMatSlots - 1}};
    ready.set_value({0, ""});
  });
  init.join();
  auto res = fut.get();
  if (res.first) {
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    delete s;
    return server_fail(nullptr, (dem_status)res.first, res.second);
  }
  const int mixed = desc->precision == DEM_MIXED;
  s->sched.reset(new Sched(&s->be, s->desc.budget_bytes, desc->tick_steps,
                           dem::scene_bytes_per_body(mixed), dem::scene_bytes_per_row(mixed),
                           desc->rows_per_body > 0 ? desc->rows_per_body : 8.0));
  s->sched->start();   // the worker makes the device current on its thread first
  *out = s;
  return DEM_OK;
}

void dem_server_destroy(dem_server *s) {
  if (!s) return;
  s->sched->stop();
  s->sched.reset();
  if (s->be.scene) {
    int old = 0;
    cudaGetDevice(&old);
    cudaSetDevice(s->desc.device);
    dem_scene_destroy(s->be.scene);
    if (s->own_stream) cudaStreamDestroy(s->own_stream);
    cudaSetDevice(old);
  }
  delete s;
}

void dem_request_init(dem_request *r) {
  if (!r) return;
  std::memset(r, 0, sizeof *r);
  dem_subscene_desc_init(&r->scene);
}

dem_status dem_server_submit(dem_server *s, const dem_request *q, long long *ticket) {
  if (!s || !q || !ticket) return server_fail(s, DEM_ERR_INVALID_ARG, "null argument");
  *ticket = 0;
  if (q->n < 1 || !q->pos || !q->radius || q->nsteps < 1)
    return server_fail(s, DEM_ERR_INVALID_ARG, "a request needs n >= 1 spheres and nsteps >= 1");
  if (q->n_materials < 1 || q->n_materials > kMaxReqMaterials || !q->materials)
    return server_fail(s, DEM_ERR_INVALID_ARG, "a request needs 1 to 64 materials");
  if (q->scene.wall_material < 0 || q->scene.wall_material >= q->n_materials)
    return server_fail(s, DEM_ERR_INVALID_ARG, "wall material outside the request's materials");
  std::unique_ptr<Req> r(new Req);
  r->n = q->n;
  r->nsteps = q->nsteps;
  r->nmat = q->n_materials;
  r->keep_state = q->keep_state ? 1 : 0;
  r->pos.assign(q->pos, q->pos + 3 * q->n);
  r->radius.assign(q->radius, q->radius + q->n);
  if (q->vel) r->vel.assign(q->vel, q->vel + 3 * q->n);
  if (q->angvel) r->angvel.assign(q->angvel, q->angvel + 3 * q->n);
  r->mats.assign(q->materials, q->materials + 4 * q->n_materials);
  r->mat.assign(q->n, 0);
  if (q->mat_id)
    for (long long i = 0; i < q->n; ++i) {
      if (q->mat_id[i] < 0 || q->mat_id[i] >= q->n_materials)
        return server_fail(s, DEM_ERR_INVALID_ARG, "material index outside the request's materials");
      r->mat[i] = q->mat_id[i];
    }
  r->desc.resize(sizeof(dem_subscene_desc));
  std::memcpy(r->desc.data(), &q->scene, sizeof(dem_subscene_desc));
  if (q->velgrad) {
    r->has_velgrad = true;
    std::memcpy(r->velgrad, q->velgrad, sizeof r->velgrad);
  }
  std::string msg;
  const int rc = s->sched->submit(std::move(r), ticket, msg);
  if (rc) return server_fail(s, (dem_status)rc, msg);
  return DEM_OK;
}

dem_status dem_server_poll(dem_server *s, long long ticket, int *state) {
  if (!s || !state) return server_fail(s, DEM_ERR_INVALID_ARG, "null argument");
  const int v = s->sched->poll(ticket);
  if (v < 0) return server_fail(s, DEM_ERR_INVALID_ARG, "unknown ticket");
  *state = v;
  return DEM_OK;
}

dem_status dem_server_wait(dem_server *s, long long ticket, double timeout_s) {
  if (!s) return server_fail(s, DEM_ERR_INVALID_ARG, "null argument");
  std::string msg;
  const int rc = s->sched->wait(ticket, timeout_s, msg);
  if (rc == -1) return server_fail(s, DEM_ERR_INVALID_ARG, "unknown ticket");
  if (rc == -2) return server_fail(s, DEM_ERR_TIMEOUT, "request not finished before the deadline");
  if (rc) return server_fail(s, (dem_status)rc, msg);
  return DEM_OK;
}

dem_status dem_server_result(dem_server *s, long long ticket, dem_request_result *info,
                             double *pos, double *vel, double *angvel, double *ori) {
  if (!s) return server_fail(s, DEM_ERR_INVALID_ARG, "null argument");
  int code = DEM_OK;
  std::string msg;
  const int rc = s->sched->with_result(ticket, [&](const Req &r) {
    if (r.state == dem_sched::kFailed) {
      code = r.err ? r.err : DEM_ERR_STATE;
      msg = r.msg;
      return;
    }
    if ((pos || vel || angvel || ori) && !r.keep_state) {
      code = DEM_ERR_INVALID_ARG;
      msg = "the request was submitted without keep_state";
      return;
    }
    if (info) {
      std::memset(info, 0, sizeof *info);
      info->ticket = r.ticket;
      info->n = r.n;
      info->nsteps = r.nsteps;
      info->iter = r.iter;
      info->time = r.time;
      info->dt = r.dt;
      info->t_submit = r.t_submit;
      info->t_admit = r.t_admit;
      info->t_done = r.t_done;
      info->latency = r.t_done - r.t_submit;
      std::memcpy(&info->stats, r.stats.data(), sizeof(dem_stats));
    }
    if (pos) std::memcpy(pos, r.out_pos.data(), sizeof(double) * r.out_pos.size());
    if (vel) std::memcpy(vel, r.out_vel.data(), sizeof(double) * r.out_vel.size());
    if (angvel) std::memcpy(angvel, r.out_angvel.data(), sizeof(double) * r.out_angvel.size());
    if (ori) std::memcpy(ori, r.out_ori.data(), sizeof(double) * r.out_ori.size());
  });
  if (rc == -1) return server_fail(s, DEM_ERR_INVALID_ARG, "unknown ticket");
  if (rc == -3) return server_fail(s, DEM_ERR_STATE, "request not finished");
  if (code) return server_fail(s, (dem_status)code, msg);
  return DEM_OK;
}

dem_status dem_server_release(dem_server *s, long long ticket) {
  if (!s) return server_fail(s, DEM_ERR_INVALID_ARG, "null argument");
  const int rc = s->sched->release(ticket);
  if (rc == -1) return server_fail(s, DEM_ERR_INVALID_ARG, "unknown ticket");
  if (rc == -3) return server_fail(s, DEM_ERR_STATE, "request not finished");
  return DEM_OK;
}

dem_status dem_server_stats(dem_server *s, dem_server_summary *out) {
  if (!s || !out) return server_fail(s, DEM_ERR_INVALID_ARG, "null argument");
  const dem_sched::Totals t = s->sched->totals();
  std::memset(out, 0, sizeof *out);
  out->submitted = t.submitted;
  out->completed = t.completed;
  out->failed = t.failed;
  out->waiting = t.waiting;
  out->resident = t.resident;
  out->resident_bodies = t.resident_bodies;
  out->max_resident = t.max_resident;
  out->ticks = t.ticks;
  out->scene_steps = t.scene_steps;
  out->body_steps = t.body_steps;
  out->budget_bytes = t.budget_bytes;
  out->resident_bytes_est = t.resident_bytes_est;
  out->device_bytes = t.device_bytes;
  out->rows_per_body = t.rows_per_body;
  out->wall_s = t.wall_s;
  out->busy_s = t.busy_s;
  out->latency_p50 = t.p50;
  out->latency_p99 = t.p99;
  out->latency_max = t.lat_max;
  out->latency_mean = t.lat_mean;
  out->concurrency_mean = t.conc_mean;
  static_assert(sizeof out->concurrency_hist / sizeof out->concurrency_hist[0] ==
                dem_sched::kConcBins, "histogram bins");
  for (int i = 0; i < dem_sched::kConcBins; ++i) out->concurrency_hist[i] = t.conc_hist[i];
  return DEM_OK;
}

const char *dem_server_last_error(dem_server *s) {
  if (!s) return dem_last_error(nullptr);
  thread_local std::string copy;
  std::lock_guard<std::mutex> lk(s->err_mu);
  copy = s->err;
  return copy.c_str();
}

}  // extern "C"
