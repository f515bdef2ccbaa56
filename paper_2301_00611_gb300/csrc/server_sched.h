// Scheduling core of the continuous-batching DEM server (host code only, no CUDA).
//
// The paper has no serving layer: this is the batching/serving pattern applied
// to the method's hot path.  Requests (one scene each and a step budget) wait in
// arrival order; a worker thread admits them as sub-scenes of one device scene
// while their estimated device footprint fits the budget (first come, first
// served: a request that does not fit blocks those behind it, so none starves),
// advances every resident scene by the same steps (one tick), and retires the
// scenes whose budget is spent: their results are read to the host, their
// sub-scenes removed, which frees room for the requests still waiting.  Scene
// state stays on the device between ticks.  A tick is the smallest remaining
// budget among the resident scenes, capped by tick_steps, so no scene overshoots
// and a finished scene leaves at the end of the tick it finished in.
//
// The footprint of a request is its bodies times (bytes per body + rows per body
// x bytes per table row), with the rows per body measured on the device after
// every tick (never below the initial estimate).
//
// `Backend` does the device work (the library's scene backend, or a host fake in
// the tests):
//   int  admit(Req &r, std::string &msg)        add r as a sub-scene (sets r.sub)
//   int  step(long long k, std::string &msg)    advance every resident sub-scene
//   int  collect(Req &r, std::string &msg)      r's statistics (and state if kept)
//   void remove(Req &r)                         drop r's sub-scene
//   double rows_per_body()                      table rows per resident body (<= 0: none)
//   long long device_bytes()                    device memory the scene holds
//   void thread_init()                          first call on the worker thread
// All of them run on the worker thread only.
#pragma once
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace dem_sched {

enum ReqState { kWaiting = 0, kResident = 1, kDone = 2, kFailed = 3 };

// One request and, once done, its result.  Scene data is copied in at submission.
struct Req {
  long long ticket = 0;
  long long n = 0, nsteps = 0, left = 0;
  int nmat = 0;
  int keep_state = 0;
  std::vector<double> pos, radius, vel, angvel, mats;   // mats: 4 per material
  std::vector<int> mat;                                  // local material index per sphere
  std::vector<unsigned char> desc;                       // the backend's scene descriptor
  bool has_velgrad = false;
  double velgrad[9] = {0};
  double t_submit = 0, t_admit = -1, t_done = -1;
  int state = kWaiting;
  int err = 0;
  std::string msg;
  // set by the backend
  int sub = -1, mat_base = -1;
  long long iter = 0;
  double time = 0, dt = 0;
  std::vector<double> stats;                             // backend-defined record
  std::vector<double> out_pos, out_vel, out_angvel, out_ori;
};

constexpr int kConcBins = 8;

// Histogram bin of a resident count r >= 1 (see Totals::conc_hist).
inline int conc_bin(long long r) {
  int b = 0;
  while (b < kConcBins - 1 && (1LL << b) < r) ++b;
  return b;
}

struct Totals {
  long long submitted = 0, completed = 0, failed = 0, waiting = 0, resident = 0;
  long long resident_bodies = 0, max_resident = 0, ticks = 0, scene_steps = 0, body_steps = 0;
  long long budget_bytes = 0, resident_bytes_est = 0, device_bytes = 0;
  double rows_per_body = 0, wall_s = 0, busy_s = 0;
  double p50 = 0, p99 = 0, lat_max = 0, lat_mean = 0, conc_mean = 0;
  // ticks by resident requests: bin 0 one, bin b (1..kConcBins-2) 2^(b-1)+1 .. 2^b,
  // the last bin more than 2^(kConcBins-2)
  long long conc_hist[kConcBins] = {};
};

// Linear interpolation between the order statistics (numpy's default percentile).
inline double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = p / 100.0 * (double)(v.size() - 1);
  const size_t i = (size_t)x;
  if (i + 1 >= v.size()) return v.back();
  return v[i] + (x - (double)i) * (v[i + 1] - v[i]);
}

template <class Backend>
class Scheduler {
 public:
  // bytes_per_body, bytes_per_row: device bytes of one body and one table row
  Scheduler(Backend *be, long long budget_bytes, long long tick_steps, double bytes_per_body,
            double bytes_per_row, double rows_per_body0)
      : be_(be), budget_(budget_bytes), tick_(tick_steps < 1 ? 1 : tick_steps),
        bpb_(bytes_per_body), bpr_(bytes_per_row), rho0_(rows_per_body0), rho_(rows_per_body0) {
    t0_ = clock_s();
  }
  ~Scheduler() { stop(); }

  void start() { worker_ = std::thread([this] { run(); }); }

  // Stop after the current tick; requests still waiting or resident fail.
  void stop() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stopping_ = true;
    }
    cv_work_.notify_all();
    if (worker_.joinable()) worker_.join();
    std::lock_guard<std::mutex> lk(mu_);
    for (auto &kv : reqs_)
      if (kv.second->state == kWaiting || kv.second->state == kResident)
        finish_failed(*kv.second, 9 /* DEM_ERR_STATE */, "server stopped");
    waiting_.clear();
    cv_done_.notify_all();
  }

  double now() const { return clock_s() - t0_; }

  // Footprint estimate of n bodies at the current rows per body.
  double footprint(long long n) const { return (double)n * (bpb_ + rho_ * bpr_); }

  // 0 and a ticket, or an error code (8: server failed, 4: larger than the budget).
  int submit(std::unique_ptr<Req> r, long long *ticket, std::string &msg) {
    std::lock_guard<std::mutex> lk(mu_);
    if (fatal_) { msg = fatal_msg_; return fatal_; }
    if (stopping_) { msg = "server stopped"; return 9; }
    if ((double)r->n * (bpb_ + rho0_ * bpr_) > (double)budget_) {
      msg = "request larger than the server's device-memory budget";
      return 4;
    }
    r->ticket = next_++;
    r->t_submit = now();
    r->left = r->nsteps;
    r->state = kWaiting;
    *ticket = r->ticket;
    waiting_.push_back(r.get());
    reqs_[r->ticket] = std::move(r);
    ++submitted_;
    cv_work_.notify_all();
    return 0;
  }

  // state of a ticket (-1: unknown)
  int poll(long long ticket) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = reqs_.find(ticket);
    return it == reqs_.end() ? -1 : it->second->state;
  }

  // 0 done, the request's error if it failed, -1 unknown ticket, -2 timed out
  int wait(long long ticket, double timeout_s, std::string &msg) {
    std::unique_lock<std::mutex> lk(mu_);
    auto it = reqs_.find(ticket);
    if (it == reqs_.end()) return -1;
    Req *r = it->second.get();
    const double lim = timeout_s < 0 ? 0 : (timeout_s > 1e7 ? 1e7 : timeout_s);
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(lim));
    while (r->state == kWaiting || r->state == kResident) {
      if (cv_done_.wait_until(lk, until) == std::cv_status::timeout &&
          (r->state == kWaiting || r->state == kResident))
        return -2;
    }
    if (r->state == kFailed) { msg = r->msg; return r->err ? r->err : 9; }
    return 0;
  }

  // Run f on a finished request under the lock (-1 unknown, -3 not finished).
  template <class F>
  int with_result(long long ticket, F f) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = reqs_.find(ticket);
    if (it == reqs_.end()) return -1;
    if (it->second->state != kDone && it->second->state != kFailed) return -3;
    f(*it->second);
    return 0;
  }

  int release(long long ticket) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = reqs_.find(ticket);
    if (it == reqs_.end()) return -1;
    if (it->second->state != kDone && it->second->state != kFailed) return -3;
    reqs_.erase(it);
    return 0;
  }

  Totals totals() {
    std::lock_guard<std::mutex> lk(mu_);
    Totals t;
    t.submitted = submitted_;
    t.completed = completed_;
    t.failed = failed_;
    t.waiting = (long long)waiting_.size();
    t.resident = (long long)resident_.size();
    t.resident_bodies = resident_bodies_;
    t.max_resident = max_resident_;
    t.ticks = ticks_;
    t.scene_steps = scene_steps_;
    t.body_steps = body_steps_;
    t.budget_bytes = budget_;
    t.resident_bytes_est = (long long)footprint(resident_bodies_);
    t.device_bytes = device_bytes_;
    t.rows_per_body = rho_;
    t.wall_s = now();
    t.busy_s = busy_;
    t.p50 = percentile(lat_, 50);
    t.p99 = percentile(lat_, 99);
    t.lat_max = lat_.empty() ? 0 : *std::max_element(lat_.begin(), lat_.end());
    double s = 0;
    for (double x : lat_) s += x;
    t.lat_mean = lat_.empty() ? 0 : s / (double)lat_.size();
    t.conc_mean = ticks_ ? (double)conc_sum_ / (double)ticks_ : 0;
    for (int i = 0; i < kConcBins; ++i) t.conc_hist[i] = conc_hist_[i];
    return t;
  }

  int fatal(std::string &msg) {
    std::lock_guard<std::mutex> lk(mu_);
    msg = fatal_msg_;
    return fatal_;
  }

 private:
  static double clock_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
  }

  void finish_failed(Req &r, int code, const std::string &msg) {   // lock held
    r.state = kFailed;
    r.err = code;
    r.msg = msg;
    r.t_done = now();
    ++failed_;
  }

  // Admission: waiting requests in arrival order while the footprint fits (one
  // request always fits an empty server: submit bounded it by the budget).
  std::vector<Req *> pick_admissions() {   // lock held
    std::vector<Req *> out;
    long long nres = resident_bodies_;
    bool any = !resident_.empty();
    while (!waiting_.empty()) {
      Req *r = waiting_.front();
      if (any && footprint(nres + r->n) > (double)budget_) break;
      waiting_.pop_front();
      out.push_back(r);
      nres += r->n;
      any = true;
    }
    return out;
  }

  void run() {
    be_->thread_init();
    while (true) {
      std::vector<Req *> adm;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_work_.wait(lk, [&] { return stopping_ || !waiting_.empty() || !resident_.empty(); });
        if (stopping_) return;
        adm = pick_admissions();
      }
      for (Req *r : adm) {   // device work outside the lock
        std::string msg;
        const int rc = be_->admit(*r, msg);
        std::lock_guard<std::mutex> lk(mu_);
        if (rc) {
          finish_failed(*r, rc, msg);
          cv_done_.notify_all();
          continue;
        }
        r->state = kResident;
        r->t_admit = now();
        resident_.push_back(r);
        resident_bodies_ += r->n;
      }
      if (resident_.empty()) continue;
      long long k = tick_;
      for (Req *r : resident_) k = std::min(k, r->left);
      std::string msg;
      const double ta = now();
      const int rc = be_->step(k, msg);
      const double tb = now();
      if (rc) {   // the device scene is unusable: every request in it fails
        std::lock_guard<std::mutex> lk(mu_);
        fatal_ = rc;
        fatal_msg_ = msg;
        for (Req *r : resident_) finish_failed(*r, rc, msg);
        for (Req *r : waiting_) finish_failed(*r, rc, msg);
        resident_.clear();
        waiting_.clear();
        resident_bodies_ = 0;
        cv_done_.notify_all();
        stopping_ = true;
        return;
      }
      std::vector<Req *> done;
      {
        std::lock_guard<std::mutex> lk(mu_);
        busy_ += tb - ta;
        ++ticks_;
        conc_sum_ += (long long)resident_.size();
        ++conc_hist_[conc_bin((long long)resident_.size())];
        max_resident_ = std::max<long long>(max_resident_, (long long)resident_.size());
        for (Req *r : resident_) {
          r->left -= k;
          scene_steps_ += k;
          body_steps_ += k * r->n;
          if (r->left == 0) done.push_back(r);
        }
      }
      const double rho = be_->rows_per_body();
      // read every finished scene before removing any (a removal changes the
      // layout until the next step)
      std::vector<int> crc(done.size());
      std::vector<std::string> cmsg(done.size());
      for (size_t i = 0; i < done.size(); ++i) crc[i] = be_->collect(*done[i], cmsg[i]);
      for (Req *r : done) be_->remove(*r);
      const long long dev = be_->device_bytes();
      std::lock_guard<std::mutex> lk(mu_);
      if (rho > 0) rho_ = std::max(rho0_, rho);
      device_bytes_ = std::max(device_bytes_, dev);
      const double t = now();
      for (size_t i = 0; i < done.size(); ++i) {
        Req *r = done[i];
        resident_bodies_ -= r->n;
        resident_.erase(std::find(resident_.begin(), resident_.end(), r));
        if (crc[i]) {
          finish_failed(*r, crc[i], cmsg[i]);
          continue;
        }
        r->state = kDone;
        r->t_done = t;
        lat_.push_back(t - r->t_submit);
        ++completed_;
      }
      if (!done.empty()) cv_done_.notify_all();
    }
  }

  Backend *be_;
  long long budget_, tick_;
  double bpb_, bpr_, rho0_, rho_;
  double t0_;
  std::thread worker_;
  std::mutex mu_;
  std::condition_variable cv_work_, cv_done_;
  std::deque<Req *> waiting_;
  std::vector<Req *> resident_;
  std::map<long long, std::unique_ptr<Req>> reqs_;
  long long next_ = 1, submitted_ = 0, completed_ = 0, failed_ = 0;
  long long resident_bodies_ = 0, max_resident_ = 0, ticks_ = 0, scene_steps_ = 0,
            body_steps_ = 0, conc_sum_ = 0, device_bytes_ = 0;
  long long conc_hist_[kConcBins] = {};
  double busy_ = 0;
  std::vector<double> lat_;
  bool stopping_ = false;
  int fatal_ = 0;
  std::string fatal_msg_;
};

}  // namespace dem_sched
