// Host-side checks of the server's scheduling core (csrc/server_sched.h) with a
// fake device backend: no GPU, no CUDA.  Built and run by tests/test_server_sched.py.
// Each scenario prints one line "<name> ok" or aborts with a message.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <set>

#include "server_sched.h"

using dem_sched::Req;
using dem_sched::Scheduler;

#define CHECK(c)                                                              \
  do {                                                                        \
    if (!(c)) {                                                               \
      std::fprintf(stderr, "%s:%d: check failed: %s\n", __FILE__, __LINE__, #c); \
      std::exit(1);                                                           \
    }                                                                         \
  } while (0)

// Fake device: every resident sub-scene advances with each step; optional gate
// that holds a step until the test releases it; optional failures.
struct Fake {
  std::mutex mu;
  std::condition_variable cv;
  std::map<int, long long> iter;     // sub -> steps taken
  std::map<int, long long> n;        // sub -> bodies
  std::vector<long long> ticks;      // step sizes
  std::vector<std::vector<int>> resident_at_tick;
  std::vector<long long> admitted;   // tickets in admission order
  int next_sub = 1;
  std::set<int> free_subs;
  double rho = 0;                    // reported rows per body
  long long fail_admit_ticket = -1;
  int fail_step_at = -1;             // step call index that fails
  bool gate = false, open = true;
  int steps_called = 0;

  void thread_init() {}
  int admit(Req &r, std::string &msg) {
    std::lock_guard<std::mutex> lk(mu);
    if (r.ticket == fail_admit_ticket) { msg = "bad scene"; return 6; }
    int sub;
    if (!free_subs.empty()) { sub = *free_subs.begin(); free_subs.erase(free_subs.begin()); }
    else sub = next_sub++;
    r.sub = sub;
    iter[sub] = 0;
    n[sub] = r.n;
    admitted.push_back(r.ticket);
    return 0;
  }
  int step(long long k, std::string &msg) {
    std::unique_lock<std::mutex> lk(mu);
    if (gate) cv.wait(lk, [&] { return open; });
    if (steps_called++ == fail_step_at) { msg = "device fault"; return 8; }
    ticks.push_back(k);
    std::vector<int> subs;
    for (auto &kv : iter) { kv.second += k; subs.push_back(kv.first); }
    resident_at_tick.push_back(subs);
    return 0;
  }
  int collect(Req &r, std::string &) {
    std::lock_guard<std::mutex> lk(mu);
    r.iter = iter[r.sub];
    r.stats.assign(1, (double)n[r.sub]);
    if (r.keep_state) r.out_pos.assign(3 * r.n, (double)r.ticket);
    return 0;
  }
  void remove(Req &r) {
    std::lock_guard<std::mutex> lk(mu);
    iter.erase(r.sub);
    n.erase(r.sub);
    free_subs.insert(r.sub);
  }
  double rows_per_body() { return rho; }
  long long device_bytes() { return 1234; }
  void set_gate(bool closed) {
    std::lock_guard<std::mutex> lk(mu);
    gate = true;
    open = !closed;
    cv.notify_all();
  }
};

static std::unique_ptr<Req> req(long long n, long long steps, int keep = 0) {
  std::unique_ptr<Req> r(new Req);
  r->n = n;
  r->nsteps = steps;
  r->keep_state = keep;
  return r;
}

static long long submit(Scheduler<Fake> &s, long long n, long long steps, int keep = 0) {
  long long t = 0;
  std::string msg;
  const int rc = s.submit(req(n, steps, keep), &t, msg);
  CHECK(rc == 0);
  return t;
}

// bytes per body 100, per row 10, 0 rows per body at start: a body costs 100 bytes
static void budget_and_order() {
  Fake f;
  f.set_gate(true);   // hold the first step so every request is queued first
  Scheduler<Fake> s(&f, 1000, 50, 100.0, 10.0, 0.0);
  s.start();
  const long long a = submit(s, 6, 120);   // 600 bytes
  const long long b = submit(s, 5, 30);    // does not fit beside a: waits
  const long long c = submit(s, 1, 30);    // would fit, but FCFS: waits behind b
  f.set_gate(false);
  std::string msg;
  CHECK(s.wait(a, 30, msg) == 0);
  CHECK(s.wait(b, 30, msg) == 0);
  CHECK(s.wait(c, 30, msg) == 0);
  // a alone first; b (and c, which fits beside b) join only once a has left
  CHECK(f.admitted.size() == 3 && f.admitted[0] == a && f.admitted[1] == b && f.admitted[2] == c);
  // ticks never overshoot a budget: a runs 50, 50, 20
  CHECK(f.ticks.size() >= 4 && f.ticks[0] == 50 && f.ticks[1] == 50 && f.ticks[2] == 20);
  s.with_result(a, [&](const Req &r) { CHECK(r.iter == 120 && r.state == dem_sched::kDone); });
  s.with_result(b, [&](const Req &r) { CHECK(r.iter == 30); });
  s.with_result(c, [&](const Req &r) { CHECK(r.iter == 30); });
  // the sub-scene index freed by a is reused
  CHECK(f.free_subs.size() >= 1);
  const dem_sched::Totals t = s.totals();
  CHECK(t.completed == 3 && t.failed == 0 && t.scene_steps == 180);
  CHECK(t.body_steps == 6 * 120 + 5 * 30 + 1 * 30);
  std::printf("budget_and_order ok\n");
}

// a request submitted while a tick runs joins at the next tick (overlap on the device)
static void join_while_running() {
  Fake f;
  f.set_gate(true);
  Scheduler<Fake> s(&f, 1 << 20, 10, 1.0, 0.0, 0.0);
  s.start();
  const long long a = submit(s, 3, 40);
  // wait for a's admission (the worker is now held inside its first step)
  for (int i = 0; i < 2000 && s.poll(a) != dem_sched::kResident; ++i)
    std::this_thread::sleep_for(std::chrono::milliseconds(1));
  CHECK(s.poll(a) == dem_sched::kResident);
  const long long b = submit(s, 2, 15);
  CHECK(s.poll(b) == dem_sched::kWaiting);
  f.set_gate(false);
  std::string msg;
  CHECK(s.wait(b, 30, msg) == 0);
  CHECK(s.wait(a, 30, msg) == 0);
  // tick 0: a alone; then a and b together until b's 15 steps are done (10 + 5)
  CHECK(f.resident_at_tick[0].size() == 1);
  CHECK(f.resident_at_tick[1].size() == 2 && f.ticks[1] == 10 && f.ticks[2] == 5);
  s.with_result(b, [&](const Req &r) { CHECK(r.iter == 15 && r.t_admit >= r.t_submit); });
  s.with_result(a, [&](const Req &r) { CHECK(r.iter == 40); });
  const dem_sched::Totals tt = s.totals();
  CHECK(tt.max_resident == 2);
  // ticks by resident count: a alone (10, then 10 and 5 after b left), a with b (10, 5)
  CHECK(tt.ticks == 5 && tt.conc_hist[0] == 3 && tt.conc_hist[1] == 2);
  // bins: 1 | 2 | 3-4 | 5-8 | ... | 33-64 | more than 64
  CHECK(dem_sched::conc_bin(1) == 0 && dem_sched::conc_bin(2) == 1 && dem_sched::conc_bin(3) == 2);
  CHECK(dem_sched::conc_bin(4) == 2 && dem_sched::conc_bin(5) == 3 && dem_sched::conc_bin(64) == 6);
  CHECK(dem_sched::conc_bin(65) == 7 && dem_sched::conc_bin(100000) == 7);
  std::printf("join_while_running ok\n");
}

// the measured rows per body enter the footprint; too large a request is refused
static void footprint_and_capacity() {
  Fake f;
  f.rho = 9.0;
  Scheduler<Fake> s(&f, 2000, 5, 100.0, 10.0, 1.0);   // 110 bytes/body at start
  s.start();
  long long t = 0;
  std::string msg;
  CHECK(s.submit(req(19, 5), &t, msg) == 4);   // 19 x 110 > 2000
  const long long a = submit(s, 10, 5);
  CHECK(s.wait(a, 30, msg) == 0);
  // after a tick the estimate is 100 + 9 x 10 = 190 bytes per body
  const dem_sched::Totals tt = s.totals();
  CHECK(std::fabs(tt.rows_per_body - 9.0) < 1e-12);
  CHECK(std::fabs(s.footprint(10) - 1900.0) < 1e-9);
  CHECK(tt.device_bytes == 1234);
  std::printf("footprint_and_capacity ok\n");
}

// an admission error fails that request only; a step error fails every request
static void failures() {
  {
    Fake f;
    f.fail_admit_ticket = 2;
    Scheduler<Fake> s(&f, 1 << 20, 7, 1.0, 0.0, 0.0);
    s.start();
    const long long a = submit(s, 2, 7), b = submit(s, 2, 7), c = submit(s, 2, 7);
    std::string msg;
    CHECK(s.wait(a, 30, msg) == 0);
    CHECK(s.wait(b, 30, msg) == 6 && msg == "bad scene");
    CHECK(s.wait(c, 30, msg) == 0);
    CHECK(s.totals().failed == 1 && s.totals().completed == 2);
  }
  {
    Fake f;
    f.fail_step_at = 1;
    Scheduler<Fake> s(&f, 1 << 20, 4, 1.0, 0.0, 0.0);
    s.start();
    const long long a = submit(s, 2, 100);
    std::string msg;
    CHECK(s.wait(a, 30, msg) == 8 && msg == "device fault");
    long long t = 0;
    CHECK(s.submit(req(1, 1), &t, msg) == 8);   // the server stays failed
  }
  std::printf("failures ok\n");
}

// wait with a deadline; unknown tickets; release; results kept only on request
static void wait_release_state() {
  Fake f;
  f.set_gate(true);
  Scheduler<Fake> s(&f, 1 << 20, 3, 1.0, 0.0, 0.0);
  s.start();
  const long long a = submit(s, 4, 6, 1);
  std::string msg;
  CHECK(s.wait(a, 0.05, msg) == -2);        // held by the gate: times out
  CHECK(s.wait(9999, 1, msg) == -1);
  CHECK(s.release(a) == -3);                // not finished
  f.set_gate(false);
  CHECK(s.wait(a, 30, msg) == 0);
  s.with_result(a, [&](const Req &r) { CHECK(r.out_pos.size() == 12 && r.out_pos[0] == (double)a); });
  CHECK(s.release(a) == 0);
  CHECK(s.poll(a) == -1);
  std::printf("wait_release_state ok\n");
}

// latencies: print them with the server's percentiles for a check against numpy
static void percentiles() {
  std::vector<double> v = {3.0, 1.0, 4.0, 1.5, 9.0, 2.6, 5.0};
  std::printf("percentiles %.17g %.17g %.17g\n", dem_sched::percentile(v, 50),
              dem_sched::percentile(v, 99), dem_sched::percentile(v, 12.5));
}

// stopping fails what is left and joins the worker
static void stop_drops_pending() {
  Fake f;
  f.set_gate(true);
  auto *s = new Scheduler<Fake>(&f, 10, 3, 1.0, 0.0, 0.0);
  s->start();
  const long long a = submit(*s, 8, 6);
  const long long b = submit(*s, 8, 6);   // waits (budget 10)
  std::thread opener([&] {
    std::this_thread::sleep_for(std::chrono::milliseconds(50));
    f.set_gate(false);
  });
  s->stop();
  opener.join();
  std::string msg;
  CHECK(s->wait(b, 1, msg) == 9);
  const int sa = s->poll(a);
  CHECK(sa == dem_sched::kDone || sa == dem_sched::kFailed);
  delete s;
  std::printf("stop_drops_pending ok\n");
}

int main() {
  budget_and_order();
  join_while_running();
  footprint_and_capacity();
  failures();
  wait_release_state();
  percentiles();
  stop_drops_pending();
  return 0;
}
