// Serving: a request loop with continuous batching over parametric RTE solves.
//
// A server holds buckets; a bucket is one discretisation (mesh, quadrature) with a batch whose
// B instances are the bucket's slots, a ROM pair for that discretisation and the solve options
// (Alg. 1 with the ROMSAD switch of Alg. 2, or another correction).  A request names a bucket
// and carries its parameters mu (cross sections, source, inflow) and its own tolerance.
//
// One worker thread drives all buckets, each on its own CUDA stream.  Per bucket it repeats:
// wait for the norms of the iteration in flight (polling, never blocking on one bucket while
// another is ready), apply the stop test and launch the corrections (si_finish), hand finished
// slots' results back, admit queued requests into free slots (parameter upload, per-slot
// tables, DSA blocks and reduced operators, initial iterate), and launch the next sweep of every
// running slot (si_launch).  A request that arrives while others are on the GPU therefore joins
// the next sweep of its bucket; its slot keeps rho, the ROM factors and the DSA blocks on the
// device until it finishes.  Each instance's arithmetic is independent of the other slots, so a
// result does not depend on what else was in the batch (up to the summation order of the sweep
// partial sums, which depends on the number of running slots through the sweep decomposition).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "common.cuh"

namespace rte {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int bucket = 0;
  std::vector<double> sigma_t, sigma_s, source, inflow;
  double eps = 0.0;
  std::vector<double> rho;
  rte_serve_report rep{};
  bool complete = false;
};

enum SlotState { kFree = 0, kRunning = 1, kDraining = 2 };

struct Bucket {
  rte_batch_t bt = nullptr;
  rte_rom_t rom_p = nullptr, rom_c = nullptr;
  rte_solve_opts o{};
  cudaStream_t st = nullptr;
  SiState s;
  double* out = nullptr;                 // pinned [B][n_dof] results of finished slots
  std::deque<Request*> queue;
  std::vector<Request*> slot_req;
  std::vector<int> state;
  std::vector<cudaEvent_t> slot_ev;
  ~Bucket() {
    for (auto e : slot_ev) cudaEventDestroy(e);
    if (out) cudaFreeHost(out);
    if (st) cudaStreamDestroy(st);
  }
};

}  // namespace
}  // namespace rte

struct rte_server_s {
  int device = 0;
  std::vector<rte::Bucket*> buckets;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::unordered_map<uint64_t, rte::Request*> reqs;
  uint64_t next_ticket = 1;
  bool started = false, stop = false;
  int error = RTE_OK;
  std::string error_msg;
  rte::Clock::time_point t0 = rte::Clock::now();
  // statistics: worker-side counters are atomics (read by rte_server_stats from other threads)
  std::atomic<long long> launches{0}, admitted{0}, max_running{0}, busy_ns{0};
  long long completed = 0, max_queue = 0;  // under mu
  ~rte_server_s() {
    for (auto* b : buckets) delete b;
    for (auto& kv : reqs) delete kv.second;
  }
};

namespace rte {
namespace {

double now_s(const rte_server_s* sv) {
  return std::chrono::duration<double>(Clock::now() - sv->t0).count();
}

// Admits queued requests of bucket k into its free slots.
int admit(rte_server_s* sv, Bucket& K) {
  std::vector<int> free_slots;
  for (int b = 0; b < K.s.B; ++b)
    if (K.state[b] == kFree) free_slots.push_back(b);
  if (free_slots.empty()) return RTE_OK;
  std::vector<Request*> take;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    while (!K.queue.empty() && take.size() < free_slots.size()) {
      take.push_back(K.queue.front());
      K.queue.pop_front();
    }
  }
  if (take.empty()) return RTE_OK;
  const rte_disc_s* d = K.bt->disc;
  const int n = (int)take.size(), nm = d->n_mat, nc = d->n_cells, ni = 2 * d->dim;
  std::vector<int> slots(n);
  std::vector<double> st((size_t)n * nm), ss((size_t)n * nm), src((size_t)n * nc), inf((size_t)n * ni);
  for (int i = 0; i < n; ++i) {
    slots[i] = free_slots[i];
    std::copy(take[i]->sigma_t.begin(), take[i]->sigma_t.end(), st.begin() + (size_t)i * nm);
    std::copy(take[i]->sigma_s.begin(), take[i]->sigma_s.end(), ss.begin() + (size_t)i * nm);
    std::copy(take[i]->source.begin(), take[i]->source.end(), src.begin() + (size_t)i * nc);
    std::copy(take[i]->inflow.begin(), take[i]->inflow.end(), inf.begin() + (size_t)i * ni);
  }
  RTE_TRY(set_slots(K.bt, n, slots.data(), st.data(), ss.data(), src.data(), inf.data(), K.st));
  double* rho0 = K.bt->work.p;  // slot rows of the current iterate
  if (K.rom_p) {
    PhaseScope ps(K.bt, 2, K.st);
    RTE_TRY(rom_guess_launch(K.rom_p, K.bt, rho0, K.bt->slot_mask.p, K.st));
  } else {
    for (int b : slots)
      RTE_CUDA_TRY(cudaMemsetAsync(rho0 + (size_t)b * d->n_dof, 0, sizeof(double) * d->n_dof, K.st));
  }
  if (K.rom_c) RTE_TRY(rom_prepare(K.rom_c, K.bt, K.st, K.bt->slot_mask.p));
  const double t = now_s(sv);
  for (int i = 0; i < n; ++i) {
    const int b = slots[i];
    K.s.begin(b, take[i]->eps);
    K.slot_req[b] = take[i];
    K.state[b] = kRunning;
    take[i]->rep.t_admit = t;
    take[i]->rep.slot = b;
  }
  sv->admitted += n;
  return RTE_OK;
}

// Moves finished slots to draining: their result copy was enqueued by si_finish.
int collect(Bucket& K) {
  for (int b = 0; b < K.s.B; ++b)
    if (K.s.done[b]) {
      K.s.done[b] = 0;
      K.state[b] = kDraining;
      Request* r = K.slot_req[b];
      r->rep.solve = K.s.rep[b];
      r->rep.status = K.s.status[b];
      RTE_CUDA_TRY(cudaEventRecord(K.slot_ev[b], K.st));
    }
  return RTE_OK;
}

// Completes draining slots whose result copy has landed in pinned memory.
int drain(rte_server_s* sv, Bucket& K, bool* progress) {
  const size_t n = K.bt->disc->n_dof;
  for (int b = 0; b < K.s.B; ++b) {
    if (K.state[b] != kDraining) continue;
    bool ready = false;
    RTE_TRY(event_ready(K.slot_ev[b], &ready));
    if (!ready) continue;
    Request* r = K.slot_req[b];
    r->rho.assign(K.out + b * n, K.out + (b + 1) * n);
    K.slot_req[b] = nullptr;
    K.state[b] = kFree;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      r->rep.t_done = now_s(sv);
      r->complete = true;
      sv->completed += 1;
    }
    sv->cv_done.notify_all();
    *progress = true;
  }
  return RTE_OK;
}

int step_bucket(rte_server_s* sv, Bucket& K, bool* progress, bool* busy) {
  if (K.s.in_flight) {
    bool ready = false;
    RTE_TRY(event_ready(K.s.ev, &ready));
    if (!ready) {
      *busy = true;
      return RTE_OK;
    }
    RTE_TRY(si_finish(K.s, K.st, nullptr));
    RTE_TRY(collect(K));
    *progress = true;
  }
  RTE_TRY(admit(sv, K));
  const int running = K.s.n_active();
  if (running > 0) {
    RTE_TRY(si_launch(K.s, K.st, nullptr));
    sv->launches += 1;
    if (running > sv->max_running.load()) sv->max_running.store(running);
    *progress = true;
  }
  *busy = *busy || K.s.in_flight;
  return RTE_OK;
}

void fail_all(rte_server_s* sv, int code, const std::string& msg) {
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->error == RTE_OK) {
    sv->error = code;
    sv->error_msg = msg;
  }
  for (auto& kv : sv->reqs)
    if (!kv.second->complete) {
      kv.second->rep.status = sv->error;
      kv.second->rep.t_done = now_s(sv);
      kv.second->complete = true;
    }
  for (auto* K : sv->buckets) K->queue.clear();
}

void worker_main(rte_server_s* sv) {
  cudaSetDevice(sv->device);
  cudaGetLastError();
  int err = RTE_OK;
  while (err == RTE_OK) {
    bool progress = false, busy = false, draining = false;
    const auto t_loop = Clock::now();
    for (auto* K : sv->buckets) {
      err = step_bucket(sv, *K, &progress, &busy);
      if (err != RTE_OK) break;
      err = drain(sv, *K, &progress);
      if (err != RTE_OK) break;
      for (int s : K->state) draining = draining || s == kDraining;
    }
    if (err != RTE_OK) break;
    if (busy)
      sv->busy_ns += std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t_loop).count();
    if (progress) continue;
    std::unique_lock<std::mutex> lk(sv->mu);
    bool queued = false;
    for (auto* K : sv->buckets) queued = queued || !K->queue.empty();
    if (sv->stop && !busy && !draining) break;
    if (!busy && !draining && !queued) {
      sv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
    } else {
      lk.unlock();
      std::this_thread::yield();
    }
  }
  if (err != RTE_OK) {
    const std::string msg = rte_last_error();
    for (auto* K : sv->buckets) cudaStreamSynchronize(K->st);
    fail_all(sv, err, msg);
  } else {
    fail_all(sv, RTE_ESTATE, "server stopped");
  }
  sv->cv_done.notify_all();
}

}  // namespace
}  // namespace rte

using namespace rte;

extern "C" int rte_server_create(int device, rte_server_t* out) {
  if (!out) return fail(RTE_EINVAL, "rte_server_create: null argument");
  auto* sv = new rte_server_s();
  sv->device = device;
  *out = sv;
  return RTE_OK;
}

extern "C" int rte_server_add_bucket(rte_server_t sv, rte_batch_t slots, rte_rom_t rom_p,
                                     rte_rom_t rom_c, const rte_solve_opts* o, int* bucket) {
  if (!sv || !slots || !o) return fail(RTE_EINVAL, "rte_server_add_bucket: null argument");
  if (sv->started) return fail(RTE_ESTATE, "rte_server_add_bucket: server already started");
  if (slots->disc->device != sv->device) return fail(RTE_EINVAL, "batch on another device");
  if (!(o->eps >= 0) || o->max_iter < 1 || o->sa < 0 || o->sa > 3 || !(o->fp32_switch >= 0) ||
      !(o->refine_kappa >= 0) || (o->refine_kappa > 0 && o->refine_inner < 1) ||
      o->gang_wait < 0 || o->schedule || o->sa_history || o->verify || o->outer_ff < 0 ||
      o->outer_ff > 1)
    return fail(RTE_EINVAL, "rte_server_add_bucket: bad options");
  if (o->sa != RTE_SA_NONE && slots->disc->dim == 2 && (!(o->dsa_rtol >= 0) || o->dsa_max_it < 1))
    return fail(RTE_EINVAL, "rte_server_add_bucket: bad DSA tolerance");
  if ((o->sa == RTE_SA_ROMSA || o->sa == RTE_SA_ROMSAD) && !rom_c)
    return fail(RTE_EINVAL, "ROMSA/ROMSAD need a correction ROM");
  for (rte_rom_t r : {rom_p, rom_c})
    if (r && r->disc != slots->disc) return fail(RTE_EINVAL, "ROM built on another discretisation");
  for (auto* K : sv->buckets)
    if (K->bt == slots || (rom_p && (K->rom_p == rom_p || K->rom_c == rom_p)) ||
        (rom_c && (K->rom_p == rom_c || K->rom_c == rom_c)))
      return fail(RTE_EINVAL, "a batch or ROM serves one bucket only");
  if (rom_p && rom_p == rom_c) return fail(RTE_EINVAL, "rom_p and rom_c must differ");
  DeviceGuard g(sv->device);
  auto* K = new Bucket();
  K->bt = slots;
  K->rom_p = rom_p;
  K->rom_c = rom_c;
  K->o = *o;
  const int B = slots->B;
  const size_t n = slots->disc->n_dof;
  int e = RTE_OK;
  if (cudaHostAlloc((void**)&K->out, sizeof(double) * n * B, cudaHostAllocDefault) != cudaSuccess)
    e = fail(RTE_ENOMEM, "rte_server_add_bucket: pinned buffer");
  if (e == RTE_OK) e = K->s.init(slots, *o, rom_c, K->out);
  K->slot_req.assign(B, nullptr);
  K->state.assign(B, kFree);
  for (int b = 0; e == RTE_OK && b < B; ++b) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      e = fail(RTE_ECUDA, "rte_server_add_bucket: event");
    else K->slot_ev.push_back(ev);
  }
  if (e != RTE_OK) {
    delete K;
    return e;
  }
  if (bucket) *bucket = (int)sv->buckets.size();
  sv->buckets.push_back(K);
  return RTE_OK;
}

extern "C" int rte_server_start(rte_server_t sv) {
  if (!sv) return fail(RTE_EINVAL, "rte_server_start: null argument");
  if (sv->started) return fail(RTE_ESTATE, "rte_server_start: already started");
  if (sv->buckets.empty()) return fail(RTE_ESTATE, "rte_server_start: no bucket");
  // one stream per bucket; cheaper buckets (fewer cell x direction solves per sweep) get higher
  // stream priority, so their short kernels are not queued behind the block backlog of the
  // expensive ones (priorities order pending blocks only; running blocks are not preempted)
  DeviceGuard g(sv->device);
  int least = 0, greatest = 0;
  RTE_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  std::vector<std::pair<double, int>> cost;
  for (int k = 0; k < (int)sv->buckets.size(); ++k) {
    const rte_disc_s* d = sv->buckets[k]->bt->disc;
    cost.emplace_back((double)d->n_cells * d->n_dirs, k);
  }
  std::sort(cost.begin(), cost.end());
  const int levels = least - greatest + 1, nb = (int)cost.size();
  for (int r = 0; r < nb; ++r) {
    const int prio = greatest + (nb > 1 ? (r * (levels - 1) + (nb - 1) / 2) / (nb - 1) : 0);
    Bucket* K = sv->buckets[cost[r].second];
    RTE_CUDA_TRY(cudaStreamCreateWithPriority(&K->st, cudaStreamNonBlocking, prio));
  }
  sv->started = true;
  sv->t0 = Clock::now();
  sv->worker = std::thread(worker_main, sv);
  return RTE_OK;
}

extern "C" int rte_server_submit(rte_server_t sv, int bucket, const double* sigma_t,
                                 const double* sigma_s, const double* source,
                                 const double* inflow, double eps, uint64_t* ticket) {
  if (!sv || !sigma_t || !sigma_s || !source || !inflow || !ticket)
    return fail(RTE_EINVAL, "rte_server_submit: null argument");
  if (bucket < 0 || bucket >= (int)sv->buckets.size()) return fail(RTE_EINVAL, "no such bucket");
  if (!(eps >= 0)) return fail(RTE_EINVAL, "rte_server_submit: bad tolerance");
  Bucket& K = *sv->buckets[bucket];
  const rte_disc_s* d = K.bt->disc;
  const int nm = d->n_mat, nc = d->n_cells, ni = 2 * d->dim;
  for (int m = 0; m < nm; ++m)
    if (!std::isfinite(sigma_t[m]) || !std::isfinite(sigma_s[m]) || !(sigma_t[m] > 0.0) ||
        sigma_s[m] < 0.0 || sigma_s[m] > sigma_t[m])
      return fail(RTE_EINVAL, "need finite sigma_t > 0 and 0 <= sigma_s <= sigma_t");
  for (int c = 0; c < nc; ++c)
    if (!std::isfinite(source[c])) return fail(RTE_EINVAL, "source is not finite");
  for (int k = 0; k < ni; ++k)
    if (!std::isfinite(inflow[k])) return fail(RTE_EINVAL, "inflow is not finite");
  auto* r = new Request();
  r->bucket = bucket;
  r->sigma_t.assign(sigma_t, sigma_t + nm);
  r->sigma_s.assign(sigma_s, sigma_s + nm);
  r->source.assign(source, source + nc);
  r->inflow.assign(inflow, inflow + ni);
  r->eps = eps;
  r->rep.bucket = bucket;
  r->rep.slot = -1;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->error != RTE_OK) {
      delete r;
      return fail(sv->error, "server failed: " + sv->error_msg);
    }
    if (!sv->started || sv->stop) {
      delete r;
      return fail(RTE_ESTATE, "rte_server_submit: server not running");
    }
    r->ticket = sv->next_ticket++;
    r->rep.t_submit = now_s(sv);
    sv->reqs[r->ticket] = r;
    K.queue.push_back(r);
    sv->max_queue = std::max<long long>(sv->max_queue, (long long)K.queue.size());
  }
  sv->cv_work.notify_one();
  *ticket = r->ticket;
  return RTE_OK;
}

extern "C" int rte_server_wait(rte_server_t sv, uint64_t ticket, double timeout_s, double* rho,
                               rte_serve_report* rep) {
  if (!sv) return fail(RTE_EINVAL, "rte_server_wait: null argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return fail(RTE_EINVAL, "rte_server_wait: unknown ticket");
  Request* r = it->second;
  const auto limit = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double>(std::max(timeout_s, 0.0)));
  while (!r->complete) {
    if (sv->cv_done.wait_until(lk, limit) == std::cv_status::timeout && !r->complete)
      return fail(RTE_ETIMEOUT, "rte_server_wait: not finished");
  }
  if (rep) *rep = r->rep;
  if (rho && !r->rho.empty()) std::memcpy(rho, r->rho.data(), sizeof(double) * r->rho.size());
  const int status = r->rep.status;
  const std::string msg = sv->error_msg;
  sv->reqs.erase(it);
  delete r;
  if (status == RTE_OK || status == RTE_ENOCONV) return status;
  return fail(status, "request failed: " + msg);
}

extern "C" int rte_server_stats(rte_server_t sv, double* out) {
  if (!sv || !out) return fail(RTE_EINVAL, "rte_server_stats: null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  long long queued = 0;
  for (auto* K : sv->buckets) queued += (long long)K->queue.size();
  out[0] = (double)sv->launches.load();
  out[1] = (double)sv->admitted.load();
  out[2] = (double)sv->completed;
  out[3] = (double)queued;
  out[4] = (double)sv->max_queue;
  out[5] = (double)sv->max_running.load();
  out[6] = 1e-9 * (double)sv->busy_ns.load();
  out[7] = sv->started ? now_s(sv) : 0.0;
  return RTE_OK;
}

extern "C" int rte_server_destroy(rte_server_t sv) {
  if (!sv) return RTE_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (auto* K : sv->buckets) {
      for (Request* r : K->queue) {
        r->rep.status = RTE_ESTATE;
        r->complete = true;
      }
      K->queue.clear();
    }
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  DeviceGuard g(sv->device);
  for (auto* K : sv->buckets)
    if (K->st) cudaStreamSynchronize(K->st);
  delete sv;
  return RTE_OK;
}
