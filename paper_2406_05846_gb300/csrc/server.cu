// Serving requests of several SDP structures (robots, horizons) behind one
// front, within one device-memory budget.
//
// A strom_batch serves one structure. The server keeps one batch per
// structure class and routes every request to its class. A class is the
// structure of the first request seen (rows, columns, blocks) and, when the
// options share the factor of cliques 2..N, that request's constraint values
// after the first clique as well: requests of the same structure whose later
// constraints differ (other obstacles, say) go to a second class of that
// structure whose batch factorises every slot in full.
//
// Memory: a class's batch is created on the first step after its first
// request arrives, with min(max_slots, what the remaining budget holds)
// slots, from its measured footprint (strom_batch_slot_bytes). When the
// budget holds no slot for a waiting class, idle batches of other classes
// (no request running or queued) are destroyed to make room; their finished
// results are kept by the server. Requests wait in host memory until their
// class has a batch.
//
// A step runs every batch that has work for the same number of iterations,
// each from its own host thread on its own stream, so the structures'
// iterations overlap on the device. The serving loop has no counterpart in
// the paper (its nearest use is the warm-started MPC loop of Sec. 5).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <exception>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Waiting {
  uint64_t ticket = 0;
  strom_sdp* sdp = nullptr;          // deep copies, freed once submitted to a batch
  strom_problem* prob = nullptr;
  double t_submit = 0.0;
};

struct Routed {
  int cls = -1;
  uint64_t bticket = 0;
  double wait = 0.0;   // seconds between the server's submit and the batch's
};

struct Finished {
  strom_result r{};
  strom_certificate c{};
  bool has_c = false;
  double latency = 0.0, service = 0.0;
};

struct Class {
  strom_sdp* tmpl = nullptr;  // copy of the first request (structure, and tail values when shared)
  bool shared = false;        // its batch shares the factor of cliques 2..N
  strom_batch* batch = nullptr;
  int32_t slots = 0;
  bool sized = false;
  int64_t base = 0, per = 0, transient = 0, reserved = 0;
  int32_t running = 0, queued = 0;
  std::deque<Waiting> waiting;
  std::vector<uint64_t> tickets;  // server tickets routed to the current batch
  uint64_t batches_made = 0;
};

void free_waiting(Waiting& w) {
  if (w.sdp) strom_sdp_destroy(w.sdp);
  if (w.prob) strom_problem_destroy(w.prob);
  w.sdp = nullptr;
  w.prob = nullptr;
}

}  // namespace

struct strom_server {
  strom_options opt{};
  int64_t budget = 0, used = 0;
  int32_t max_slots = 0;
  std::vector<std::unique_ptr<Class>> cls;
  std::unordered_map<uint64_t, int> waiting_cls;
  std::unordered_map<uint64_t, Routed> routed;
  std::unordered_map<uint64_t, Finished> done;
  uint64_t next = 1;
  ~strom_server() {
    for (auto& c : cls) {
      for (auto& w : c->waiting) free_waiting(w);
      if (c->batch) strom_batch_destroy(c->batch);
      if (c->tmpl) strom_sdp_destroy(c->tmpl);
    }
  }
};

namespace {

using strom::StatusError;

template <typename F>
int guard(F&& f) {
  try {
    return f();
  } catch (const StatusError& e) {
    strom::set_error(e.what());
    return e.status;
  } catch (const strom::CudaError& e) {
    strom::set_error(e.what());
    return STROM_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    strom::set_error("host allocation failed");
    return STROM_ERR_OOM;
  } catch (const std::exception& e) {
    strom::set_error(e.what());
    return STROM_ERR_INVALID;
  }
}

bool same_rows(const strom::Sdp& a, const strom::Sdp& b) {
  return a.nsvec == b.nsvec && a.m() == b.m() && a.nnz() == b.nnz() && a.block_n == b.block_n &&
         a.rowptr == b.rowptr && a.col == b.col && a.row_kind == b.row_kind && a.row_clique == b.row_clique;
}

// the constraint values a shared tail factor depends on: every row outside
// the first clique, and the first clique's consensus rows
bool same_tail(const strom::Sdp& a, const strom::Sdp& b) {
  for (int64_t r = 0; r < a.m(); ++r) {
    if (a.row_clique[r] == 0 && a.row_kind[r] != STROM_ROW_CONS) continue;
    for (int64_t e = a.rowptr[r]; e < a.rowptr[r + 1]; ++e)
      if (a.val[e] != b.val[e]) return false;
  }
  return true;
}

strom_sdp* copy_sdp(const strom_sdp* s) { return new strom_sdp{new strom::Sdp(*s->s)}; }

int class_of(strom_server* S, const strom_sdp* sdp) {
  const strom::Sdp& q = *sdp->s;
  int general = -1;
  bool structure_seen = false;
  for (size_t c = 0; c < S->cls.size(); ++c) {
    const Class& k = *S->cls[c];
    if (!same_rows(*k.tmpl->s, q)) continue;
    structure_seen = true;
    if (!k.shared) general = (int)c;
    else if (same_tail(*k.tmpl->s, q)) return (int)c;
  }
  if (general >= 0) return general;
  auto k = std::make_unique<Class>();
  k->tmpl = copy_sdp(sdp);
  k->shared = S->opt.share_tail != 0 && !structure_seen;
  S->cls.push_back(std::move(k));
  return (int)S->cls.size() - 1;
}

strom_options class_options(const strom_server* S, const Class& k) {
  strom_options o = S->opt;
  o.share_tail = k.shared ? 1 : 0;
  return o;
}

void harvest(strom_server* S, int c) {
  Class& k = *S->cls[c];
  std::vector<uint64_t> keep;
  for (uint64_t t : k.tickets) {
    const Routed& r = S->routed[t];
    Finished f;
    const int st = strom_batch_poll(k.batch, r.bticket, &f.r, &f.c, &f.latency, &f.service);
    if (st == STROM_PENDING) {
      keep.push_back(t);
      continue;
    }
    if (st != STROM_OK) throw StatusError(st, std::string("strom_server: ") + strom_last_error());
    f.has_c = f.c.max_ratio == f.c.max_ratio;
    f.latency += r.wait;
    S->done[t] = f;
    S->routed.erase(t);
  }
  k.tickets.swap(keep);
}

void evict(strom_server* S, int c) {
  Class& k = *S->cls[c];
  harvest(S, c);
  if (!k.tickets.empty()) throw StatusError(STROM_ERR_INVALID, "strom_server: evicting a batch with requests");
  strom_batch_destroy(k.batch);
  k.batch = nullptr;
  k.slots = 0;
  S->used -= k.reserved;
  k.reserved = 0;
}

// a batch for class c if the budget (after evicting idle batches) holds a slot
void provision(strom_server* S, int c) {
  Class& k = *S->cls[c];
  if (k.batch || k.waiting.empty()) return;
  const strom_options o = class_options(S, k);
  if (!k.sized) {
    const int st = strom_batch_slot_bytes(k.tmpl, &o, &k.base, &k.per, &k.transient);
    if (st != STROM_OK) throw StatusError(st, std::string("strom_server: ") + strom_last_error());
    k.sized = true;
  }
  const int64_t fixed = k.base + k.transient;
  if (fixed + k.per > S->budget) {
    // not one slot of this structure fits the whole budget: its requests
    // finish at once with STROM_ERR_OOM instead of waiting forever
    const double t = now_s();
    for (Waiting& w : k.waiting) {
      Finished f;
      f.r.status = STROM_ERR_OOM;
      f.latency = t - w.t_submit;
      S->done[w.ticket] = f;
      S->waiting_cls.erase(w.ticket);
      free_waiting(w);
    }
    k.waiting.clear();
    return;
  }
  auto fits = [&]() { return S->budget - S->used - fixed >= k.per; };
  if (!fits()) {
    for (size_t e = 0; e < S->cls.size() && !fits(); ++e) {
      Class& o2 = *S->cls[e];
      if ((int)e == c || !o2.batch || o2.running > 0 || o2.queued > 0 || !o2.waiting.empty()) continue;
      evict(S, (int)e);
    }
  }
  if (!fits()) return;  // waits for memory
  int64_t slots = (S->budget - S->used - fixed) / k.per;
  slots = std::min<int64_t>(slots, S->max_slots);
  strom_batch* b = nullptr;
  const int st = strom_batch_create(k.tmpl, (int32_t)slots, &o, &b);
  if (st != STROM_OK) throw StatusError(st, std::string("strom_server: ") + strom_last_error());
  k.batch = b;
  k.slots = (int32_t)slots;
  k.reserved = fixed + slots * k.per;
  S->used += k.reserved;
  ++k.batches_made;
}

void route_waiting(strom_server* S, int c) {
  Class& k = *S->cls[c];
  if (!k.batch) return;
  const double t = now_s();
  while (!k.waiting.empty()) {
    Waiting& w = k.waiting.front();
    uint64_t bt = 0;
    const int st = strom_batch_submit(k.batch, w.sdp, w.prob, nullptr, nullptr, &bt);
    if (st != STROM_OK) throw StatusError(st, std::string("strom_server: ") + strom_last_error());
    S->routed[w.ticket] = Routed{c, bt, t - w.t_submit};
    S->waiting_cls.erase(w.ticket);
    k.tickets.push_back(w.ticket);
    ++k.queued;
    free_waiting(w);
    k.waiting.pop_front();
  }
}

}  // namespace

extern "C" int strom_server_create(int64_t budget_bytes, int32_t max_slots, const strom_options* opt,
                                   strom_server** out) {
  return guard([&]() -> int {
    if (budget_bytes <= 0 || max_slots < 1 || !out) throw StatusError(STROM_ERR_INVALID, "strom_server_create: bad arguments");
    size_t free_b = 0, total_b = 0;
    STROM_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if ((uint64_t)budget_bytes > (uint64_t)free_b)
      throw StatusError(STROM_ERR_OOM, "strom_server_create: budget of " + std::to_string(budget_bytes) +
                                           " bytes exceeds the device's free memory (" + std::to_string(free_b) +
                                           " bytes)");
    std::unique_ptr<strom_server> S(new strom_server());
    if (opt) S->opt = *opt;
    else strom_options_default(&S->opt);
    S->budget = budget_bytes;
    S->max_slots = max_slots;
    *out = S.release();
    return STROM_OK;
  });
}

extern "C" void strom_server_destroy(strom_server* S) { delete S; }

extern "C" int strom_server_submit(strom_server* S, const strom_sdp* sdp, const strom_problem* problem,
                                   uint64_t* ticket) {
  return guard([&]() -> int {
    if (!S || !sdp || !sdp->s || !ticket) throw StatusError(STROM_ERR_INVALID, "strom_server_submit: bad arguments");
    const int c = class_of(S, sdp);
    Waiting w;
    w.ticket = S->next++;
    w.sdp = copy_sdp(sdp);
    if (problem) w.prob = new strom_problem{problem->p};
    w.t_submit = now_s();
    S->waiting_cls[w.ticket] = c;
    *ticket = w.ticket;
    S->cls[c]->waiting.push_back(w);
    return STROM_OK;
  });
}

extern "C" int strom_server_step(strom_server* S, int32_t iters, void* stream, int32_t* n_running,
                                 int32_t* n_waiting) {
  return guard([&]() -> int {
    if (!S || iters < 0) throw StatusError(STROM_ERR_INVALID, "strom_server_step: bad arguments");
    const int nc = (int)S->cls.size();
    for (int c = 0; c < nc; ++c) {
      provision(S, c);
      route_waiting(S, c);
    }
    // every batch with work steps at once, one host thread each
    std::vector<int> work;
    for (int c = 0; c < nc; ++c)
      if (S->cls[c]->batch && (S->cls[c]->running > 0 || S->cls[c]->queued > 0)) work.push_back(c);
    std::vector<int> st(work.size(), STROM_OK);
    std::vector<std::string> err(work.size());
    int dev = 0;
    STROM_CUDA(cudaGetDevice(&dev));
    std::vector<std::thread> th;
    for (size_t t = 0; t < work.size(); ++t)
      th.emplace_back([&, t] {
        cudaSetDevice(dev);
        Class& k = *S->cls[work[t]];
        st[t] = strom_batch_step(k.batch, iters, stream, &k.running, &k.queued);
        if (st[t] != STROM_OK) err[t] = strom_last_error();
      });
    for (auto& x : th) x.join();
    for (size_t t = 0; t < work.size(); ++t)
      if (st[t] != STROM_OK) throw StatusError(st[t], "strom_server_step: " + err[t]);
    int32_t run = 0, wait = 0;
    for (int c = 0; c < nc; ++c) {
      Class& k = *S->cls[c];
      if (k.batch) harvest(S, c);
      run += k.running + k.queued;
      wait += (int32_t)k.waiting.size();
    }
    if (n_running) *n_running = run;
    if (n_waiting) *n_waiting = wait;
    return STROM_OK;
  });
}

extern "C" int strom_server_poll(strom_server* S, uint64_t ticket, strom_result* r, strom_certificate* c,
                                 double* latency_s, double* service_s) {
  return guard([&]() -> int {
    if (!S) throw StatusError(STROM_ERR_INVALID, "strom_server_poll: null server");
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
      if (ticket == 0 || ticket >= S->next) throw StatusError(STROM_ERR_INVALID, "strom_server_poll: unknown ticket");
      return (int)STROM_PENDING;
    }
    if (r) *r = it->second.r;
    if (c && it->second.has_c) *c = it->second.c;
    if (latency_s) *latency_s = it->second.latency;
    if (service_s) *service_s = it->second.service;
    return STROM_OK;
  });
}

extern "C" int strom_server_info(const strom_server* S, int32_t cap, strom_server_class* out, int32_t* nclass,
                                 int64_t* used_bytes) {
  return guard([&]() -> int {
    if (!S || cap < 0 || (cap > 0 && !out)) throw StatusError(STROM_ERR_INVALID, "strom_server_info: bad arguments");
    const int n = (int)S->cls.size();
    for (int c = 0; c < std::min(n, cap); ++c) {
      const Class& k = *S->cls[c];
      strom_server_class& o = out[c];
      std::memset(&o, 0, sizeof(o));
      o.N = k.tmpl->s->N;
      o.nsvec = k.tmpl->s->nsvec;
      o.m = k.tmpl->s->m();
      o.shared_tail = k.shared ? 1 : 0;
      o.slots = k.slots;
      o.running = k.running;
      o.queued = k.queued;
      o.waiting = (int32_t)k.waiting.size();
      o.slot_bytes = k.per;
      o.reserved_bytes = k.reserved;
      o.batches_created = (int32_t)k.batches_made;
    }
    if (nclass) *nclass = n;
    if (used_bytes) *used_bytes = S->used;
    return STROM_OK;
  });
}
