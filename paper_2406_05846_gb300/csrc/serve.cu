// Serving by continuous batching: a FIFO of solve requests fed into the
// slots of one batched solver. Finished requests free their slot at once,
// so a slow request never holds up the others.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <deque>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "solver_impl.cuh"
#include "warm.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  std::vector<double> val, b, C, X0, S0;
  std::vector<double> key;  // warm-start key (empty: not keyed)
  bool has_prob = false;
  strom::Problem prob;
  double t_submit = 0.0;
  double t_admit = 0.0;
};

struct Done {
  strom_result r{};
  strom_certificate c{};
  bool has_c = false;
  double latency = 0.0;   // submit -> retirement
  double service = 0.0;   // admission -> retirement
};

}  // namespace

struct strom_batch {
  strom_solver* s = nullptr;
  int slots = 0;
  int64_t nsvec = 0, m = 0, nnz = 0;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<int64_t> at_perm;   // A^T order -> CSR entry, inside one instance
  std::vector<double> tmpl_val;   // template's A values (the shared factor of cliques 2..N comes from them)
  std::vector<int32_t> row_clique;
  std::vector<int8_t> row_kind;
  std::deque<Request> queue;
  std::vector<int64_t> slot_ticket;
  std::vector<Request> slot_req;
  std::unordered_map<uint64_t, Done> done;
  uint64_t next = 1;
  strom_warm* warm = nullptr;  // warm-start store for keyed requests (not owned)
  bool record = false;         // add converged keyed requests to it
  ~strom_batch() { strom_solver_destroy(s); }
};

namespace {

template <typename F>
int guard(F&& f) {
  try {
    return f();
  } catch (const StatusError& e) {
    set_error(e.what());
    return e.status;
  } catch (const CudaError& e) {
    set_error(e.what());
    return STROM_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return STROM_ERR_OOM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return STROM_ERR_INVALID;
  }
}

void admit(strom_batch* B) {
  NvtxRange nv("strom.batch.admit");
  strom_solver* s = B->s;
  std::vector<int> adm;
  for (int i = 0; i < B->slots && !B->queue.empty(); ++i) {
    if (B->slot_ticket[i] >= 0) continue;
    Request rq = std::move(B->queue.front());
    B->queue.pop_front();
    cudaStream_t st = s->stream;
    const int64_t no = s->inst_nnz_off[i];
    copy_h2d(s->val.p + no, rq.val.data(), sizeof(double) * B->nnz, st);
    std::vector<double> at(B->nnz);
    for (int64_t k = 0; k < B->nnz; ++k) at[k] = rq.val[B->at_perm[k]];
    copy_h2d(s->atval.p + no, at.data(), sizeof(double) * B->nnz, st);
    copy_h2d(s->b.p + s->row_off[i], rq.b.data(), sizeof(double) * B->m, st);
    copy_h2d(s->C.p + s->svec_off[i], rq.C.data(), sizeof(double) * B->nsvec, st);
    double nc = 0.0;
    for (double c : rq.C) nc += c * c;
    nc = std::sqrt(nc);
    copy_h2d(s->norm_C.p + i, &nc, sizeof(double), st);
    STROM_CUDA(cudaStreamSynchronize(st));  // `at` and `nc` are stack data
    s->meta[i].b = rq.b;
    rq.t_admit = now_s();
    B->slot_ticket[i] = (int64_t)rq.ticket;
    B->slot_req[i] = std::move(rq);
    adm.push_back(i);
  }
  if (adm.empty()) return;
  factor_instances(s, adm);
  reset_instances(s, adm);
  std::vector<double> wsig(s->ninst, 0.0);
  bool any_warm = false;
  for (int i : adm) {
    const Request& rq = B->slot_req[i];
    if (!rq.X0.empty()) copy_h2d(s->X.p + s->svec_off[i], rq.X0.data(), sizeof(double) * B->nsvec, s->stream);
    if (!rq.S0.empty()) copy_h2d(s->S.p + s->svec_off[i], rq.S0.data(), sizeof(double) * B->nsvec, s->stream);
    if (!rq.key.empty() && B->warm &&
        warm_apply(B->warm, rq.key.data(), s->X.p + s->svec_off[i], s->S.p + s->svec_off[i], &wsig[i], s->stream))
      any_warm = true;
  }
  if (any_warm) {
    std::vector<double> sg(s->ninst);
    copy_d2h(sg.data(), s->sigma.p, sizeof(double) * s->ninst, s->stream);
    STROM_CUDA(cudaStreamSynchronize(s->stream));
    for (int i : adm)
      if (wsig[i] > 0) sg[i] = wsig[i];
    copy_h2d(s->sigma.p, sg.data(), sizeof(double) * s->ninst, s->stream);
  }
  STROM_CUDA(cudaStreamSynchronize(s->stream));
}

void retire(strom_batch* B) {
  NvtxRange nv("strom.batch.retire");
  strom_solver* s = B->s;
  const int n = s->ninst;
  std::vector<uint8_t> flag(n);
  std::vector<int32_t> it(n);
  std::vector<double> stats(8 * (size_t)n), sg(n);
  copy_d2h(flag.data(), s->inst_flag.p, n, s->stream);
  copy_d2h(it.data(), s->iters.p, sizeof(int32_t) * n, s->stream);
  copy_d2h(stats.data(), s->stats.p, sizeof(double) * stats.size(), s->stream);
  copy_d2h(sg.data(), s->sigma.p, sizeof(double) * n, s->stream);
  STROM_CUDA(cudaStreamSynchronize(s->stream));
  std::vector<int> fin, cert;
  for (int i = 0; i < B->slots; ++i)
    if (B->slot_ticket[i] >= 0 && flag[i] != 0) {
      fin.push_back(i);
      if (B->slot_req[i].has_prob) cert.push_back(i);
    }
  if (fin.empty()) return;
  std::vector<double> lamX, topX, lamZ, topZ;
  std::vector<int64_t> lo;
  if (!cert.empty()) {
    eig_instances(s, cert, false, lamX, topX, lo);
    eig_instances(s, cert, true, lamZ, topZ, lo);
  }
  const double t = now_s();
  for (int i : fin) {
    Done d;
    const double* st = stats.data() + 8 * (size_t)i;
    d.r.status = flag[i] == 1 ? STROM_OK : flag[i] == 2 ? STROM_ERR_NUMERICAL : STROM_MAXITER;
    d.r.iterations = it[i];
    d.r.eta_p = st[0]; d.r.eta_d = st[1]; d.r.eta_g = st[2]; d.r.pobj = st[3]; d.r.dobj = st[4];
    d.r.sigma = sg[i];
    d.r.m_kept = s->m_kept[i];
    const Request& rq = B->slot_req[i];
    if (rq.has_prob) {
      const InstMeta& mt = s->meta[i];
      certify_one(rq.prob, mt.block_n, mt.block_kind, mt.block_clique, lo.data() + s->inst_blk_off[i], lamX.data(),
                  topX.data(), lamZ.data(), st[4], 1e-4, 1e-2, &d.c, nullptr, nullptr);
      d.has_c = true;
    }
    if (flag[i] == 1 && B->warm && B->record && !rq.key.empty())
      warm_append(B->warm, rq.key.data(), s->X.p + s->svec_off[i], s->S.p + s->svec_off[i], sg[i], s->stream);
    d.latency = t - rq.t_submit;
    d.service = t - rq.t_admit;
    B->done[rq.ticket] = d;
    B->slot_ticket[i] = -1;
  }
}

}  // namespace

namespace {

// Device footprint of a batch of this structure: a solver of one slot and one
// of two slots are built (set-up included: row reduction and factorisation)
// with the allocation tally attached. The second slot's bytes are the bytes
// of every further slot (every slot but the first refers to the first one's
// shared tail factor); the peak minus the resident bytes is the transient
// scratch of the set-up.
void slot_bytes(const strom_sdp* tmpl, const strom_options* opt, int64_t* base, int64_t* per_slot,
                int64_t* transient) {
  int64_t live[2], peak[2];
  for (int k = 0; k < 2; ++k) {
    AllocTally t;
    AllocTally* prev = g_alloc_tally;
    g_alloc_tally = &t;
    strom_solver* s = nullptr;
    const strom_sdp* v[2] = {tmpl, tmpl};
    const int st = strom_solver_create(v, k + 1, opt, &s);
    g_alloc_tally = prev;
    live[k] = t.live;
    peak[k] = t.peak;
    strom_solver_destroy(s);
    if (st != STROM_OK) throw StatusError(st, std::string("strom_batch_slot_bytes: ") + strom_last_error());
  }
  *per_slot = std::max<int64_t>(1, live[1] - live[0]);
  *base = std::max<int64_t>(0, live[0] - *per_slot);
  *transient = std::max<int64_t>(0, std::max(peak[0] - live[0], peak[1] - live[1]));
}

}  // namespace

extern "C" int strom_batch_slot_bytes(const strom_sdp* tmpl, const strom_options* opt, int64_t* base_bytes,
                                      int64_t* slot_bytes_out, int64_t* transient_bytes) {
  return guard([&]() -> int {
    if (!tmpl || !tmpl->s || !slot_bytes_out) throw StatusError(STROM_ERR_INVALID, "strom_batch_slot_bytes: bad arguments");
    int64_t b = 0, p = 0, t = 0;
    slot_bytes(tmpl, opt, &b, &p, &t);
    if (base_bytes) *base_bytes = b;
    *slot_bytes_out = p;
    if (transient_bytes) *transient_bytes = t;
    return STROM_OK;
  });
}

extern "C" int strom_batch_create_budget(const strom_sdp* tmpl, int64_t budget_bytes, const strom_options* opt,
                                         strom_batch** out, int32_t* slots_out) {
  return guard([&]() -> int {
    if (!tmpl || !tmpl->s || !out || budget_bytes <= 0)
      throw StatusError(STROM_ERR_INVALID, "strom_batch_create_budget: bad arguments");
    size_t free_b = 0, total_b = 0;
    STROM_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if ((uint64_t)budget_bytes > (uint64_t)free_b)
      throw StatusError(STROM_ERR_OOM, "strom_batch_create_budget: budget of " + std::to_string(budget_bytes) +
                                           " bytes exceeds the device's free memory (" + std::to_string(free_b) +
                                           " bytes)");
    int64_t base = 0, per = 0, tr = 0;
    slot_bytes(tmpl, opt, &base, &per, &tr);
    const int64_t room = budget_bytes - base - tr;
    const int64_t slots = room > 0 ? room / per : 0;
    if (slots < 1)
      throw StatusError(STROM_ERR_INVALID, "strom_batch_create_budget: budget below one slot (" +
                                               std::to_string(base + tr + per) + " bytes)");
    if (slots > INT32_MAX) throw StatusError(STROM_ERR_INVALID, "strom_batch_create_budget: too many slots");
    const int st = strom_batch_create(tmpl, (int32_t)slots, opt, out);
    if (st == STROM_OK && slots_out) *slots_out = (int32_t)slots;
    return st;
  });
}

extern "C" int strom_batch_create(const strom_sdp* tmpl, int32_t slots, const strom_options* opt, strom_batch** out) {
  return guard([&]() -> int {
    if (!tmpl || !tmpl->s || slots < 1 || !out) throw StatusError(STROM_ERR_INVALID, "strom_batch_create: bad arguments");
    std::unique_ptr<strom_batch> B(new strom_batch());
    std::vector<const strom_sdp*> v(slots, tmpl);
    int st = strom_solver_create(v.data(), slots, opt, &B->s);
    if (st != STROM_OK) return st;
    const Sdp& q = *tmpl->s;
    B->slots = slots;
    B->nsvec = q.nsvec;
    B->m = q.m();
    B->nnz = q.nnz();
    B->rowptr = q.rowptr;
    B->col = q.col;
    B->tmpl_val = q.val;
    B->row_clique = q.row_clique;
    B->row_kind = q.row_kind;
    // A^T order of the entries of one instance (columns ascending, rows ascending)
    std::vector<int64_t> cnt(q.nsvec + 1, 0);
    for (int32_t c : q.col) cnt[c + 1]++;
    for (int64_t p = 0; p < q.nsvec; ++p) cnt[p + 1] += cnt[p];
    B->at_perm.assign(q.nnz(), 0);
    for (int64_t r = 0; r < q.m(); ++r)
      for (int64_t e = q.rowptr[r]; e < q.rowptr[r + 1]; ++e) B->at_perm[cnt[q.col[e]]++] = e;
    B->slot_ticket.assign(slots, -1);
    B->slot_req.resize(slots);
    // every slot starts empty
    STROM_CUDA(cudaMemsetAsync(B->s->inst_active.p, 0, slots, B->s->stream));
    STROM_CUDA(cudaStreamSynchronize(B->s->stream));
    *out = B.release();
    return STROM_OK;
  });
}

extern "C" void strom_batch_destroy(strom_batch* b) { delete b; }

namespace {

int submit(strom_batch* B, const strom_sdp* sdp, const strom_problem* problem, const double* X0, const double* S0,
           const double* key, uint64_t* ticket) {
  return guard([&]() -> int {
    if (!B || !sdp || !sdp->s || !ticket) throw StatusError(STROM_ERR_INVALID, "strom_batch_submit: bad arguments");
    const Sdp& q = *sdp->s;
    if (q.nsvec != B->nsvec || q.m() != B->m || q.nnz() != B->nnz || q.rowptr != B->rowptr || q.col != B->col)
      throw StatusError(STROM_ERR_INVALID, "strom_batch_submit: SDP structure differs from the batch template");
    if (B->s->shared_tail) {
      for (int64_t r = 0; r < B->m; ++r) {
        if (B->row_clique[r] == 0 && B->row_kind[r] != STROM_ROW_CONS) continue;
        for (int64_t e = B->rowptr[r]; e < B->rowptr[r + 1]; ++e)
          if (q.val[e] != B->tmpl_val[e])
            throw StatusError(STROM_ERR_INVALID, "strom_batch_submit: the batch shares the factor of cliques 2..N and "
                                                 "this request's constraints there differ from the template's "
                                                 "(create the batch with share_tail = 0)");
      }
    }
    Request rq;
    rq.ticket = B->next++;
    rq.val = q.val;
    rq.b = q.b;
    rq.C = q.C;
    if (problem) {
      rq.has_prob = true;
      rq.prob = problem->p;
    }
    if (X0) rq.X0.assign(X0, X0 + q.nsvec);
    if (S0) rq.S0.assign(S0, S0 + q.nsvec);
    if (key) {
      if (!B->warm) throw StatusError(STROM_ERR_INVALID, "strom_batch_submit_keyed: no warm-start store attached");
      for (int t = 0; t < B->warm->d; ++t)
        if (!std::isfinite(key[t])) throw StatusError(STROM_ERR_INVALID, "strom_batch_submit_keyed: non-finite key");
      rq.key.assign(key, key + B->warm->d);
    }
    rq.t_submit = now_s();
    *ticket = rq.ticket;
    B->queue.push_back(std::move(rq));
    return STROM_OK;
  });
}

}  // namespace

extern "C" int strom_batch_submit(strom_batch* B, const strom_sdp* sdp, const strom_problem* problem, const double* X0,
                                  const double* S0, uint64_t* ticket) {
  return submit(B, sdp, problem, X0, S0, nullptr, ticket);
}

extern "C" int strom_batch_submit_keyed(strom_batch* B, const strom_sdp* sdp, const strom_problem* problem,
                                        const double* key, uint64_t* ticket) {
  if (!key) {
    set_error("strom_batch_submit_keyed: null key");
    return STROM_ERR_INVALID;
  }
  return submit(B, sdp, problem, nullptr, nullptr, key, ticket);
}

extern "C" int strom_batch_set_warm(strom_batch* B, strom_warm* w, int32_t record) {
  return guard([&]() -> int {
    if (!B) throw StatusError(STROM_ERR_INVALID, "strom_batch_set_warm: null batch");
    if (w && w->nsvec != B->nsvec)
      throw StatusError(STROM_ERR_INVALID, "strom_batch_set_warm: the store's svec length differs from the batch's");
    B->warm = w;
    B->record = w && record != 0;
    return STROM_OK;
  });
}

extern "C" int strom_batch_step(strom_batch* B, int32_t iters, void* stream, int32_t* n_running, int32_t* n_queued) {
  return guard([&]() -> int {
    if (!B || iters < 0) throw StatusError(STROM_ERR_INVALID, "strom_batch_step: bad arguments");
    admit(B);
    int32_t act = 0;
    run_iterations(B->s, iters, (cudaStream_t)stream, &act);
    retire(B);
    admit(B);
    int run = 0;
    for (int64_t t : B->slot_ticket) run += t >= 0;
    if (n_running) *n_running = run;
    if (n_queued) *n_queued = (int32_t)B->queue.size();
    return STROM_OK;
  });
}

extern "C" int strom_batch_poll(strom_batch* B, uint64_t ticket, strom_result* r, strom_certificate* c,
                                double* latency_s, double* service_s) {
  return guard([&]() -> int {
    if (!B) throw StatusError(STROM_ERR_INVALID, "strom_batch_poll: null batch");
    auto it = B->done.find(ticket);
    if (it == B->done.end()) {
      if (ticket == 0 || ticket >= B->next) throw StatusError(STROM_ERR_INVALID, "strom_batch_poll: unknown ticket");
      return (int)STROM_PENDING;
    }
    if (r) *r = it->second.r;
    if (c && it->second.has_c) *c = it->second.c;
    if (latency_s) *latency_s = it->second.latency;
    if (service_s) *service_s = it->second.service;
    return STROM_OK;
  });
}
