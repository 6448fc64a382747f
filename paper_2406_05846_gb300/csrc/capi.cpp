// C ABI: errors, problem descriptions and the relaxation builder.
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>

#include "internal.h"

namespace {
thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_h2d{0}, g_d2h{0};
thread_local int64_t t_launches = 0;  // launches issued by this host thread
}  // namespace

namespace strom {
void set_error(const std::string& msg) { g_err = msg; }
void count_launches(int64_t n) {
  g_launches.fetch_add((uint64_t)n);
  t_launches += n;
}
int64_t thread_launch_count() { return t_launches; }
void count_h2d(uint64_t b) { g_h2d.fetch_add(b); }
void count_d2h(uint64_t b) { g_d2h.fetch_add(b); }
}  // namespace strom

extern "C" uint64_t strom_launch_count(void) { return g_launches.load(); }
extern "C" void strom_transfer_bytes(uint64_t* h2d, uint64_t* d2h) {
  if (h2d) *h2d = g_h2d.load();
  if (d2h) *d2h = g_d2h.load();
}

using namespace strom;

extern "C" const char* strom_last_error(void) { return g_err.c_str(); }
extern "C" const char* strom_version(void) { return "strom-gb300 0.1 (sm_103a)"; }

namespace {
Poly copy_poly(const strom_poly& q, int nv, int max_deg, const char* what) {
  if (q.nterms < 0 || (q.nterms > 0 && (!q.coef || !q.expo)))
    throw std::invalid_argument(std::string(what) + ": bad term arrays");
  Poly p;
  p.coef.assign(q.coef, q.coef + q.nterms);
  p.expo.assign(q.expo, q.expo + (size_t)q.nterms * nv);
  for (double c : p.coef)
    if (!std::isfinite(c)) throw std::invalid_argument(std::string(what) + ": non-finite coefficient");
  if (p.degree(nv) > max_deg) throw std::invalid_argument(std::string(what) + ": degree too high");
  return p;
}
}  // namespace

extern "C" int strom_problem_create(const strom_problem_desc* d, strom_problem** out) {
  try {
    if (!d || !out) throw std::invalid_argument("null argument");
    if (d->N < 1 || d->dx < 1 || d->du < 0 || !d->cliques) throw std::invalid_argument("N >= 1, dx >= 1, du >= 0 required");
    if (d->kappa != 2) throw std::invalid_argument("relaxation order kappa must be 2");
    if (!(d->R > 0)) throw std::invalid_argument("bound R must be positive");
    const int nv = 2 * d->dx + d->du;
    // the builder takes cliques of up to 21 variables (moment blocks up to
    // s(21, 2) = 253); the solver's PSD kernels take blocks up to 160, i.e.
    // cliques of up to 16 variables, and strom_solver_create checks that
    if (nv > 21) throw std::invalid_argument("at most 21 variables per clique");
    std::unique_ptr<strom_problem> p(new strom_problem());
    p->p.N = d->N; p->p.dx = d->dx; p->p.du = d->du; p->p.kappa = d->kappa; p->p.R = d->R;
    for (int k = 0; k < d->N; ++k) {
      const strom_clique& c = d->cliques[k];
      CliqueData cd;
      cd.f = copy_poly(c.f, nv, 2 * d->kappa, "objective");
      if (c.ng < 0 || c.nh < 0 || (c.ng > 0 && !c.g) || (c.nh > 0 && !c.h))
        throw std::invalid_argument("bad constraint arrays");
      for (int i = 0; i < c.ng; ++i) {
        cd.g.push_back(copy_poly(c.g[i], nv, 2, "inequality"));
        if (cd.g.back().degree(nv) < 1) throw std::invalid_argument("inequality of degree 0");
      }
      for (int j = 0; j < c.nh; ++j) cd.h.push_back(copy_poly(c.h[j], nv, 2 * d->kappa, "equality"));
      p->p.cl.push_back(std::move(cd));
    }
    *out = p.release();
    return STROM_OK;
  } catch (const std::exception& e) {
    set_error(std::string("strom_problem_create: ") + e.what());
    return STROM_ERR_INVALID;
  }
}

extern "C" void strom_problem_destroy(strom_problem* p) { delete p; }

extern "C" int strom_relax(const strom_problem* p, strom_sdp** out) {
  try {
    if (!p || !out) throw std::invalid_argument("null argument");
    std::unique_ptr<strom_sdp> s(new strom_sdp());
    s->s = build_relaxation(p->p);
    *out = s.release();
    return STROM_OK;
  } catch (const std::bad_alloc&) {
    set_error("strom_relax: out of host memory");
    return STROM_ERR_OOM;
  } catch (const std::exception& e) {
    set_error(std::string("strom_relax: ") + e.what());
    return STROM_ERR_INVALID;
  }
}

extern "C" int strom_sdp_info_get(const strom_sdp* s, strom_sdp_info* info) {
  if (!s || !info) {
    set_error("strom_sdp_info_get: null argument");
    return STROM_ERR_INVALID;
  }
  const Sdp& q = *s->s;
  info->N = q.N;
  info->nv = q.nv;
  info->nblocks = (int32_t)q.block_n.size();
  info->nsvec = q.nsvec;
  info->m = q.m();
  info->nnz = q.nnz();
  for (int k = 0; k < 5; ++k) info->rows_by_kind[k] = 0;
  for (int8_t k : q.row_kind) info->rows_by_kind[k]++;
  return STROM_OK;
}

extern "C" int strom_sdp_export(const strom_sdp* s, int32_t* block_n, int64_t* block_off, int8_t* block_kind,
                                int32_t* block_clique, double* C, int64_t* rowptr, int32_t* col, double* val,
                                double* b, int8_t* row_kind, int32_t* row_clique) {
  if (!s) {
    set_error("strom_sdp_export: null sdp");
    return STROM_ERR_INVALID;
  }
  const Sdp& q = *s->s;
  auto cp = [](auto* dst, const auto& v) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  cp(block_n, q.block_n);
  cp(block_off, q.block_off);
  cp(block_kind, q.block_kind);
  cp(block_clique, q.block_clique);
  cp(C, q.C);
  cp(rowptr, q.rowptr);
  cp(col, q.col);
  cp(val, q.val);
  cp(b, q.b);
  cp(row_kind, q.row_kind);
  cp(row_clique, q.row_clique);
  return STROM_OK;
}

extern "C" void strom_sdp_destroy(strom_sdp* s) {
  if (s) delete s->s;
  delete s;
}
