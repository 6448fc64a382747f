// The sparse factor inside the batched solver: symbolic patterns (one per
// row structure, shared by the instances that have it), value storage,
// factorisation of a set of instances (the whole batch at set-up, single
// slots at serving admission) and the y-solve with it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <exception>
#include <mutex>
#include <string>
#include <thread>

#include "solver_impl.cuh"

namespace strom {
namespace {

void upload_solve_arrays(SpPatHost& P, cudaStream_t st) {
  const SpSymbolic& y = *P.sym;
  P.fptr.upload(y.fptr.data(), y.fptr.size(), st);
  P.bptr.upload(y.bptr.data(), y.bptr.size(), st);
  if (y.fcol.empty()) {
    P.fcol.alloc(1);
    P.brow.alloc(1);
  } else {
    P.fcol.upload(y.fcol.data(), y.fcol.size(), st);
    P.brow.upload(y.brow.data(), y.brow.size(), st);
  }
  P.fsplit.upload(y.fsplit.data(), y.fsplit.size(), st);
  P.bsplit.upload(y.bsplit.data(), y.bsplit.size(), st);
  P.fgrp.upload(y.fgrp.data(), y.fgrp.size(), st);
  P.bgrp.upload(y.bgrp.data(), y.bgrp.size(), st);
  P.grp_ptr.upload(y.grp_ptr.data(), y.grp_ptr.size(), st);
  P.blk_grp.upload(y.blk_grp.data(), y.blk_grp.size(), st);
  P.can_local.upload(y.can_local.data(), y.can_local.size(), st);
}

// the host copies of the index arrays the device now holds (large for long
// horizons; the factorisation needs only fmap and the S entries on the host)
void release_host_indices(SpSymbolic& y) {
  std::vector<int32_t>().swap(y.fcol);
  std::vector<int32_t>().swap(y.brow);
}

void upload_fac_arrays(SpPatHost& P, cudaStream_t st) {
  if (P.fac_on_device) return;
  const SpSymbolic& y = *P.sym;
  if (y.fmap.empty()) P.fmap.alloc(1);
  else P.fmap.upload(y.fmap.data(), y.fmap.size(), st);
  P.s_ri.upload(y.s_ri.data(), y.s_ri.size(), st);
  P.s_rj.upload(y.s_rj.data(), y.s_rj.size(), st);
  P.s_dst.upload(y.s_dst.data(), y.s_dst.size(), st);
  P.fac_on_device = true;
}

void drop_fac_arrays(SpPatHost& P) {
  P.fmap.release();
  P.s_ri.release(); P.s_rj.release(); P.s_dst.release();
  P.fac_on_device = false;
}

size_t fac_bytes(const SpSymbolic& y) { return y.fmap.size() * 4 + y.s_ri.size() * (4 + 4 + 8); }

void refresh_pattern_views(strom_solver* s) {
  SparseState& sp = s->sp;
  sp.pats_h.resize(sp.pats.size());
  for (size_t p = 0; p < sp.pats.size(); ++p) {
    const SpPatHost& P = *sp.pats[p];
    const SpSymbolic& y = *P.sym;
    SpPatDev v{};
    v.n = y.n; v.n_tail = y.n_tail; v.ngroups = y.ngroups; v.max_group = y.max_group;
    v.fptr = P.fptr.p; v.fcol = P.fcol.p; v.bptr = P.bptr.p; v.brow = P.brow.p; v.grp_ptr = P.grp_ptr.p;
    v.can_local = P.can_local.p; v.fsplit = P.fsplit.p; v.bsplit = P.bsplit.p;
    v.fgrp = P.fgrp.p; v.bgrp = P.bgrp.p; v.blk_grp = P.blk_grp.p;
    v.nblk = y.nblk; v.tail_blk = y.blk_grp[y.ngroups - 1];
    v.fmap = P.fmap.p; v.s_ri = P.s_ri.p; v.s_rj = P.s_rj.p; v.s_dst = P.s_dst.p;
    v.ns = (int64_t)y.s_dst.size(); v.ns_tail = y.ns_tail;
    v.tail_fwd = y.fptr[y.n_tail]; v.tail_bwd = y.bptr[y.n_tail];
    sp.pats_h[p] = v;
  }
  sp.pats_dev.upload(sp.pats_h.data(), sp.pats_h.size(), s->stream);
  sp.dev.pats = sp.pats_dev.p;
  STROM_CUDA(cudaStreamSynchronize(s->stream));
}

int pick_tile(const strom_solver* s) {
  const SparseState& sp = s->sp;
  int R = 1;
  if (s->shared_tail) {
    const int sms = 152;
    R = s->ninst >= 4 * sms ? 4 : s->ninst >= 2 * sms ? 2 : 1;
    if (const char* e = std::getenv("STROM_TILE_R")) {
      const int v = std::atoi(e);
      if (v == 1 || v == 2 || v == 4 || v == 8) R = v;
    }
  }
  while (R > 1 && sizeof(double) * 2 * (size_t)R * sp.dev.max_group > 200 * 1024) R /= 2;
  return R;
}

}  // namespace

void sparse_setup(strom_solver* s, const strom_sdp* const* sdps, int count) {
  SparseState& sp = s->sp;
  cudaStream_t st = s->stream;
  // ---- patterns: one per row structure
  sp.inst_pat.assign(count, -1);
  std::vector<int> rep;
  for (int i = 0; i < count; ++i) {
    if (s->shared_tail && i > 0) { sp.inst_pat[i] = 0; continue; }
    for (size_t p = 0; p < rep.size() && sp.inst_pat[i] < 0; ++p)
      if (same_structure(*sdps[rep[p]]->s, *sdps[i]->s)) sp.inst_pat[i] = (int32_t)p;
    if (sp.inst_pat[i] < 0) {
      sp.inst_pat[i] = (int32_t)rep.size();
      rep.push_back(i);
    }
  }
  // ---- symbolic analyses, in parallel over patterns
  const auto t0 = std::chrono::steady_clock::now();
  sp.pats.resize(rep.size());
  for (auto& P : sp.pats) P.reset(new SpPatHost());
  {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nth = (int)std::min<size_t>(rep.size(), hw);
    std::exception_ptr err;
    std::mutex mu;
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t)
      th.emplace_back([&, t] {
        for (size_t p = t; p < rep.size(); p += nth) {
          try {
            sp.pats[p]->sym.reset(sparse_symbolic(*sdps[rep[p]]->s));
          } catch (...) {
            std::lock_guard<std::mutex> lk(mu);
            if (!err) err = std::current_exception();
          }
        }
      });
    for (auto& x : th) x.join();
    if (err) std::rethrow_exception(err);
  }
  sp.symbolic_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  // ---- value storage and per-instance views
  int max_col = 0, max_span = 0, max_group = 0;
  size_t fac_total = 0;
  for (auto& P : sp.pats) {
    const SpSymbolic& y = *P->sym;
    if (y.ngroups > kSpMaxGroups)
      throw StatusError(STROM_ERR_INVALID, "sparse factor: horizons above " + std::to_string(kSpMaxGroups) +
                                               " cliques are not supported");
    max_col = std::max(max_col, y.max_col);
    max_span = std::max(max_span, y.max_span);
    max_group = std::max(max_group, y.max_group);
    sp.max_n = std::max(sp.max_n, y.n);
    fac_total += fac_bytes(y);
  }
  sp.inst_h.assign(count, SpInstDev{});
  int64_t af = 0, ab = 0, ad = 0, aw = 0, av = 0;
  std::vector<int64_t> base_f(count), base_b(count), base_d(count), base_v(count);
  constexpr int64_t BB = (int64_t)kSpBlock * kSpBlock;
  for (int i = 0; i < count; ++i) {
    const SpSymbolic& y = *sp.pats[sp.inst_pat[i]]->sym;
    const bool owner = !(s->shared_tail && i > 0);
    const int64_t tail_fwd = y.fptr[y.n_tail], tail_bwd = y.bptr[y.n_tail];
    base_f[i] = af;
    base_b[i] = ab;
    base_d[i] = ad;
    af += owner ? y.nnz() : y.nnz() - tail_fwd;
    ab += owner ? y.nnz() : y.nnz() - tail_bwd;
    ad += owner ? y.n : y.n - y.n_tail;
    const int64_t tail_blk = y.blk_grp[y.ngroups - 1];
    base_v[i] = av;
    av += BB * (owner ? y.nblk : y.nblk - tail_blk);
    SpInstDev& I = sp.inst_h[i];
    I.v_tail = owner ? base_v[i] : base_v[0];
    I.v_own = owner ? base_v[i] : base_v[i] - BB * tail_blk;
    I.pat = sp.inst_pat[i];
    I.f_tail = owner ? base_f[i] : base_f[0];
    I.f_own = owner ? base_f[i] : base_f[i] - tail_fwd;
    I.b_tail = owner ? base_b[i] : base_b[0];
    I.b_own = owner ? base_b[i] : base_b[i] - tail_bwd;
    I.d_tail = owner ? base_d[i] : base_d[0];
    I.d_own = owner ? base_d[i] : base_d[i] - y.n_tail;
    I.w_off = aw;
    I.row_off = s->row_off[i];
    aw += y.n;
  }
  sp.fval_entries = af + ab;
  sp.fval.alloc(std::max<int64_t>(1, af));
  sp.bval.alloc(std::max<int64_t>(1, ab));
  sp.dinv.alloc(std::max<int64_t>(1, ad));
  sp.dinvb.alloc(std::max<int64_t>(1, av));
  sp.sdiag.alloc(std::max<int64_t>(1, ad));
  sp.w.alloc(std::max<int64_t>(1, aw));
  sp.w.zero(st);
  sp.inst_dev.upload(sp.inst_h.data(), sp.inst_h.size(), st);
  // ---- patterns to the device; the factorisation arrays stay when they are small
  sp.keep_fac = sp.pats.size() == 1 || fac_total <= ((size_t)2 << 30);
  for (auto& P : sp.pats) {
    upload_solve_arrays(*P, st);
    if (sp.keep_fac) upload_fac_arrays(*P, st);
    STROM_CUDA(cudaStreamSynchronize(st));
    release_host_indices(*P->sym);
  }
  SpDev& d = sp.dev;
  d.inst = sp.inst_dev.p;
  d.ninst = count;
  d.fval = sp.fval.p;
  d.bval = sp.bval.p;
  d.dinv = sp.dinv.p;
  d.dinvb = sp.dinvb.p;
  d.sdiag = sp.sdiag.p;
  d.w = sp.w.p;
  d.keep = s->keep.p;
  d.inst_active = nullptr;
  d.max_col = max_col;
  d.max_span = max_span;
  d.max_group = max_group;
  d.tile_r = 1;
  d.tile_r = pick_tile(s);
  refresh_pattern_views(s);
  sparse_configure(d);
}

void sparse_factor_instances(strom_solver* s, const std::vector<int>& inst, bool tail) {
  if (inst.empty()) return;
  SparseState& sp = s->sp;
  cudaStream_t st = s->stream;
  const bool sh = s->shared_tail;
  std::vector<int> full, first;
  for (int i : inst) {
    if (sh && !(tail && i == 0)) first.push_back(i);
    else full.push_back(i);
  }
  auto run = [&](const std::vector<int>& list, bool first_only) {
    // waves: the factorisation arrays of the patterns involved must be on the
    // device together (they are when keep_fac)
    size_t k = 0;
    while (k < list.size()) {
      std::vector<int> wave;
      std::vector<int> uploaded;
      size_t bytes = 0;
      while (k < list.size()) {
        const int i = list[k];
        SpPatHost& P = *sp.pats[sp.inst_pat[i]];
        if (!P.fac_on_device) {
          const size_t b = fac_bytes(*P.sym);
          if (!wave.empty() && bytes + b > ((size_t)16 << 30)) break;
          upload_fac_arrays(P, st);
          uploaded.push_back(sp.inst_pat[i]);
          bytes += b;
        }
        wave.push_back(i);
        ++k;
      }
      if (!uploaded.empty()) refresh_pattern_views(s);
      int64_t max_ns = 0, max_nnz = 0;
      int max_blk = 0;
      for (int i : wave) {
        const SpInstDev& I = sp.inst_h[i];
        const SpSymbolic& y = *sp.pats[I.pat]->sym;
        const int64_t tail_bwd = y.bptr[y.n_tail];
        const int64_t start = first_only ? I.b_own + tail_bwd : I.b_own;
        const int64_t cnt = y.nnz() - (first_only ? tail_bwd : 0);
        if (cnt > 0) STROM_CUDA(cudaMemsetAsync(sp.bval.p + start, 0, sizeof(double) * cnt, st));
        max_ns = std::max<int64_t>(max_ns, (int64_t)y.s_dst.size() - (first_only ? y.ns_tail : 0));
        max_nnz = std::max<int64_t>(max_nnz, y.nnz() - (first_only ? y.fptr[y.n_tail] : 0));
        max_blk = std::max(max_blk, y.nblk);
      }
      std::vector<int32_t> il(wave.begin(), wave.end());
      DevBuf<int32_t> ild;
      ild.upload(il.data(), il.size(), st);
      sparse_factor(sp.dev, s->yd, ild.p, (int)il.size(), first_only, s->opt.rank_tol, st, max_ns, max_nnz, max_blk);
      STROM_CUDA(cudaStreamSynchronize(st));
      if (!sp.keep_fac) {
        for (int p : uploaded) drop_fac_arrays(*sp.pats[p]);
        if (!uploaded.empty()) refresh_pattern_views(s);
      }
    }
  };
  run(full, false);
  run(first, true);
  // keep flags: an instance sharing the tail takes the owner's decisions there
  std::vector<uint8_t> keep(s->m);
  copy_d2h(keep.data(), s->keep.p, s->m, st);
  STROM_CUDA(cudaStreamSynchronize(st));
  if (sh && !first.empty()) {
    const SpSymbolic& y = *sp.pats[0]->sym;
    for (int i : first) {
      for (int p = 0; p < y.n_tail; ++p) keep[s->row_off[i] + y.can_local[p]] = keep[s->row_off[0] + y.can_local[p]];
      copy_h2d(s->keep.p + s->row_off[i], keep.data() + s->row_off[i], s->row_off[i + 1] - s->row_off[i], st);
    }
  }
  // ||b_K|| and |K| of the refactorised instances
  std::vector<double> nb(s->ninst);
  copy_d2h(nb.data(), s->norm_b.p, sizeof(double) * s->ninst, st);
  STROM_CUDA(cudaStreamSynchronize(st));
  for (int i : inst) {
    const auto& bv = s->meta[i].b;
    double acc = 0.0;
    int64_t kept = 0;
    for (int64_t r = 0; r < (int64_t)bv.size(); ++r)
      if (keep[s->row_off[i] + r]) { acc += bv[r] * bv[r]; ++kept; }
    nb[i] = std::sqrt(acc);
    s->m_kept[i] = kept;
  }
  copy_h2d(s->norm_b.p, nb.data(), sizeof(double) * s->ninst, st);
  STROM_CUDA(cudaStreamSynchronize(st));
}

void ysolve_run(strom_solver* s, const YsolveDev& yd, const double* r, double* y, double* rho, cudaStream_t st) {
  if (s->factor_kind != STROM_FACTOR_SPARSE) {
    ysolve_apply(yd, s->ninst, s->max_group, r, y, rho, st);
    return;
  }
  ysolve_star_pre(yd, r, rho, st);
  SpDev d = s->sp.dev;
  d.inst_active = yd.inst_active;
  sparse_solve(d, yd, r, rho, y, st, s->sp.max_n);
  ysolve_star_post(yd, r, y, st);
}

}  // namespace strom
