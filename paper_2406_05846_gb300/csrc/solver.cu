// Batched sGS-ADMM solver (Algorithm 1) behind the C ABI: setup (upload, row
// reduction + factorisation of A A^T), the iteration loop captured as a CUDA
// graph, results, state access and the kernel-level entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "admm.cuh"
#include "common.cuh"
#include "factor.cuh"

namespace strom {
void build_classes(const int32_t* blk_n, int nblk, std::vector<int32_t>& list, PsdClasses& c);
}

#include "solver_impl.cuh"

using namespace strom;

namespace {
constexpr int64_t kChunk = 4096;
}  // namespace

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

void make_chunks(const std::vector<int64_t>& off, std::vector<Chunk>& ch, std::vector<int32_t>& first) {
  ch.clear();
  first.assign(off.size(), 0);
  for (size_t i = 0; i + 1 < off.size(); ++i) {
    first[i] = (int32_t)ch.size();
    for (int64_t s = off[i]; s < off[i + 1]; s += kChunk) ch.push_back({s, std::min(off[i + 1], s + kChunk), (int32_t)i, 0});
  }
  first.back() = (int32_t)ch.size();
}

PsdArgs psd_args(strom_solver* s, const double* in, double* out, const uint8_t* act, bool admm, bool warm = false,
                 bool warm64 = false) {
  PsdArgs a{};
  if ((warm || warm64) && s->opt.eig_warm_period > 0) {
    a.vstore = warm ? s->vstore.p : nullptr;
    a.vstore64 = warm64 ? s->vstore64.p : nullptr;
    a.vstore_off = s->vstore_off.p;
    a.blk_inst = s->blk_inst.p;
    a.inst_iter = s->iters.p;
    a.inst_iter64 = s->iters64.p;
    a.warm_period = s->opt.eig_warm_period;
    a.reorth = s->opt.eig_reorth;
  }
  a.Xb = in;
  a.out = out;
  a.blk_off = s->blk_off.p;
  a.blk_n = s->blk_n.p;
  a.blk_list = s->blk_list.p;
  a.blk_inv_sigma = admm ? s->blk_inv_sigma.p : nullptr;
  a.blk_active = act;
  a.lam_off = s->lam_off.p;
  a.vscratch = s->vscratch.p;
  return a;
}

void enqueue_iteration(strom_solver* s, cudaStream_t st) {
  const AdmmDev& d = s->ad;
  YsolveDev yd = s->yd;
  yd.inst_active = s->inst_active.p;
  admm_block_mode(d, st);
  // Step 1: r = b/sigma - A(X/sigma + S - C), y^{k+1/2} = (A A^*)^{-1} r
  admm_residual_rhs(d, s->S.p, s->r.p, st);
  ysolve_run(s, yd, s->r.p, s->yh.p, s->rho.p, st);
  // Step 2: X_b = X + sigma (A^* y - C), S = (Pi(X_b) - X_b) / sigma
  admm_xb(d, s->yh.p, s->Xb.p, st);
  psd_launch(psd_args(s, s->Xb.p, s->S.p, s->blk_act32.p, true, true), s->cls, STROM_PREC_FP32, st);
  psd_launch(psd_args(s, s->Xb.p, s->S.p, s->blk_act64.p, true, false, true), s->cls, STROM_PREC_FP64, st);
  // Step 3: r = b/sigma - A(X/sigma + S - C), y^{k+1} = (A A^*)^{-1} r
  admm_residual_rhs(d, s->S.p, s->r.p, st);
  ysolve_run(s, yd, s->r.p, s->y.p, s->rho.p, st);
  // Step 4: X = X + tau sigma (S + A^* y - C), residuals, stop test, sigma rule
  admm_xupdate(d, s->y.p, s->opt.tau, st);
  admm_primal_res(d, s->y.p, st);
  admm_finalize(d, s->prm, st);
}

void build_graph(strom_solver* s) {
  if (s->graph) return;
  psd_configure();
  STROM_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  const int64_t before = thread_launch_count();  // other host threads may launch meanwhile
  try {
    enqueue_iteration(s, s->stream);
  } catch (...) {
    cudaGraph_t g;
    cudaStreamEndCapture(s->stream, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  STROM_CUDA(cudaStreamEndCapture(s->stream, &s->graph_def));
  s->graph_kernels = thread_launch_count() - before;
  count_launches(-s->graph_kernels);  // captured, not launched
  STROM_CUDA(cudaGraphInstantiate(&s->graph, s->graph_def, 0));
}

void reset_state(strom_solver* s) {
  s->X.zero(s->stream);
  s->S.zero(s->stream);
  s->y.zero(s->stream);
  s->yh.zero(s->stream);
  s->iters.zero(s->stream);
  s->iters64.zero(s->stream);
  s->inst_flag.zero(s->stream);
  s->stats.zero(s->stream);
  std::vector<double> sg(s->ninst, s->opt.sigma0);
  std::vector<uint8_t> one(s->ninst, 1);
  std::vector<uint8_t> prec(s->ninst, (uint8_t)(s->opt.precision == STROM_PREC_FP64 ? STROM_PREC_FP64 : STROM_PREC_FP32));
  copy_h2d(s->sigma.p, sg.data(), sizeof(double) * s->ninst, s->stream);
  copy_h2d(s->inst_active.p, one.data(), s->ninst, s->stream);
  copy_h2d(s->inst_prec.p, prec.data(), s->ninst, s->stream);
  STROM_CUDA(cudaStreamSynchronize(s->stream));
}

// row reduction + factorisation of A A^T from the device data, ||b_K|| per
// instance, and a fresh state
void refactor(strom_solver* s) {
  std::vector<int> all(s->ninst);
  for (int i = 0; i < s->ninst; ++i) all[i] = i;
  s->m_kept.assign(s->ninst, 0);
  factor_instances(s, all, true);
  reset_state(s);
}

// true when b's constraint rows of cliques 2..N (and the consensus rows of
// clique 1, which couple to clique 2) equal a's exactly, with the same layout
bool same_tail(const Sdp& a, const Sdp& b) {
  if (a.N != b.N || a.nv != b.nv || a.nsvec != b.nsvec || a.m() != b.m() || a.nnz() != b.nnz()) return false;
  if (a.rowptr != b.rowptr || a.col != b.col || a.row_kind != b.row_kind || a.block_n != b.block_n) return false;
  for (int64_t r = 0; r < a.m(); ++r) {
    if (a.row_clique[r] == 0 && a.row_kind[r] != STROM_ROW_CONS) continue;
    for (int64_t e = a.rowptr[r]; e < a.rowptr[r + 1]; ++e)
      if (a.val[e] != b.val[e]) return false;
  }
  return true;
}

void solver_setup(strom_solver* s, const strom_sdp* const* sdps, int count) {
  NvtxRange nv("strom.setup");
  s->ninst = count;
  s->svec_off.assign(count + 1, 0);
  s->row_off.assign(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    const Sdp& q = *sdps[i]->s;
    s->svec_off[i + 1] = s->svec_off[i] + q.nsvec;
    s->row_off[i + 1] = s->row_off[i] + q.m();
  }
  s->nsvec = s->svec_off[count];
  s->m = s->row_off[count];
  s->shared_tail = (s->opt.share_tail != 0) && count > 1;
  s->row_clique_h0 = sdps[0]->s->row_clique;
  for (int i = 1; i < count && s->shared_tail; ++i) s->shared_tail = same_tail(*sdps[0]->s, *sdps[i]->s);
  if (s->nsvec > INT32_MAX || s->m > INT32_MAX) throw StatusError(STROM_ERR_INVALID, "batch too large for int32 indices");
  // ---- concatenated host arrays
  std::vector<int64_t> dinv_off, rowptr(1, 0), star_rep, star_row, oth_rows, grp_beg, fac_off, coup_off, blk_off,
      lam_off;
  std::vector<int32_t> col, row_inst, star_ptr, star_inst, inst_grp(1, 0), coup_n, blk_n, blk_inst;
  std::vector<double> val, b, C, omega, inv_rep_s, star_c, star_d, star_inv_s2;
  std::vector<int8_t> row_kind;
  std::vector<double> normC(count);
  s->inst_blk_off.assign(count + 1, 0);
  int64_t lam_acc = 0, dinv_acc = 0, vstore_acc = 0, fac_acc = 0, coup_acc = 0;
  std::vector<int64_t> vstore_off;
  for (int i = 0; i < count; ++i) {
    const Sdp& q = *sdps[i]->s;
    const int64_t so = s->svec_off[i], ro = s->row_off[i];
    InstMeta mt;
    mt.N = q.N; mt.nv = q.nv; mt.dx = q.dx; mt.du = q.du; mt.nsvec = q.nsvec; mt.m = q.m();
    mt.block_n = q.block_n; mt.block_clique = q.block_clique; mt.block_off = q.block_off; mt.block_kind = q.block_kind;
    mt.b = q.b;
    s->meta.push_back(std::move(mt));
    for (int64_t r = 0; r < q.m(); ++r) {
      for (int64_t e = q.rowptr[r]; e < q.rowptr[r + 1]; ++e) {
        col.push_back((int32_t)(q.col[e] + so));
        val.push_back(q.val[e]);
      }
      rowptr.push_back((int64_t)val.size());
      row_inst.push_back(i);
    }
    b.insert(b.end(), q.b.begin(), q.b.end());
    C.insert(C.end(), q.C.begin(), q.C.end());
    double nc = 0.0;
    for (double c : q.C) nc += c * c;
    normC[i] = std::sqrt(nc);
    omega.insert(omega.end(), q.omega.begin(), q.omega.end());
    inv_rep_s.insert(inv_rep_s.end(), q.inv_rep_s.begin(), q.inv_rep_s.end());
    row_kind.insert(row_kind.end(), q.row_kind.begin(), q.row_kind.end());
    const int32_t sp0 = (int32_t)star_row.size();
    for (size_t c = 0; c < q.star_rep.size(); ++c) {
      star_rep.push_back(q.star_rep[c] + so);
      star_c.push_back(q.star_c[c]);
      star_d.push_back(q.star_d[c]);
      star_ptr.push_back(sp0 + q.star_ptr[c]);
      star_inst.push_back(i);
    }
    for (size_t e = 0; e < q.star_row.size(); ++e) {
      star_row.push_back(q.star_row[e] + ro);
      star_inv_s2.push_back(q.star_inv_s2[e]);
    }
    const int64_t oth0 = (int64_t)oth_rows.size();
    for (int64_t r : q.oth_rows) oth_rows.push_back(r + ro);
    for (int k = 0; k < q.N; ++k) {
      const int64_t mk = q.grp_ptr[k + 1] - q.grp_ptr[k];
      grp_beg.push_back(oth0 + q.grp_ptr[k]);
      s->grp_full_len.push_back((int32_t)mk);
      s->grp_full_cons.push_back(q.grp_cons[k]);
      const int cprev = (k > 0) ? q.grp_cons[k - 1] : 0;
      coup_n.push_back(cprev);
      if (s->shared_tail && i > 0 && k > 0) {
        // cliques 2..N share instance 0's factor storage
        fac_off.push_back(fac_off[k]);
        coup_off.push_back(coup_off[k]);
        dinv_off.push_back(dinv_off[k]);
      } else {
        fac_off.push_back(fac_acc);
        coup_off.push_back(coup_acc);
        dinv_off.push_back(dinv_acc);
        fac_acc += mk * mk;
        coup_acc += mk * cprev;
        dinv_acc += ((mk + 31) / 32) * 1024;
      }
      s->max_group = std::max<int>(s->max_group, (int)mk);
    }
    inst_grp.push_back((int32_t)grp_beg.size());
    s->inst_nnz_off.push_back((int64_t)val.size());
    s->inst_blk_off[i] = (int64_t)blk_n.size();
    for (size_t k = 0; k < q.block_n.size(); ++k) {
      blk_off.push_back(q.block_off[k] + so);
      blk_n.push_back(q.block_n[k]);
      blk_inst.push_back(i);
      lam_off.push_back(lam_acc);
      lam_acc += q.block_n[k];
      const int64_t npk = q.block_n[k] + (q.block_n[k] & 1);
      vstore_off.push_back(vstore_acc);
      vstore_acc += npk * npk;
    }
  }
  s->inst_blk_off[count] = (int64_t)blk_n.size();
  s->inst_nnz_off.insert(s->inst_nnz_off.begin(), 0);
  s->inst_grp_h = inst_grp;
  star_ptr.push_back((int32_t)star_row.size());
  s->nblk = (int)blk_n.size();
  s->ngroups = (int)grp_beg.size();
  s->full_oth = oth_rows;
  s->grp_beg_h = grp_beg;
  s->grp_len_h = s->grp_full_len;
  s->coup_n_h = coup_n;
  s->dropped_h.assign(count, {});
  // ---- A^T (CSR over svec positions, rows ascending)
  std::vector<int64_t> atptr(s->nsvec + 1, 0);
  for (int32_t c : col) atptr[c + 1]++;
  for (int64_t p = 0; p < s->nsvec; ++p) atptr[p + 1] += atptr[p];
  std::vector<int32_t> atrow(col.size());
  std::vector<double> atval(col.size());
  {
    std::vector<int64_t> fill(atptr.begin(), atptr.end() - 1);
    for (int64_t r = 0; r < s->m; ++r)
      for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
        const int64_t dst = fill[col[e]]++;
        atrow[dst] = (int32_t)r;
        atval[dst] = val[e];
      }
  }
  // ---- chunks
  std::vector<Chunk> sch, rch;
  std::vector<int32_t> sfirst, rfirst;
  make_chunks(s->svec_off, sch, sfirst);
  make_chunks(s->row_off, rch, rfirst);
  // ---- PSD classes
  std::vector<int32_t> list;
  build_classes(blk_n.data(), s->nblk, list, s->cls);
  // ---- upload
  cudaStream_t st = s->stream;
  s->rowptr.upload(rowptr.data(), rowptr.size(), st);
  s->col.upload(col.data(), col.size(), st);
  s->val.upload(val.data(), val.size(), st);
  s->atptr.upload(atptr.data(), atptr.size(), st);
  s->atrow.upload(atrow.data(), atrow.size(), st);
  s->atval.upload(atval.data(), atval.size(), st);
  s->b.upload(b.data(), b.size(), st);
  s->C.upload(C.data(), C.size(), st);
  s->omega.upload(omega.data(), omega.size(), st);
  s->inv_rep_s.upload(inv_rep_s.data(), inv_rep_s.size(), st);
  s->row_kind.upload(row_kind.data(), row_kind.size(), st);
  s->row_inst.upload(row_inst.data(), row_inst.size(), st);
  s->star_rep.upload(star_rep.data(), star_rep.size(), st);
  s->star_c.upload(star_c.data(), star_c.size(), st);
  s->star_d.upload(star_d.data(), star_d.size(), st);
  s->star_ptr.upload(star_ptr.data(), star_ptr.size(), st);
  s->star_row.upload(star_row.data(), star_row.size(), st);
  s->star_inv_s2.upload(star_inv_s2.data(), star_inv_s2.size(), st);
  s->star_inst.upload(star_inst.data(), star_inst.size(), st);
  s->oth_rows.upload(oth_rows.data(), oth_rows.size(), st);
  s->grp_beg.upload(grp_beg.data(), grp_beg.size(), st);
  s->grp_len.upload(s->grp_full_len.data(), s->grp_full_len.size(), st);
  s->inst_grp.upload(inst_grp.data(), inst_grp.size(), st);
  s->coup_n.upload(coup_n.data(), coup_n.size(), st);
  s->fac_off.upload(fac_off.data(), fac_off.size(), st);
  s->coup_off.upload(coup_off.data(), coup_off.size(), st);
  s->blk_off.upload(blk_off.data(), blk_off.size(), st);
  s->blk_n.upload(blk_n.data(), blk_n.size(), st);
  s->blk_list.upload(list.data(), list.size(), st);
  s->blk_inst.upload(blk_inst.data(), blk_inst.size(), st);
  s->lam_off.upload(lam_off.data(), lam_off.size(), st);
  s->vstore_off.upload(vstore_off.data(), vstore_off.size(), st);
  s->vstore.alloc(std::max<int64_t>(1, vstore_acc));
  s->vstore64.alloc(std::max<int64_t>(1, vstore_acc));
  s->svec_chunks.upload(sch.data(), sch.size(), st);
  s->row_chunks.upload(rch.data(), rch.size(), st);
  s->inst_svec_chunk.upload(sfirst.data(), sfirst.size(), st);
  s->inst_row_chunk.upload(rfirst.data(), rfirst.size(), st);
  s->norm_C.upload(normC.data(), normC.size(), st);
  // the factorisation of the y-solve: dense per-clique groups or the sparse factor
  {
    int fk = s->opt.factor;
    const double dense_bytes = 8.0 * (2.0 * (double)fac_acc + (double)coup_acc + (double)dinv_acc);
    if (fk == STROM_FACTOR_AUTO) {
      // dense per-clique groups while they are small (their block steps are
      // shorter than the sparse factor's) and take at most a quarter of the
      // device's free memory; the sparse factor otherwise
      size_t free_b = 0, total_b = 0;
      STROM_CUDA(cudaMemGetInfo(&free_b, &total_b));
      fk = (s->max_group <= 800 && dense_bytes <= 0.25 * (double)free_b) ? STROM_FACTOR_DENSE : STROM_FACTOR_SPARSE;
    }
    s->factor_kind = fk;
  }
  const bool dense = s->factor_kind == STROM_FACTOR_DENSE;
  s->fac.alloc(dense ? std::max<int64_t>(1, fac_acc) : 1);
  s->lt.alloc(dense ? std::max<int64_t>(1, fac_acc) : 1);
  s->coup.alloc(dense ? std::max<int64_t>(1, coup_acc) : 1);
  s->diag0.alloc(dense ? std::max<size_t>(1, oth_rows.size()) : 1);
  s->keep.alloc(s->m);
  s->keep_oth.alloc(dense ? std::max<size_t>(1, oth_rows.size()) : 1);
  s->yo.alloc(dense ? std::max<size_t>(1, oth_rows.size()) : 1);
  s->yo.zero(st);
  s->inv_piv.alloc(dense ? std::max<size_t>(1, oth_rows.size()) : 1);
  s->dinv.alloc(dense ? std::max<int64_t>(1, dinv_acc) : 1);
  s->dinv_off.upload(dinv_off.data(), dinv_off.size(), st);
  STROM_CUDA(cudaMemsetAsync(s->keep.p, 1, s->m, st));
  for (auto* v : {&s->X, &s->S, &s->Xb, &s->rho, &s->tmp_svec}) v->alloc(s->nsvec);
  s->rho.zero(st);
  for (auto* v : {&s->y, &s->yh, &s->r}) v->alloc(s->m);
  s->norm_b.alloc(count);
  s->sigma.alloc(count);
  s->stats.alloc(8 * (size_t)count);
  s->part_svec.alloc(2 * sch.size());
  s->part_rows.alloc(2 * rch.size());
  s->blk_inv_sigma.alloc(s->nblk);
  s->inst_active.alloc(count);
  s->inst_flag.alloc(count);
  s->inst_prec.alloc(count);
  s->iters.alloc(count);
  s->iters64.alloc(count);
  s->eta_ref.alloc(count);
  s->it_ref.alloc(count);
  STROM_CUDA(cudaMemsetAsync(s->it_ref.p, 0xFF, sizeof(int32_t) * count, st));  // -1: no checkpoint yet
  STROM_CUDA(cudaMemsetAsync(s->eta_ref.p, 0, sizeof(double) * count, st));
  s->n_active.alloc(1);
  s->blk_act32.alloc(s->nblk);
  s->blk_act64.alloc(s->nblk);
  s->lam.alloc(std::max<int64_t>(1, lam_acc));
  s->topvec.alloc(std::max<int64_t>(1, lam_acc));
  if (s->cls.count[3] > 0) s->vscratch.alloc((size_t)s->cls.count[3] * kVScratchPerBlock);
  // ---- device views
  YsolveDev& yd = s->yd;
  yd.rowptr = s->rowptr.p; yd.col = s->col.p; yd.val = s->val.p;
  yd.atptr = s->atptr.p; yd.atrow = s->atrow.p; yd.atval = s->atval.p;
  yd.row_kind = s->row_kind.p; yd.row_inst = s->row_inst.p;
  yd.nclass = (int64_t)star_rep.size();
  yd.star_rep = s->star_rep.p; yd.star_c = s->star_c.p; yd.star_d = s->star_d.p; yd.star_ptr = s->star_ptr.p;
  yd.star_row = s->star_row.p; yd.star_inv_s2 = s->star_inv_s2.p; yd.star_inst = s->star_inst.p;
  yd.omega = s->omega.p; yd.inv_rep_s = s->inv_rep_s.p;
  yd.noth = (int64_t)oth_rows.size(); yd.oth_rows = s->oth_rows.p; yd.grp_beg = s->grp_beg.p; yd.grp_len = s->grp_len.p;
  yd.dropped = nullptr; yd.ndropped = 0;
  yd.inst_grp = s->inst_grp.p; yd.coup_n = s->coup_n.p;
  yd.fac = s->fac.p; yd.lt = s->lt.p; yd.fac_off = s->fac_off.p; yd.coup = s->coup.p; yd.coup_off = s->coup_off.p;
  yd.diag0 = s->diag0.p; yd.keep = s->keep.p; yd.keep_oth = s->keep_oth.p; yd.yo = s->yo.p; yd.inv_piv = s->inv_piv.p; yd.dinv = s->dinv.p; yd.dinv_off = s->dinv_off.p;
  yd.inst_active = nullptr;
  // tiles of the multi-right-hand-side solve (shared tail only): enough tiles
  // to keep every SM busy; STROM_TILE_R overrides (1, 2, 4 or 8)
  yd.tile_r = 1;
  if (s->shared_tail) {
    const int sms = 152;
    yd.tile_r = count >= 2 * sms ? 2 : 1;  // measured best for the pendulum (L2-resident shared part)
    if (const char* e = std::getenv("STROM_TILE_R")) {
      const int v = std::atoi(e);
      if (v == 1 || v == 2 || v == 4 || v == 8) yd.tile_r = v;
    }
  }
  if (dense) ysolve_configure(s->max_group);
  else sparse_setup(s, sdps, count);
  AdmmDev& ad = s->ad;
  ad.ninst = count; ad.nblk = s->nblk;
  ad.n_svec_chunks = (int)sch.size(); ad.n_row_chunks = (int)rch.size();
  ad.svec_chunks = s->svec_chunks.p; ad.row_chunks = s->row_chunks.p;
  ad.inst_svec_chunk = s->inst_svec_chunk.p; ad.inst_row_chunk = s->inst_row_chunk.p;
  ad.rowptr = s->rowptr.p; ad.col = s->col.p; ad.val = s->val.p;
  ad.atptr = s->atptr.p; ad.atrow = s->atrow.p; ad.atval = s->atval.p;
  ad.b = s->b.p; ad.C = s->C.p; ad.keep = s->keep.p; ad.norm_b = s->norm_b.p; ad.norm_C = s->norm_C.p;
  ad.X = s->X.p; ad.S = s->S.p; ad.sigma = s->sigma.p; ad.inst_active = s->inst_active.p;
  ad.inst_flag = s->inst_flag.p; ad.inst_prec = s->inst_prec.p; ad.iters = s->iters.p; ad.iters64 = s->iters64.p; ad.stats = s->stats.p;
  ad.eta_ref = s->eta_ref.p; ad.it_ref = s->it_ref.p;
  ad.part_svec = s->part_svec.p; ad.part_rows = s->part_rows.p; ad.n_active = s->n_active.p;
  ad.blk_inst = s->blk_inst.p; ad.blk_act32 = s->blk_act32.p; ad.blk_act64 = s->blk_act64.p;
  ad.blk_inv_sigma = s->blk_inv_sigma.p;
  AdmmParams& p = s->prm;
  p.tol = s->opt.tol; p.maxiter = s->opt.maxiter; p.sigma_every = s->opt.sigma_every;
  p.sigma_ratio = s->opt.sigma_ratio; p.sigma_factor = s->opt.sigma_factor;
  p.sigma_min = s->opt.sigma_min; p.sigma_max = s->opt.sigma_max;
  p.precision = s->opt.precision; p.polish_eta = s->opt.polish_eta;
  // ---- row reduction + factorisation (once)
  refactor(s);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" void strom_options_default(strom_options* o) {
  if (!o) return;
  o->tol = 1e-6;
  o->maxiter = 50000;
  o->sigma0 = 10.0;
  o->tau = 1.618;
  o->sigma_every = 20;
  o->sigma_ratio = 5.0;
  o->sigma_factor = 2.0;
  o->sigma_min = 1e-4;
  o->sigma_max = 1e4;
  o->rank_tol = 1e-8;
  o->precision = STROM_PREC_FP64;
  o->polish_eta = 1e-5;
  o->check_every = 50;
  o->time_budget_s = 0.0;
  o->eig_warm_period = 20;
  o->eig_reorth = 0;
  o->share_tail = 1;
  o->factor = STROM_FACTOR_AUTO;
}

extern "C" int strom_solver_create(const strom_sdp* const* sdps, int32_t count, const strom_options* opt,
                                   strom_solver** out) {
  return guard([&] {
    if (!sdps || count < 1 || !out) throw StatusError(STROM_ERR_INVALID, "strom_solver_create: bad arguments");
    for (int i = 0; i < count; ++i)
      if (!sdps[i] || !sdps[i]->s) throw StatusError(STROM_ERR_INVALID, "strom_solver_create: null sdp");
    std::unique_ptr<strom_solver> s(new strom_solver());
    if (opt) s->opt = *opt;
    else strom_options_default(&s->opt);
    const auto& o = s->opt;
    if (!(o.tol > 0) || o.maxiter < 1 || !(o.sigma0 > 0) || !(o.tau > 0 && o.tau < 2) || !(o.rank_tol > 0) ||
        o.precision < 0 || o.precision > 2 || o.check_every < 1 || o.eig_warm_period < 0 || o.eig_reorth < 0 || o.eig_reorth > 1 || o.factor < 0 ||
        o.factor > 2)
      throw StatusError(STROM_ERR_INVALID, "strom_solver_create: invalid options");
    // the PSD kernels keep a block of up to 160 rows in shared memory
    for (int i = 0; i < count; ++i)
      for (int32_t n : sdps[i]->s->block_n)
        if (n < 1 || n > 160)
          throw StatusError(STROM_ERR_INVALID, "strom_solver_create: a block of size " + std::to_string(n) +
                                                   "; the solver takes blocks of 1..160 (cliques of at most 16 "
                                                   "variables)");
    STROM_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    solver_setup(s.get(), sdps, count);
    *out = s.release();
    return STROM_OK;
  });
}

extern "C" void strom_solver_destroy(strom_solver* s) { delete s; }
extern "C" int32_t strom_solver_factor_kind(const strom_solver* s) { return s ? s->factor_kind : -1; }
extern "C" int32_t strom_solver_count(const strom_solver* s) { return s ? s->ninst : 0; }
extern "C" int64_t strom_solver_nsvec_total(const strom_solver* s) { return s ? s->nsvec : 0; }
extern "C" int64_t strom_solver_m_total(const strom_solver* s) { return s ? s->m : 0; }

extern "C" int strom_solver_offsets(const strom_solver* s, int32_t i, int64_t* so, int64_t* ro) {
  return guard([&] {
    if (!s || i < 0 || i >= s->ninst) throw StatusError(STROM_ERR_INVALID, "strom_solver_offsets: bad instance");
    if (so) *so = s->svec_off[i];
    if (ro) *ro = s->row_off[i];
    return STROM_OK;
  });
}

int strom::run_iterations(strom_solver* s, int iters, cudaStream_t user, int32_t* n_active) {
  NvtxRange nv("strom.iterations");
  build_graph(s);
  if (user) {  // order after the caller's prior work
    cudaEvent_t ev;
    STROM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    STROM_CUDA(cudaEventRecord(ev, user));
    STROM_CUDA(cudaStreamWaitEvent(s->stream, ev, 0));
    STROM_CUDA(cudaEventDestroy(ev));
  }
  int32_t act = 1;
  int done = 0;
  while (done < iters) {
    const int n = std::min(iters - done, s->opt.check_every);
    for (int k = 0; k < n; ++k) STROM_CUDA(cudaGraphLaunch(s->graph, s->stream));
    count_launches(s->graph_kernels * n);
    done += n;
    copy_d2h(&act, s->n_active.p, sizeof(int32_t), s->stream);
    STROM_CUDA(cudaStreamSynchronize(s->stream));
    if (act == 0) break;
  }
  if (user) {
    cudaEvent_t ev;
    STROM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    STROM_CUDA(cudaEventRecord(ev, s->stream));
    STROM_CUDA(cudaStreamWaitEvent(user, ev, 0));
    STROM_CUDA(cudaEventDestroy(ev));
  }
  if (n_active) *n_active = act;
  return done;
}

extern "C" int strom_solver_step(strom_solver* s, int32_t iters, void* stream, int32_t* n_active) {
  return guard([&] {
    if (!s || iters < 0) throw StatusError(STROM_ERR_INVALID, "strom_solver_step: bad arguments");
    run_iterations(s, iters, (cudaStream_t)stream, n_active);
    return STROM_OK;
  });
}

// upload the group lists (oth_rows slices, lengths, coupling counts) of a set
// of instances from the host copies
static void upload_groups(strom_solver* s, const std::vector<int>& inst, const std::vector<int64_t>& oth) {
  for (int i : inst) {
    const int g0 = s->inst_grp_h[i], g1 = s->inst_grp_h[i + 1];
    const int64_t b0 = s->grp_beg_h[g0];
    const int64_t b1 = s->grp_beg_h[g1 - 1] + s->grp_full_len[g1 - 1];
    copy_h2d(s->oth_rows.p + b0, oth.data() + b0, sizeof(int64_t) * (b1 - b0), s->stream);
    copy_h2d(s->grp_len.p + g0, s->grp_len_h.data() + g0, sizeof(int32_t) * (g1 - g0), s->stream);
    copy_h2d(s->coup_n.p + g0, s->coup_n_h.data() + g0, sizeof(int32_t) * (g1 - g0), s->stream);
  }
}

// Factorise a subset of instances. Pass 1 runs the pivot-skipping Cholesky on
// all other rows and decides which rows are dependent; pass 2 factorises
// again on the kept rows only, so the triangular solves of every iteration
// carry no dropped rows. Each group keeps its full-size storage, so one
// instance can be refactorised without moving the others.
//
// With a shared tail (every instance has instance 0's rows after the first
// clique), instance 0 owns the factor of cliques 2..N; `tail` = true
// (re)computes it. Every other instance factorises its first clique only,
// reusing instance 0's coupling: in pass 1 through the saved Schur update of
// the first group (all consensus rows), in pass 2 through instance 0's E.
void strom::factor_instances(strom_solver* s, const std::vector<int>& inst, bool tail) {
  if (inst.empty()) return;
  NvtxRange nv("strom.factor");
  if (s->factor_kind == STROM_FACTOR_SPARSE) {
    sparse_factor_instances(s, inst, tail);
    return;
  }
  cudaStream_t st = s->stream;
  const bool sh = s->shared_tail;
  if (sh && tail && inst.size() > 1 && std::find(inst.begin(), inst.end(), 0) != inst.end()) {
    // the other instances need instance 0's kept pattern and saved Schur
    // update, so instance 0's two passes run to completion first
    factor_instances(s, {0}, true);
    std::vector<int> rest;
    for (int i : inst)
      if (i != 0) rest.push_back(i);
    factor_instances(s, rest, false);
    return;
  }
  std::vector<int> full, first;
  for (int i : inst) {
    if (sh && (i != 0 || !tail)) first.push_back(i);
    else full.push_back(i);
  }
  if (sh && !first.empty() && s->tail_keep.empty() &&
      std::find(full.begin(), full.end(), 0) == full.end())
    throw StatusError(STROM_ERR_INVALID, "shared factor of cliques 2..N has not been computed");
  auto run = [&](const std::vector<int>& which, bool first_only, double* zsave, const double* zuse) {
    if (which.empty()) return;
    std::vector<int32_t> gl, il(which.begin(), which.end());
    for (int i : which) {
      if (first_only) gl.push_back(s->inst_grp_h[i]);
      else
        for (int g = s->inst_grp_h[i]; g < s->inst_grp_h[i + 1]; ++g) gl.push_back(g);
    }
    DevBuf<int32_t> gd, id;
    gd.upload(gl.data(), gl.size(), st);
    id.upload(il.data(), il.size(), st);
    ysolve_factor(s->yd, (int)gl.size(), (int)il.size(), s->opt.rank_tol, st, gd.p, id.p, first_only, zsave, zuse);
    STROM_CUDA(cudaStreamSynchronize(st));
  };
  // local row of instance i whose keep flag instance 0 decided (rows after the first clique)
  const int N0 = s->meta[0].N;
  auto tail_row = [&](int i, int64_t local) -> bool {
    (void)i;
    return s->row_clique_h0[local] != 0;
  };
  (void)N0;
  // tail groups of a first-only instance take instance 0's kept pattern
  auto tail_lists = [&](int i, std::vector<int64_t>& oth, std::vector<int32_t>& kept_cons) {
    for (int g = s->inst_grp_h[i] + 1; g < s->inst_grp_h[i + 1]; ++g) {
      const int64_t b = s->grp_beg_h[g];
      const int L = s->grp_full_len[g], C = s->grp_full_cons[g];
      int len = 0, cons = 0;
      for (int q = 0; q < L; ++q) {
        const int64_t row = s->full_oth[b + q];
        if (s->tail_keep[row - s->row_off[i]]) {
          oth[b + len++] = row;
          if (q >= L - C) ++cons;
        }
      }
      for (int q = len; q < L; ++q) oth[b + q] = -1;
      s->grp_len_h[g] = len;
      kept_cons[g] = cons;
    }
  };
  std::vector<int64_t> oth = s->full_oth;
  std::vector<int32_t> kept_cons(s->ngroups, 0);
  // ---- pass 1: all rows (first-only instances: their first clique's rows)
  for (int i : full)
    for (int g = s->inst_grp_h[i]; g < s->inst_grp_h[i + 1]; ++g) {
      s->grp_len_h[g] = s->grp_full_len[g];
      s->coup_n_h[g] = (g > s->inst_grp_h[i]) ? s->grp_full_cons[g - 1] : 0;
    }
  for (int i : first) {
    const int g0 = s->inst_grp_h[i];
    s->grp_len_h[g0] = s->grp_full_len[g0];
    s->coup_n_h[g0] = 0;
    tail_lists(i, oth, kept_cons);
    if (g0 + 1 < s->inst_grp_h[i + 1]) s->coup_n_h[g0 + 1] = s->grp_full_cons[g0];  // all consensus rows, Z layout
    for (int g = g0 + 2; g < s->inst_grp_h[i + 1]; ++g) s->coup_n_h[g] = kept_cons[g - 1];
  }
  upload_groups(s, inst, oth);
  std::vector<uint8_t> keep(s->m);
  for (int i : inst) {
    const int64_t ro = s->row_off[i], m = s->row_off[i + 1] - ro;
    for (int64_t r = 0; r < m; ++r) keep[ro + r] = 1;
    if (std::find(first.begin(), first.end(), i) != first.end())
      for (int64_t r = 0; r < m; ++r)
        if (tail_row(i, r)) keep[ro + r] = s->tail_keep[r];
    copy_h2d(s->keep.p + ro, keep.data() + ro, m, st);
  }
  if (sh && s->zshared.n == 0) s->zshared.alloc((size_t)s->grp_full_cons[0] * s->grp_full_cons[0] + 1);
  run(full, false, sh ? s->zshared.p : nullptr, nullptr);
  run(first, true, nullptr, s->zshared.p);
  copy_d2h(keep.data(), s->keep.p, s->m, st);
  STROM_CUDA(cudaStreamSynchronize(st));
  if (sh && std::find(full.begin(), full.end(), 0) != full.end())
    s->tail_keep.assign(keep.begin() + s->row_off[0], keep.begin() + s->row_off[1]);
  // ---- pass 2: kept rows only
  oth.assign(s->full_oth.size(), -1);
  std::vector<int64_t> keep_oth_ones;
  for (int i : inst) {
    const bool fo = std::find(first.begin(), first.end(), i) != first.end();
    s->dropped_h[i].clear();
    for (int g = s->inst_grp_h[i]; g < s->inst_grp_h[i + 1]; ++g) {
      const int64_t b = s->grp_beg_h[g];
      const int L = s->grp_full_len[g], C = s->grp_full_cons[g];
      int len = 0, cons = 0;
      for (int q = 0; q < L; ++q) {
        const int64_t row = s->full_oth[b + q];
        if (keep[row]) {
          oth[b + len++] = row;
          if (q >= L - C) ++cons;
        } else {
          s->dropped_h[i].push_back(row);
        }
      }
      s->grp_len_h[g] = len;
      kept_cons[g] = cons;
      if (fo && g > s->inst_grp_h[i])
        for (int q = 0; q < len; ++q) keep_oth_ones.push_back(b + q);
    }
    for (int g = s->inst_grp_h[i]; g < s->inst_grp_h[i + 1]; ++g)
      s->coup_n_h[g] = (g > s->inst_grp_h[i]) ? kept_cons[g - 1] : 0;
    if (fo) {
      // the shared coupling has one column per consensus row instance 0 kept
      const int g0 = s->inst_grp_h[i];
      const int64_t r0 = s->row_off[i];
      const int64_t b = s->grp_beg_h[g0];
      const int L = s->grp_full_len[g0], C = s->grp_full_cons[g0];
      for (int q = L - C; q < L; ++q) {
        const int64_t row = s->full_oth[b + q];
        if (keep[row] != s->tail_keep[row - r0])
          throw StatusError(STROM_ERR_NOT_PD, "instance's consensus rows reduce differently from the shared "
                                              "factor of cliques 2..N (use share_tail = 0)");
      }
    }
  }
  upload_groups(s, inst, oth);
  if (!keep_oth_ones.empty()) {
    std::vector<uint8_t> ko(s->full_oth.size(), 0);
    copy_d2h(ko.data(), s->keep_oth.p, ko.size(), st);
    STROM_CUDA(cudaStreamSynchronize(st));
    for (int64_t q : keep_oth_ones) ko[q] = 1;
    copy_h2d(s->keep_oth.p, ko.data(), ko.size(), st);
  }
  run(full, false, nullptr, nullptr);
  run(first, true, nullptr, nullptr);
  // rows removed by the reduction, all instances
  std::vector<int64_t> dr;
  for (const auto& v : s->dropped_h) dr.insert(dr.end(), v.begin(), v.end());
  s->dropped.upload(dr.data(), dr.size(), st);
  s->yd.dropped = s->dropped.p;
  s->yd.ndropped = (int64_t)dr.size();
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

// X = S = y = 0, sigma = sigma0, active, iteration count 0, for a set of instances
void strom::reset_instances(strom_solver* s, const std::vector<int>& inst) {
  cudaStream_t st = s->stream;
  std::vector<double> sg(s->ninst);
  std::vector<uint8_t> act(s->ninst), flag(s->ninst), prec(s->ninst);
  std::vector<int32_t> it(s->ninst);
  copy_d2h(sg.data(), s->sigma.p, sizeof(double) * s->ninst, st);
  copy_d2h(act.data(), s->inst_active.p, s->ninst, st);
  copy_d2h(flag.data(), s->inst_flag.p, s->ninst, st);
  copy_d2h(prec.data(), s->inst_prec.p, s->ninst, st);
  copy_d2h(it.data(), s->iters.p, sizeof(int32_t) * s->ninst, st);
  STROM_CUDA(cudaStreamSynchronize(st));
  const uint8_t p0 = (uint8_t)(s->opt.precision == STROM_PREC_FP64 ? STROM_PREC_FP64 : STROM_PREC_FP32);
  for (int i : inst) {
    const int64_t so = s->svec_off[i], n = s->svec_off[i + 1] - so;
    const int64_t ro = s->row_off[i], m = s->row_off[i + 1] - ro;
    STROM_CUDA(cudaMemsetAsync(s->X.p + so, 0, n * sizeof(double), st));
    STROM_CUDA(cudaMemsetAsync(s->S.p + so, 0, n * sizeof(double), st));
    STROM_CUDA(cudaMemsetAsync(s->y.p + ro, 0, m * sizeof(double), st));
    STROM_CUDA(cudaMemsetAsync(s->yh.p + ro, 0, m * sizeof(double), st));
    sg[i] = s->opt.sigma0;
    act[i] = 1;
    flag[i] = 0;
    prec[i] = p0;
    it[i] = 0;
  }
  copy_h2d(s->sigma.p, sg.data(), sizeof(double) * s->ninst, st);
  copy_h2d(s->inst_active.p, act.data(), s->ninst, st);
  copy_h2d(s->inst_flag.p, flag.data(), s->ninst, st);
  copy_h2d(s->inst_prec.p, prec.data(), s->ninst, st);
  copy_h2d(s->iters.p, it.data(), sizeof(int32_t) * s->ninst, st);
  std::vector<int32_t> it64(s->ninst);
  copy_d2h(it64.data(), s->iters64.p, sizeof(int32_t) * s->ninst, st);
  STROM_CUDA(cudaStreamSynchronize(st));
  for (int i : inst) it64[i] = 0;
  copy_h2d(s->iters64.p, it64.data(), sizeof(int32_t) * s->ninst, st);
  STROM_CUDA(cudaStreamSynchronize(st));
}

extern "C" int strom_solver_factor(strom_solver* s, void* stream) {
  return guard([&] {
    if (!s) throw StatusError(STROM_ERR_INVALID, "strom_solver_factor: null solver");
    if (stream) STROM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    refactor(s);
    return STROM_OK;
  });
}

extern "C" int strom_solve(strom_solver* s, void* stream) {
  int32_t act = 1;
  bool out_of_time = false;
  if (s && s->opt.time_budget_s > 0.0) {
    // time budget: run check_every iterations at a time and stop once the
    // budget is spent; every instance stops by itself at maxiter, so the
    // loop ends even without a deadline
    const auto t0 = std::chrono::steady_clock::now();
    while (act > 0) {
      const int st = strom_solver_step(s, s->opt.check_every, stream, &act);
      if (st != STROM_OK) return st;
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (act > 0 && el >= s->opt.time_budget_s) {
        out_of_time = true;
        break;
      }
    }
  } else {
    const int st = strom_solver_step(s, s ? s->opt.maxiter : 0, stream, &act);
    if (st != STROM_OK) return st;
  }
  std::vector<uint8_t> flag(s->ninst);
  try {
    copy_d2h(flag.data(), s->inst_flag.p, s->ninst, s->stream);
    STROM_CUDA(cudaStreamSynchronize(s->stream));
  } catch (const std::exception& e) {
    set_error(std::string("strom_solve: ") + e.what());
    return STROM_ERR_CUDA;
  }
  for (uint8_t f : flag)
    if (f == 2) { set_error("strom_solve: NaN or Inf in an instance"); return STROM_ERR_NUMERICAL; }
  if (out_of_time) {
    set_error("strom_solve: time budget exhausted (state and results valid up to the last iteration run)");
    return STROM_ERR_TIMEOUT;
  }
  for (uint8_t f : flag)
    if (f != 1) return STROM_MAXITER;
  return STROM_OK;
}

extern "C" int strom_solver_reset(strom_solver* s, int32_t i, const double* X0, const double* S0, double sigma) {
  return guard([&] {
    if (!s || i < -1 || i >= s->ninst) throw StatusError(STROM_ERR_INVALID, "strom_solver_reset: bad instance");
    if (i == -1) {
      reset_state(s);
      return STROM_OK;
    }
    const int64_t so = s->svec_off[i], n = s->svec_off[i + 1] - so;
    const int64_t ro = s->row_off[i], m = s->row_off[i + 1] - ro;
    cudaStream_t st = s->stream;
    if (X0) copy_h2d(s->X.p + so, X0, n * sizeof(double), st);
    else STROM_CUDA(cudaMemsetAsync(s->X.p + so, 0, n * sizeof(double), st));
    if (S0) copy_h2d(s->S.p + so, S0, n * sizeof(double), st);
    else STROM_CUDA(cudaMemsetAsync(s->S.p + so, 0, n * sizeof(double), st));
    STROM_CUDA(cudaMemsetAsync(s->y.p + ro, 0, m * sizeof(double), st));
    const double sg = sigma > 0 ? sigma : s->opt.sigma0;
    const uint8_t one = 1, zero = 0;
    const uint8_t prec = (uint8_t)(s->opt.precision == STROM_PREC_FP64 ? STROM_PREC_FP64 : STROM_PREC_FP32);
    const int32_t zi = 0;
    copy_h2d(s->sigma.p + i, &sg, sizeof(double), st);
    copy_h2d(s->inst_active.p + i, &one, 1, st);
    copy_h2d(s->inst_flag.p + i, &zero, 1, st);
    copy_h2d(s->inst_prec.p + i, &prec, 1, st);
    copy_h2d(s->iters.p + i, &zi, sizeof(int32_t), st);
    copy_h2d(s->iters64.p + i, &zi, sizeof(int32_t), st);
    STROM_CUDA(cudaStreamSynchronize(st));
    return STROM_OK;
  });
}

extern "C" int strom_get_result(const strom_solver* s, int32_t i, strom_result* r) {
  return guard([&] {
    if (!s || !r || i < 0 || i >= s->ninst) throw StatusError(STROM_ERR_INVALID, "strom_get_result: bad arguments");
    double st[8];
    int32_t it;
    uint8_t flag;
    double sg;
    copy_d2h(st, s->stats.p + 8 * (int64_t)i, sizeof(st), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
    copy_d2h(&it, s->iters.p + i, sizeof(int32_t), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
    copy_d2h(&flag, s->inst_flag.p + i, 1, s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
    copy_d2h(&sg, s->sigma.p + i, sizeof(double), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
    r->status = flag == 1 ? STROM_OK : flag == 2 ? STROM_ERR_NUMERICAL : STROM_MAXITER;
    r->iterations = it;
    r->eta_p = st[0]; r->eta_d = st[1]; r->eta_g = st[2]; r->pobj = st[3]; r->dobj = st[4];
    r->sigma = sg;
    r->m_kept = s->m_kept[i];
    return STROM_OK;
  });
}

extern "C" int strom_get_state(const strom_solver* s, int32_t i, double* X, double* S, double* y) {
  return guard([&] {
    if (!s || i < 0 || i >= s->ninst) throw StatusError(STROM_ERR_INVALID, "strom_get_state: bad instance");
    const int64_t so = s->svec_off[i], n = s->svec_off[i + 1] - so;
    const int64_t ro = s->row_off[i], m = s->row_off[i + 1] - ro;
    if (X) copy_d2h(X, s->X.p + so, n * sizeof(double), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
    if (S) copy_d2h(S, s->S.p + so, n * sizeof(double), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
    if (y) copy_d2h(y, s->y.p + ro, m * sizeof(double), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
    return STROM_OK;
  });
}

extern "C" int strom_get_kept_rows(const strom_solver* s, int32_t i, uint8_t* keep) {
  return guard([&] {
    if (!s || !keep || i < 0 || i >= s->ninst) throw StatusError(STROM_ERR_INVALID, "strom_get_kept_rows: bad arguments");
    const int64_t ro = s->row_off[i], m = s->row_off[i + 1] - ro;
    copy_d2h(keep, s->keep.p + ro, m, s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
    return STROM_OK;
  });
}

extern "C" int strom_get_moment(const strom_solver* s, int32_t i, int32_t k, double* Mk) {
  return guard([&] {
    if (!s || !Mk || i < 0 || i >= s->ninst) throw StatusError(STROM_ERR_INVALID, "strom_get_moment: bad arguments");
    const InstMeta& mt = s->meta[i];
    int blk = -1;
    for (size_t b = 0; b < mt.block_n.size(); ++b)
      if (mt.block_kind[b] == 0 && mt.block_clique[b] == k) blk = (int)b;
    if (blk < 0) throw StatusError(STROM_ERR_INVALID, "strom_get_moment: no such clique");
    const int n = mt.block_n[blk];
    std::vector<double> v((size_t)n * (n + 1) / 2);
    copy_d2h(v.data(), s->X.p + s->svec_off[i] + mt.block_off[blk], v.size() * sizeof(double), s->stream);
    STROM_CUDA(cudaStreamSynchronize(s->stream));
    for (int j = 0; j < n; ++j)
      for (int q = 0; q <= j; ++q) {
        const double x = v[(size_t)j * (j + 1) / 2 + q] * (q == j ? 1.0 : 0.70710678118654752440);
        Mk[(size_t)j * n + q] = x;
        Mk[(size_t)q * n + j] = x;
      }
    return STROM_OK;
  });
}

extern "C" int strom_kernel_A(const strom_solver* s, const double* x_dev, double* Ax_dev, void* stream) {
  return guard([&] {
    if (!s || !x_dev || !Ax_dev) throw StatusError(STROM_ERR_INVALID, "strom_kernel_A: bad arguments");
    csr_spmv(s->rowptr.p, s->col.p, s->val.p, s->m, x_dev, Ax_dev, (cudaStream_t)stream);
    return STROM_OK;
  });
}

extern "C" int strom_kernel_spmv_csr(const int64_t* rowptr_dev, const int32_t* col_dev, const double* val_dev,
                                     int64_t nrows, const double* x_dev, double* y_dev, void* stream) {
  return guard([&] {
    if (nrows < 0 || (nrows > 0 && (!rowptr_dev || !col_dev || !val_dev || !x_dev || !y_dev || x_dev == y_dev)))
      throw StatusError(STROM_ERR_INVALID, "strom_kernel_spmv_csr: bad arguments");
    csr_spmv(rowptr_dev, col_dev, val_dev, nrows, x_dev, y_dev, (cudaStream_t)stream);
    return STROM_OK;
  });
}

extern "C" int strom_kernel_At(const strom_solver* s, const double* y_dev, double* x_dev, void* stream) {
  return guard([&] {
    if (!s || !x_dev || !y_dev) throw StatusError(STROM_ERR_INVALID, "strom_kernel_At: bad arguments");
    csr_spmv(s->atptr.p, s->atrow.p, s->atval.p, s->nsvec, y_dev, x_dev, (cudaStream_t)stream);
    return STROM_OK;
  });
}

extern "C" int strom_kernel_solve(const strom_solver* s, const double* r_dev, double* y_dev, void* stream) {
  return guard([&] {
    if (!s || !r_dev || !y_dev || r_dev == y_dev) throw StatusError(STROM_ERR_INVALID, "strom_kernel_solve: bad arguments");
    YsolveDev yd = s->yd;
    yd.inst_active = nullptr;
    ysolve_run(const_cast<strom_solver*>(s), yd, r_dev, y_dev, const_cast<double*>(s->rho.p), (cudaStream_t)stream);
    return STROM_OK;
  });
}

namespace {
struct EventPair {  // both events are destroyed even when creating the second one fails
  cudaEvent_t a = nullptr, b = nullptr;
  void create() {
    STROM_CUDA(cudaEventCreate(&a));
    STROM_CUDA(cudaEventCreate(&b));
  }
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};
}  // namespace

extern "C" int strom_solver_tune(strom_solver* s, int32_t reps, void* stream, strom_tune_report* out) {
  return guard([&] {
    if (!s || !out || reps < 1 || reps > 1000) throw StatusError(STROM_ERR_INVALID, "strom_solver_tune: bad arguments");
    std::memset(out, 0, sizeof(*out));
    if (stream) STROM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    cudaStream_t st = s->stream;
    // candidate tiles: several instances per CTA need the shared tail
    const bool sparse = s->factor_kind == STROM_FACTOR_SPARSE;
    std::vector<int> cand = {1};
    if (s->shared_tail)
      for (int r : {2, 4, 8})
        if (r <= s->ninst && (!sparse || sizeof(double) * 2 * (size_t)r * s->sp.dev.max_group <= 200 * 1024))
          cand.push_back(r);
    DevBuf<double> rhs, sol;
    rhs.alloc(s->m);
    sol.alloc(s->m);
    std::vector<double> ones(s->m, 1.0);
    copy_h2d(rhs.p, ones.data(), sizeof(double) * s->m, st);
    YsolveDev yd = s->yd;
    yd.inst_active = nullptr;
    EventPair ev;
    ev.create();
    const int old_tile = sparse ? s->sp.dev.tile_r : s->yd.tile_r;
    int best = old_tile;
    double best_ms = -1.0;
    auto set_tile = [&](int r) {
      if (sparse) {
        s->sp.dev.tile_r = r;
        sparse_configure(s->sp.dev);
      } else {
        yd.tile_r = r;
      }
    };
    for (size_t c = 0; c < cand.size(); ++c) {
      set_tile(cand[c]);
      ysolve_run(s, yd, rhs.p, sol.p, s->rho.p, st);  // warm-up
      STROM_CUDA(cudaEventRecord(ev.a, st));
      for (int k = 0; k < reps; ++k) ysolve_run(s, yd, rhs.p, sol.p, s->rho.p, st);
      STROM_CUDA(cudaEventRecord(ev.b, st));
      STROM_CUDA(cudaEventSynchronize(ev.b));
      float ms = 0.0f;
      STROM_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
      out->tile[c] = cand[c];
      out->ms[c] = (double)ms / reps;
      if (best_ms < 0.0 || out->ms[c] < best_ms) {
        best_ms = out->ms[c];
        best = cand[c];
      }
    }
    set_tile(best);
    if (!sparse) s->yd.tile_r = best;
    out->ncand = (int32_t)cand.size();
    out->chosen = best;
    // eigensolver launch shapes: each size class alone, each candidate
    // thread count, cold sweeps on a fixed pseudo-random input of the
    // solver's block layout (the state is not touched)
    bool eig_changed = false;
    {
      DevBuf<double> xin, xout;
      xin.alloc(s->nsvec);
      xout.alloc(s->nsvec);
      psd_fill_test_input(xin.p, s->nsvec, st);
      const int precs[2] = {STROM_PREC_FP64, STROM_PREC_FP32};
      for (int pi = 0; pi < 2; ++pi) {
        if (precs[pi] == STROM_PREC_FP32 && s->opt.precision == STROM_PREC_FP64) continue;
        for (int k = 0; k < 4; ++k) {
          if (s->cls.count[k] == 0) continue;
          int cands[3];
          const int nc = psd_threads_candidates(precs[pi], k, cands);
          PsdClasses one{};
          one.start[k] = s->cls.start[k];
          one.count[k] = s->cls.count[k];
          one.max_n[k] = s->cls.max_n[k];
          PsdArgs a = psd_args(s, xin.p, xout.p, nullptr, false);
          double bms = -1.0;
          int bth = cands[0];
          for (int c = 0; c < nc; ++c) {
            one.threads[pi][k] = cands[c];
            psd_launch(a, one, precs[pi], st);  // warm-up
            STROM_CUDA(cudaEventRecord(ev.a, st));
            for (int r = 0; r < reps; ++r) psd_launch(a, one, precs[pi], st);
            STROM_CUDA(cudaEventRecord(ev.b, st));
            STROM_CUDA(cudaEventSynchronize(ev.b));
            float ms = 0.0f;
            STROM_CUDA(cudaEventElapsedTime(&ms, ev.a, ev.b));
            const double m = (double)ms / reps;
            if (bms < 0.0 || m < bms) { bms = m; bth = cands[c]; }
          }
          const int old = s->cls.threads[pi][k] ? s->cls.threads[pi][k] : cands[0];
          if (bth != old) eig_changed = true;
          s->cls.threads[pi][k] = bth;
          out->eig_threads[pi][k] = bth;
          out->eig_ms[pi][k] = bms;
        }
      }
    }
    if (best != old_tile || eig_changed) {
      // the captured iteration holds the old launch shape: capture again on the next step
      if (s->graph) { STROM_CUDA(cudaGraphExecDestroy(s->graph)); s->graph = nullptr; }
      if (s->graph_def) { STROM_CUDA(cudaGraphDestroy(s->graph_def)); s->graph_def = nullptr; }
    }
    return STROM_OK;
  });
}

// helpers for the certificate (certify.cpp)
namespace strom {
struct CertDevice {
  const strom_solver* s;
};
void solver_eig_blocks(strom_solver* s, int inst, bool use_Z, std::vector<double>& lam, std::vector<double>& topvec);
void solver_eig_all(strom_solver* s, bool use_Z, std::vector<double>& lam, std::vector<double>& topvec,
                    std::vector<int64_t>& lam_off, std::vector<double>& stats);
int solver_inst_blocks(const strom_solver* s, int inst, std::vector<int32_t>& n, std::vector<int8_t>& kind,
                       std::vector<int32_t>& clique, int64_t* first_blk);
}  // namespace strom

namespace {
__global__ void z_kernel(const int64_t* atptr, const int32_t* atrow, const double* atval, const double* y, const double* C,
                         int64_t begin, int64_t end, double* Z) {
  const int64_t p = begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= end) return;
  double acc = 0.0;
  for (int64_t e = atptr[p]; e < atptr[p + 1]; ++e) acc += atval[e] * y[atrow[e]];
  Z[p] = C[p] - acc;
}
}  // namespace

// eigenvalues (ascending) and top eigenvectors of the blocks of a set of
// instances, for X or Z = C - A^T y; lam_off receives the global offsets
void strom::eig_instances(strom_solver* s, const std::vector<int>& inst, bool use_Z, std::vector<double>& lam,
                          std::vector<double>& topvec, std::vector<int64_t>& lam_off) {
  NvtxRange nv("strom.certify.eig");
  const double* in = s->X.p;
  if (use_Z) {
    for (int i : inst) {
      const int64_t so = s->svec_off[i], se = s->svec_off[i + 1];
      z_kernel<<<ceil_div(se - so, 256), 256, 0, s->stream>>>(s->atptr.p, s->atrow.p, s->atval.p, s->y.p, s->C.p, so,
                                                            se, s->tmp_svec.p);
      STROM_CUDA(cudaGetLastError());
      count_launches(1);
    }
    in = s->tmp_svec.p;
  }
  std::vector<int32_t> nall(s->nblk);
  copy_d2h(nall.data(), s->blk_n.p, sizeof(int32_t) * s->nblk, s->stream);
  STROM_CUDA(cudaStreamSynchronize(s->stream));
  PsdClasses cls;
  std::vector<std::vector<int32_t>> per(4);
  for (int i : inst)
    for (int64_t b = s->inst_blk_off[i]; b < s->inst_blk_off[i + 1]; ++b) {
      const int n = nall[b];
      per[n <= 16 ? 0 : n <= 40 ? 1 : n <= 80 ? 2 : 3].push_back((int32_t)b);
    }
  std::vector<int32_t> ids;
  for (int k = 0; k < 4; ++k) {
    cls.start[k] = (int)ids.size();
    cls.count[k] = (int)per[k].size();
    for (int b : per[k]) ids.push_back(b);
  }
  DevBuf<int32_t> list;
  list.upload(ids.data(), ids.size(), s->stream);
  DevBuf<double> vs;
  if (cls.count[3] > 0) vs.alloc((size_t)cls.count[3] * kVScratchPerBlock);
  PsdArgs a{};
  a.Xb = in;
  a.blk_off = s->blk_off.p;
  a.blk_n = s->blk_n.p;
  a.blk_list = list.p;
  a.lam = s->lam.p;
  a.lam_off = s->lam_off.p;
  a.topvec = s->topvec.p;
  a.vscratch = vs.p;
  psd_launch(a, cls, STROM_PREC_FP64, s->stream);
  lam.assign(s->lam.n, 0.0);
  topvec.assign(s->topvec.n, 0.0);
  lam_off.assign(s->nblk, 0);
  copy_d2h(lam.data(), s->lam.p, sizeof(double) * lam.size(), s->stream);
  copy_d2h(topvec.data(), s->topvec.p, sizeof(double) * topvec.size(), s->stream);
  copy_d2h(lam_off.data(), s->lam_off.p, sizeof(int64_t) * s->nblk, s->stream);
  STROM_CUDA(cudaStreamSynchronize(s->stream));
}

// eigenvalues (ascending, per block) and top eigenvectors of instance `inst`
// for X (use_Z = false) or Z = C - A^T y (use_Z = true); FP64 Jacobi on the GPU
void strom::solver_eig_blocks(strom_solver* s, int inst, bool use_Z, std::vector<double>& lam, std::vector<double>& topvec) {
  const int64_t so = s->svec_off[inst], se = s->svec_off[inst + 1];
  const double* in = s->X.p;
  if (use_Z) {
    z_kernel<<<ceil_div(se - so, 256), 256, 0, s->stream>>>(s->atptr.p, s->atrow.p, s->atval.p, s->y.p, s->C.p, so, se,
                                                          s->tmp_svec.p);
    STROM_CUDA(cudaGetLastError());
    count_launches(1);
    in = s->tmp_svec.p;
  }
  // a block list with only this instance's blocks
  const int b0 = (int)s->inst_blk_off[inst], b1 = (int)s->inst_blk_off[inst + 1];
  std::vector<int32_t> bn(b1 - b0), ids;
  std::vector<int32_t> nall(s->nblk);
  copy_d2h(nall.data(), s->blk_n.p, sizeof(int32_t) * s->nblk, s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
  PsdClasses cls;
  std::vector<std::vector<int32_t>> per(4);
  for (int b = b0; b < b1; ++b) {
    const int n = nall[b];
    per[n <= 16 ? 0 : n <= 40 ? 1 : n <= 80 ? 2 : 3].push_back(b);
  }
  for (int k = 0; k < 4; ++k) {
    cls.start[k] = (int)ids.size();
    cls.count[k] = (int)per[k].size();
    for (int b : per[k]) ids.push_back(b);
  }
  DevBuf<int32_t> list;
  list.upload(ids.data(), ids.size(), s->stream);
  DevBuf<double> vs;
  if (cls.count[3] > 0) vs.alloc((size_t)cls.count[3] * kVScratchPerBlock);
  PsdArgs a{};
  a.Xb = in;
  a.out = nullptr;
  a.blk_off = s->blk_off.p;
  a.blk_n = s->blk_n.p;
  a.blk_list = list.p;
  a.lam = s->lam.p;
  a.lam_off = s->lam_off.p;
  a.topvec = s->topvec.p;
  a.vscratch = vs.p;
  psd_launch(a, cls, STROM_PREC_FP64, s->stream);
  STROM_CUDA(cudaStreamSynchronize(s->stream));
  lam.assign(s->lam.n, 0.0);
  topvec.assign(s->topvec.n, 0.0);
  copy_d2h(lam.data(), s->lam.p, sizeof(double) * lam.size(), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
  copy_d2h(topvec.data(), s->topvec.p, sizeof(double) * topvec.size(), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
}

// eigenvalues (ascending) and top eigenvectors of every block of the batch,
// for X (use_Z = false) or Z = C - A^T y (use_Z = true); FP64 Jacobi
void strom::solver_eig_all(strom_solver* s, bool use_Z, std::vector<double>& lam, std::vector<double>& topvec,
                           std::vector<int64_t>& lam_off, std::vector<double>& stats) {
  const double* in = s->X.p;
  if (use_Z) {
    z_kernel<<<ceil_div(s->nsvec, 256), 256, 0, s->stream>>>(s->atptr.p, s->atrow.p, s->atval.p, s->y.p, s->C.p, 0,
                                                            s->nsvec, s->tmp_svec.p);
    STROM_CUDA(cudaGetLastError());
    count_launches(1);
    in = s->tmp_svec.p;
  }
  PsdArgs a{};
  a.Xb = in;
  a.out = nullptr;
  a.blk_off = s->blk_off.p;
  a.blk_n = s->blk_n.p;
  a.blk_list = s->blk_list.p;
  a.lam = s->lam.p;
  a.lam_off = s->lam_off.p;
  a.topvec = s->topvec.p;
  a.vscratch = s->vscratch.p;
  psd_launch(a, s->cls, STROM_PREC_FP64, s->stream);
  lam.assign(s->lam.n, 0.0);
  topvec.assign(s->topvec.n, 0.0);
  lam_off.assign(s->nblk, 0);
  stats.assign(8 * (size_t)s->ninst, 0.0);
  copy_d2h(lam.data(), s->lam.p, sizeof(double) * lam.size(), s->stream);
  copy_d2h(topvec.data(), s->topvec.p, sizeof(double) * topvec.size(), s->stream);
  copy_d2h(lam_off.data(), s->lam_off.p, sizeof(int64_t) * s->nblk, s->stream);
  copy_d2h(stats.data(), s->stats.p, sizeof(double) * stats.size(), s->stream);
  STROM_CUDA(cudaStreamSynchronize(s->stream));
}

int strom::solver_inst_blocks(const strom_solver* s, int inst, std::vector<int32_t>& n, std::vector<int8_t>& kind,
                              std::vector<int32_t>& clique, int64_t* first_blk) {
  const InstMeta& mt = s->meta[inst];
  n = mt.block_n;
  kind = mt.block_kind;
  clique = mt.block_clique;
  *first_blk = s->inst_blk_off[inst];
  return mt.N;
}

namespace strom {
int solver_blocks_of(const strom_solver* s, int inst, std::vector<int32_t>& n, std::vector<int8_t>& kind,
                     std::vector<int32_t>& clique, std::vector<int64_t>& lam_off, double* by) {
  const InstMeta& mt = s->meta[inst];
  n = mt.block_n;
  kind = mt.block_kind;
  clique = mt.block_clique;
  lam_off.clear();
  std::vector<int64_t> all(s->nblk);
  copy_d2h(all.data(), s->lam_off.p, sizeof(int64_t) * s->nblk, s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
  for (int64_t b = s->inst_blk_off[inst]; b < s->inst_blk_off[inst + 1]; ++b) lam_off.push_back(all[b]);
  double st[8];
  copy_d2h(st, s->stats.p + 8 * (int64_t)inst, sizeof(st), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
  // <b, y> over kept rows of this instance, recomputed from the current y
  const int64_t ro = s->row_off[inst], m = s->row_off[inst + 1] - ro;
  std::vector<double> y(m);
  std::vector<uint8_t> keep(m);
  copy_d2h(y.data(), s->y.p + ro, m * sizeof(double), s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
  copy_d2h(keep.data(), s->keep.p + ro, m, s->stream); STROM_CUDA(cudaStreamSynchronize(s->stream));
  double acc = 0.0;
  for (int64_t r = 0; r < m; ++r)
    if (keep[r]) acc += mt.b[r] * y[r];
  *by = acc;
  return mt.N;
}
}  // namespace strom
