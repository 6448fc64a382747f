// An SDP given by arrays (the layout strom_sdp_export writes) instead of by
// polynomial data. The data of the star elimination and the clique groups of
// the y-solve are derived from the rows themselves; the input is checked for
// the chain structure (Definition 1, Sec. 2.3) that the solver relies on.
#include <cmath>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace {

using strom::Sdp;

struct Invalid : std::runtime_error {
  using std::runtime_error::runtime_error;
};

void need(bool ok, const std::string& what) {
  if (!ok) throw Invalid("strom_sdp_import: " + what);
}

// (i, j), i <= j, of svec position t inside a block (column-major upper)
void svec_ij(int64_t t, int* i, int* j) {
  int jj = (int)((std::sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(jj + 1) * (jj + 2) / 2 <= t) ++jj;
  while ((int64_t)jj * (jj + 1) / 2 > t) --jj;
  *j = jj;
  *i = (int)(t - (int64_t)jj * (jj + 1) / 2);
}

double svec_scale(bool diag) { return diag ? 1.0 : 1.0 / std::sqrt(2.0); }

int64_t binom(int n, int k) {
  int64_t r = 1;
  for (int t = 1; t <= k; ++t) r = r * (n - k + t) / t;
  return r;
}

Sdp* import(const strom_sdp_desc& d) {
  need(d.N >= 1 && d.dx >= 1 && d.du >= 0, "need N >= 1, dx >= 1, du >= 0");
  const int nv = 2 * d.dx + d.du;
  need(nv <= 16, "at most 16 variables per clique");
  need(d.nblocks >= d.N && d.block_n && d.block_kind && d.block_clique, "block arrays missing");
  need(d.m >= 1 && d.rowptr && d.col && d.val && d.b && d.row_kind && d.row_clique && d.C, "row arrays missing");
  std::unique_ptr<Sdp> s(new Sdp());
  s->N = d.N; s->nv = nv; s->dx = d.dx; s->du = d.du; s->kappa = 2;
  const int nM = (int)binom(nv + 2, 2);

  // ---- blocks: cliques in order, each led by its moment block of size s(nv, 2)
  int64_t off = 0;
  std::vector<int> mblk(d.N, -1), blk_clique(d.nblocks);
  std::vector<int> nloc(d.N, 0);
  for (int k = 0; k < d.nblocks; ++k) {
    const int n = d.block_n[k], c = d.block_clique[k], kind = d.block_kind[k];
    need(n >= 1 && n <= 160, "block size outside 1..160");
    need(c >= 0 && c < d.N, "block clique outside 0..N-1");
    need(kind == 0 || kind == 1, "block kind must be 0 (moment) or 1 (localizing)");
    need(k == 0 || c >= d.block_clique[k - 1], "blocks must be ordered by clique");
    if (kind == 0) {
      need(mblk[c] < 0, "more than one moment block in a clique");
      need(k == 0 || d.block_clique[k - 1] < c, "a clique's moment block must come first");
      need(n == nM, "moment block size differs from s(2 dx + du, 2)");
      mblk[c] = k;
    } else {
      need(mblk[c] >= 0, "a clique's moment block must come first");
    }
    s->block_n.push_back(n);
    s->block_off.push_back(off);
    s->block_kind.push_back((int8_t)kind);
    s->block_clique.push_back(c);
    s->block_index.push_back(kind == 0 ? -1 : (d.block_index ? d.block_index[k] : nloc[c]));
    if (kind == 1) ++nloc[c];
    blk_clique[k] = c;
    off += (int64_t)n * (n + 1) / 2;
  }
  for (int c = 0; c < d.N; ++c) need(mblk[c] >= 0, "a clique has no moment block");
  need(off <= INT32_MAX, "svec length exceeds int32 column indices");
  s->nsvec = off;
  // block of every svec position
  std::vector<int32_t> pos_blk(off);
  for (int k = 0; k < d.nblocks; ++k)
    for (int64_t t = 0; t < (int64_t)s->block_n[k] * (s->block_n[k] + 1) / 2; ++t) pos_blk[s->block_off[k] + t] = k;
  s->C.assign(d.C, d.C + off);
  for (double v : s->C) need(std::isfinite(v), "non-finite entry of C");

  // ---- rows
  const int64_t m = d.m;
  need(d.rowptr[0] == 0, "rowptr[0] must be 0");
  for (int64_t r = 0; r < m; ++r) need(d.rowptr[r + 1] >= d.rowptr[r], "rowptr must be non-decreasing");
  const int64_t nnz = d.rowptr[m];
  s->rowptr.assign(d.rowptr, d.rowptr + m + 1);
  s->col.assign(d.col, d.col + nnz);
  s->val.assign(d.val, d.val + nnz);
  s->b.assign(d.b, d.b + m);
  s->row_kind.assign(d.row_kind, d.row_kind + m);
  s->row_clique.assign(d.row_clique, d.row_clique + m);
  for (int64_t e = 0; e < nnz; ++e) {
    need(d.col[e] >= 0 && d.col[e] < off, "column index outside 0..nsvec-1");
    need(std::isfinite(d.val[e]), "non-finite entry of A");
  }
  for (int64_t r = 0; r < m; ++r) {
    const int k = d.row_clique[r], kind = d.row_kind[r];
    need(std::isfinite(d.b[r]), "non-finite entry of b");
    need(k >= 0 && k < d.N, "row clique outside 0..N-1");
    need(r == 0 || k >= d.row_clique[r - 1], "rows must be ordered by clique");
    need(kind >= STROM_ROW_MOM && kind <= STROM_ROW_CONS, "unknown row kind");
    need(kind != STROM_ROW_CONS || k + 1 < d.N, "a consensus row in the last clique");
    for (int64_t e = d.rowptr[r]; e < d.rowptr[r + 1]; ++e) {
      need(e == d.rowptr[r] || d.col[e] > d.col[e - 1], "columns of a row must be strictly increasing");
      const int bk = pos_blk[d.col[e]];
      const int c = blk_clique[bk];
      // a row stays in its clique; a consensus row also reaches the next moment block
      need(c == k || (kind == STROM_ROW_CONS && c == k + 1 && bk == mblk[k + 1]),
           "a row reaches outside its clique (chain structure)");
    }
  }

  // ---- star elimination data and Gram weights, clique by clique
  s->omega.assign(off, 0.0);
  s->inv_rep_s.assign(off, 0.0);
  std::vector<uint8_t> is_dup(off, 0);
  s->grp_ptr.push_back(0);
  int64_t r = 0;
  for (int k = 0; k < d.N; ++k) {
    const int64_t Mo = s->block_off[mblk[k]];
    std::unordered_map<int64_t, int> cls_of;
    std::vector<std::vector<std::pair<int64_t, double>>> per_cls;
    std::vector<int64_t> cls_rep;
    std::unordered_map<int64_t, double> occ;  // occurrences of each representative's monomial
    bool seen_cons = false;
    int ncons = 0;
    for (; r < m && d.row_clique[r] == k; ++r) {
      const int kind = d.row_kind[r];
      if (kind == STROM_ROW_MOM) {
        const int64_t e0 = d.rowptr[r];
        need(d.rowptr[r + 1] - e0 == 2, "an A_mom row must have exactly two entries");
        const int64_t qr = d.col[e0], qp = d.col[e0 + 1];
        need(pos_blk[qr] == mblk[k] && pos_blk[qp] == mblk[k], "an A_mom row must lie in its clique's moment block");
        int ir, jr, ip, jp;
        svec_ij(qr - Mo, &ir, &jr);
        svec_ij(qp - Mo, &ip, &jp);
        const double sr = svec_scale(ir == jr), sp = svec_scale(ip == jp);
        need(std::fabs(d.val[e0] + sr) <= 1e-12 && std::fabs(d.val[e0 + 1] - sp) <= 1e-12,
             "an A_mom row must be s_p X_p - s_r X_r with the representative first");
        need(d.b[r] == 0.0, "an A_mom row must have b = 0");
        need(!is_dup[qp], "an entry is the duplicate of two A_mom rows");
        need(!is_dup[qr], "a representative is itself a duplicate");
        is_dup[qp] = 1;
        auto it = cls_of.find(qr);
        if (it == cls_of.end()) {
          it = cls_of.emplace(qr, (int)per_cls.size()).first;
          per_cls.emplace_back();
          cls_rep.push_back(qr);
        }
        per_cls[it->second].push_back({r, 1.0 / (sp * sp)});
        occ[qr] += (ip == jp) ? 1.0 : 2.0;
      } else {
        if (kind == STROM_ROW_CONS) {
          seen_cons = true;
          ++ncons;
        } else {
          need(!seen_cons, "consensus rows must close their clique's rows");
        }
        s->oth_rows.push_back(r);
      }
    }
    for (const auto& q : cls_of) need(!is_dup[q.first], "a representative is itself a duplicate");
    for (size_t c = 0; c < per_cls.size(); ++c) {
      int ir, jr;
      svec_ij(cls_rep[c] - Mo, &ir, &jr);
      const double sc = svec_scale(ir == jr);
      s->star_rep.push_back(cls_rep[c]);
      s->star_c.push_back(sc * sc);
      s->star_ptr.push_back((int32_t)s->star_row.size());
      double dd = 0.0;
      for (auto& rv : per_cls[c]) {
        s->star_row.push_back(rv.first);
        s->star_inv_s2.push_back(rv.second);
        dd += rv.second;
      }
      s->star_d.push_back(dd);
    }
    // weights of the moment block: 1 / (occurrences s_r^2) at representatives
    const int64_t tM = (int64_t)nM * (nM + 1) / 2;
    for (int64_t t = 0; t < tM; ++t) {
      const int64_t q = Mo + t;
      if (is_dup[q]) continue;
      int i, j;
      svec_ij(t, &i, &j);
      const double sr = svec_scale(i == j);
      double oc = (i == j) ? 1.0 : 2.0;
      auto it = occ.find(q);
      if (it != occ.end()) oc += it->second;
      s->omega[q] = (1.0 / oc) / (sr * sr);
      s->inv_rep_s[q] = 1.0 / sr;
    }
    // localizing blocks: weight 1
    for (int b = 0; b < d.nblocks; ++b)
      if (s->block_clique[b] == k && s->block_kind[b] == 1)
        for (int64_t t = 0; t < (int64_t)s->block_n[b] * (s->block_n[b] + 1) / 2; ++t)
          s->omega[s->block_off[b] + t] = 1.0;
    s->grp_ptr.push_back((int32_t)s->oth_rows.size());
    s->grp_cons.push_back(ncons);
  }
  need(r == m, "row cliques must cover 0..N-1 in order");
  s->star_ptr.push_back((int32_t)s->star_row.size());
  return s.release();
}

}  // namespace

extern "C" int strom_sdp_import(const strom_sdp_desc* d, strom_sdp** out) {
  if (!d || !out) {
    strom::set_error("strom_sdp_import: null argument");
    return STROM_ERR_INVALID;
  }
  try {
    Sdp* s = import(*d);
    *out = new strom_sdp{s};
    return STROM_OK;
  } catch (const Invalid& e) {
    strom::set_error(e.what());
    return STROM_ERR_INVALID;
  } catch (const std::bad_alloc&) {
    strom::set_error("strom_sdp_import: host allocation failed");
    return STROM_ERR_OOM;
  } catch (const std::exception& e) {
    strom::set_error(std::string("strom_sdp_import: ") + e.what());
    return STROM_ERR_INVALID;
  }
}

extern "C" int strom_sdp_star_export(const strom_sdp* s, int64_t* nclass, int64_t* nstar, int64_t* rep, double* c,
                                     double* dsum, int32_t* ptr, int64_t* row, double* inv_s2, double* omega,
                                     double* inv_rep_s) {
  if (!s || !s->s) {
    strom::set_error("strom_sdp_star_export: null sdp");
    return STROM_ERR_INVALID;
  }
  const Sdp& q = *s->s;
  if (nclass) *nclass = (int64_t)q.star_rep.size();
  if (nstar) *nstar = (int64_t)q.star_row.size();
  auto cp = [](auto* dst, const auto& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  cp(rep, q.star_rep);
  cp(c, q.star_c);
  cp(dsum, q.star_d);
  cp(ptr, q.star_ptr);
  cp(row, q.star_row);
  cp(inv_s2, q.star_inv_s2);
  cp(omega, q.omega);
  cp(inv_rep_s, q.inv_rep_s);
  return STROM_OK;
}
