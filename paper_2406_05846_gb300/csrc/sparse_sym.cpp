// Symbolic analysis of the sparse factor of the y-solve (see sparse.h).
//
// The elimination tree and the row patterns of L follow the standard
// symbolic Cholesky (for row i, the pattern of L[i, :i] is the set of nodes
// reached by climbing the elimination tree from every k with S_ik != 0 until
// a node already reached for row i); no numerical values are involved.
#include <algorithm>
#include <climits>
#include <memory>
#include <numeric>
#include <string>

#include "common.cuh"
#include "sparse.h"

namespace strom {

bool same_structure(const Sdp& a, const Sdp& b) {
  return a.N == b.N && a.nv == b.nv && a.nsvec == b.nsvec && a.m() == b.m() && a.nnz() == b.nnz() &&
         a.rowptr == b.rowptr && a.col == b.col && a.row_kind == b.row_kind && a.block_n == b.block_n &&
         a.oth_rows == b.oth_rows && a.grp_ptr == b.grp_ptr;
}

SpSymbolic* sparse_symbolic(const Sdp& q) {
  auto* s = new SpSymbolic();
  const int N = q.N;
  // ---- canonical positions: cliques N..1, natural order inside a clique
  std::vector<int32_t> pos_of_row(q.m(), -1);
  s->grp_ptr.push_back(0);
  for (int k = N - 1; k >= 0; --k) {
    for (int32_t t = q.grp_ptr[k]; t < q.grp_ptr[k + 1]; ++t) {
      const int64_t row = q.oth_rows[t];
      pos_of_row[row] = (int32_t)s->can_local.size();
      s->can_local.push_back((int32_t)row);
    }
    s->grp_ptr.push_back((int32_t)s->can_local.size());
  }
  const int n = (int)s->can_local.size();
  s->n = n;
  s->ngroups = N;
  s->n_tail = s->grp_ptr[N - 1];
  std::vector<int32_t> grp_of(n);
  for (int g = 0; g < N; ++g) {
    for (int p = s->grp_ptr[g]; p < s->grp_ptr[g + 1]; ++p) grp_of[p] = g;
    s->max_group = std::max(s->max_group, s->grp_ptr[g + 1] - s->grp_ptr[g]);
  }
  // ---- incidence: positions touching each weighted svec column
  std::vector<int64_t> cptr(q.nsvec + 1, 0);
  for (int p = 0; p < n; ++p) {
    const int64_t row = s->can_local[p];
    for (int64_t e = q.rowptr[row]; e < q.rowptr[row + 1]; ++e)
      if (q.omega[q.col[e]] != 0.0) cptr[q.col[e] + 1]++;
  }
  for (int64_t c = 0; c < q.nsvec; ++c) cptr[c + 1] += cptr[c];
  std::vector<int32_t> cpos(cptr[q.nsvec]);
  {
    std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
    for (int p = 0; p < n; ++p) {  // ascending p: each column's list is sorted
      const int64_t row = s->can_local[p];
      for (int64_t e = q.rowptr[row]; e < q.rowptr[row + 1]; ++e)
        if (q.omega[q.col[e]] != 0.0) cpos[fill[q.col[e]]++] = p;
    }
  }
  // ---- lower pattern of S by rows: S_pq != 0 (q < p) when rows share a column
  std::vector<int64_t> sptr(n + 1, 0);
  std::vector<int32_t> sidx;
  std::vector<int32_t> mark(n, -1);
  for (int p = 0; p < n; ++p) {
    const int64_t row = s->can_local[p];
    const size_t start = sidx.size();
    for (int64_t e = q.rowptr[row]; e < q.rowptr[row + 1]; ++e) {
      const int32_t c = q.col[e];
      if (q.omega[c] == 0.0) continue;
      for (int64_t t = cptr[c]; t < cptr[c + 1]; ++t) {
        const int32_t o = cpos[t];
        if (o >= p) break;
        if (mark[o] != p) {
          mark[o] = p;
          sidx.push_back(o);
        }
      }
    }
    std::sort(sidx.begin() + start, sidx.end());
    sptr[p + 1] = (int64_t)sidx.size();
  }
  // ---- elimination tree (with path compression through `anc`)
  std::vector<int32_t> parent(n, -1), anc(n, -1);
  for (int i = 0; i < n; ++i)
    for (int64_t t = sptr[i]; t < sptr[i + 1]; ++t) {
      int r = sidx[t];
      while (r != -1 && r < i) {
        const int next = anc[r];
        anc[r] = i;
        if (next == -1) parent[r] = i;
        r = next;
      }
    }
  // ---- row patterns of L
  std::fill(mark.begin(), mark.end(), -1);
  s->fptr.assign(n + 1, 0);
  std::vector<int32_t> stack;
  for (int i = 0; i < n; ++i) {
    mark[i] = i;
    const size_t start = s->fcol.size();
    for (int64_t t = sptr[i]; t < sptr[i + 1]; ++t)
      for (int r = sidx[t]; r != -1 && mark[r] != i; r = parent[r]) {
        mark[r] = i;
        s->fcol.push_back(r);
      }
    std::sort(s->fcol.begin() + start, s->fcol.end());
    s->fptr[i + 1] = (int64_t)s->fcol.size();
  }
  const int64_t nnz = (int64_t)s->fcol.size();
  s->nnz_ = nnz;
  if (nnz > INT32_MAX) {
    delete s;
    throw StatusError(STROM_ERR_INVALID, "sparse factor: more than 2^31 entries for one instance");
  }
  // ---- block bidiagonal check: row i of group g reaches only groups g and g - 1
  for (int i = 0; i < n; ++i)
    for (int64_t e = s->fptr[i]; e < s->fptr[i + 1]; ++e) {
      const int d = grp_of[i] - grp_of[s->fcol[e]];
      if (d != 0 && d != 1) {
        delete s;
        throw StatusError(STROM_ERR_INVALID, "sparse factor: rows are not chain-ordered (a row of clique " +
                                                 std::to_string(N - 1 - grp_of[i]) + " reaches clique " +
                                                 std::to_string(N - 1 - grp_of[s->fcol[e]]) + ")");
      }
    }
  // ---- columns of L (backward), and the maps between the two orders
  s->bptr.assign(n + 1, 0);
  for (int64_t e = 0; e < nnz; ++e) s->bptr[s->fcol[e] + 1]++;
  for (int j = 0; j < n; ++j) s->bptr[j + 1] += s->bptr[j];
  s->brow.resize(nnz);
  s->fmap.resize(nnz);
  {
    std::vector<int64_t> fill(s->bptr.begin(), s->bptr.end() - 1);
    for (int i = 0; i < n; ++i)  // ascending rows: each column's list is sorted
      for (int64_t e = s->fptr[i]; e < s->fptr[i + 1]; ++e) {
        const int64_t d = fill[s->fcol[e]]++;
        s->brow[d] = i;
        s->fmap[e] = (int32_t)d;
      }
  }
  s->nnz_tail_b = s->bptr[s->n_tail];
  for (int j = 0; j < n; ++j) {
    const int64_t len = s->bptr[j + 1] - s->bptr[j];
    s->max_col = std::max<int32_t>(s->max_col, (int32_t)len);
    if (len > 0) s->max_span = std::max<int32_t>(s->max_span, s->brow[s->bptr[j + 1] - 1] - j);
  }
  // ---- substitution blocks and the split of each row / column at its block
  s->blk_grp.assign(1, 0);
  s->fsplit.resize(n);
  s->bsplit.resize(n);
  s->fgrp.resize(n);
  s->bgrp.resize(n);
  for (int g = 0; g < N; ++g) {
    const int a = s->grp_ptr[g], b = s->grp_ptr[g + 1];
    for (int p = a; p < b; ++p) {
      const int b0 = a + ((p - a) / kSpBlock) * kSpBlock;
      const int b1 = std::min(b, b0 + kSpBlock);
      int64_t e = s->fptr[p];
      while (e < s->fptr[p + 1] && s->fcol[e] < a) ++e;
      s->fgrp[p] = e;
      while (e < s->fptr[p + 1] && s->fcol[e] < b0) ++e;
      s->fsplit[p] = e;
      int64_t f = s->bptr[p];
      while (f < s->bptr[p + 1] && s->brow[f] < b1) ++f;
      s->bsplit[p] = f;
      while (f < s->bptr[p + 1] && s->brow[f] < b) ++f;
      s->bgrp[p] = f;
    }
    s->blk_grp.push_back(s->blk_grp.back() + (b - a + kSpBlock - 1) / kSpBlock);
  }
  s->nblk = s->blk_grp.back();
  // ---- entries of S to assemble: tail columns first
  for (int pass = 0; pass < 2; ++pass) {
    for (int p = 0; p < n; ++p) {
      // the diagonal
      if ((pass == 0) == (p < s->n_tail)) {
        s->s_ri.push_back(s->can_local[p]);
        s->s_rj.push_back(p);
        s->s_dst.push_back(-1);
      }
      for (int64_t t = sptr[p]; t < sptr[p + 1]; ++t) {
        const int32_t o = sidx[t];
        if ((pass == 0) != (o < s->n_tail)) continue;
        // position of (p, o) in column o
        const int32_t* b = s->brow.data() + s->bptr[o];
        const int32_t* e = s->brow.data() + s->bptr[o + 1];
        const int32_t* it = std::lower_bound(b, e, p);
        s->s_ri.push_back(s->can_local[p]);
        s->s_rj.push_back(o);
        s->s_dst.push_back(s->bptr[o] + (it - b));
      }
    }
    if (pass == 0) s->ns_tail = (int64_t)s->s_dst.size();
  }
  // ---- level schedules inside each group
  std::vector<int32_t> lev(n, 0);
  auto schedule = [&](bool fwd, std::vector<int32_t>& lptr, std::vector<int32_t>& lrows, std::vector<int32_t>& lgrp) {
    lptr.assign(1, 0);
    lrows.clear();
    lgrp.assign(1, 0);
    for (int g = 0; g < N; ++g) {
      const int a = s->grp_ptr[g], b = s->grp_ptr[g + 1];
      int depth = 0;
      if (fwd) {
        for (int i = a; i < b; ++i) {
          int l = 0;
          for (int64_t e = s->fptr[i]; e < s->fptr[i + 1]; ++e)
            if (s->fcol[e] >= a) l = std::max(l, lev[s->fcol[e]] + 1);
          lev[i] = l;
          depth = std::max(depth, l + 1);
        }
      } else {
        for (int j = b - 1; j >= a; --j) {
          int l = 0;
          for (int64_t e = s->bptr[j]; e < s->bptr[j + 1]; ++e)
            if (s->brow[e] < b) l = std::max(l, lev[s->brow[e]] + 1);
          lev[j] = l;
          depth = std::max(depth, l + 1);
        }
      }
      std::vector<int32_t> cnt(depth + 1, 0);
      for (int i = a; i < b; ++i) cnt[lev[i] + 1]++;
      for (int l = 0; l < depth; ++l) cnt[l + 1] += cnt[l];
      const int32_t base = (int32_t)lrows.size();
      lrows.resize(base + (b - a));
      std::vector<int32_t> fillc(cnt.begin(), cnt.end() - 1);
      for (int i = a; i < b; ++i) lrows[base + fillc[lev[i]]++] = i;  // ascending inside a level
      for (int l = 0; l < depth; ++l) lptr.push_back(base + cnt[l + 1]);
      lgrp.push_back((int32_t)lptr.size() - 1);
    }
  };
  schedule(true, s->flev_ptr, s->flev_rows, s->flev_grp);
  schedule(false, s->blev_ptr, s->blev_rows, s->blev_grp);
  return s;
}

}  // namespace strom

// ---------------------------------------------------------------------------
// C ABI: size of the sparse factor of one SDP (host only)
// ---------------------------------------------------------------------------
extern "C" int strom_sdp_factor_info(const strom_sdp* sdp, strom_factor_info* out) {
  using namespace strom;
  try {
    if (!sdp || !sdp->s || !out) throw StatusError(STROM_ERR_INVALID, "strom_sdp_factor_info: bad arguments");
    std::unique_ptr<SpSymbolic> s(sparse_symbolic(*sdp->s));
    out->n_other = s->n;
    out->n_tail = s->n_tail;
    out->nnz_L = s->nnz();
    out->nnz_S = (int64_t)s->s_dst.size() - s->n;
    out->levels_fwd = (int32_t)s->flev_ptr.size() - 1;
    out->levels_bwd = (int32_t)s->blev_ptr.size() - 1;
    out->max_group = s->max_group;
    out->max_col = s->max_col;
    out->max_span = s->max_span;
    int64_t dense = 0;
    for (int g = 0; g < s->ngroups; ++g) {
      const int64_t m = s->grp_ptr[g + 1] - s->grp_ptr[g];
      dense += m * (m + 1) / 2;
    }
    out->dense_entries = dense;
    return STROM_OK;
  } catch (const StatusError& e) {
    set_error(e.what());
    return e.status;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return STROM_ERR_OOM;
  } catch (const std::exception& e) {
    set_error(e.what());
    return STROM_ERR_INVALID;
  }
}
