// Host relaxation builder: polynomial data with chain-like sparsity
// (Definition 1) -> order-2 sparse moment relaxation (Prop. 1) -> PSD-only
// standard SDP {C, A, b} (Sec. 2.3, eq. standardsdp).
//
// Layout: blocks M_1, L_{1,1..}, M_2, ...; X in svec form (SDPT3: column-major
// upper triangle, off-diagonal entries times sqrt(2)); rows by clique, inside
// clique k: A_mom, A_ineq, A_eq, phi_0 = 1, consensus with clique k+1.
// A monomial of M_k is represented by its first occurrence in column-major
// upper order (reproduces the indices printed in Sec. 2.3).
//
// The builder also emits the data of the star elimination used by the
// y-solve: every A_mom row ties one duplicate entry p of monomial alpha to
// its representative r, s_p e_p - s_r e_r. Eliminating these rows from
// A A^T leaves, on the other rows, the weighted Gram A_o diag(omega) A_o^T
// with omega_r = w_alpha / s_r^2 at representatives, w_alpha = 1 / (number of
// occurrences of alpha in the full symmetric matrix), and omega = 1 on the
// entries of localizing blocks.
#include <algorithm>
#include <cmath>
#include <map>
#include <stdexcept>
#include <unordered_map>

#include "internal.h"

namespace strom {

int Poly::degree(int nv) const {
  int d = 0;
  for (int t = 0; t < nterms(); ++t) {
    int s = 0;
    for (int i = 0; i < nv; ++i) s += expo[(size_t)t * nv + i];
    d = std::max(d, s);
  }
  return d;
}

std::vector<std::vector<uint8_t>> monomial_basis(int nv, int d) {
  // graded; inside a degree, index multisets i1 <= i2 <= ... in lexicographic order
  std::vector<std::vector<uint8_t>> out;
  for (int deg = 0; deg <= d; ++deg) {
    std::vector<int> idx(deg, 0);
    while (true) {
      std::vector<uint8_t> e(nv, 0);
      for (int i : idx) e[i]++;
      out.push_back(e);
      int pos = deg - 1;
      while (pos >= 0 && idx[pos] == nv - 1) --pos;
      if (pos < 0) break;
      idx[pos]++;
      for (int q = pos + 1; q < deg; ++q) idx[q] = idx[pos];
    }
  }
  return out;
}

namespace {

constexpr double kInvSqrt2 = 0.70710678118654752440;

inline int64_t svec_index(int i, int j) {
  if (i > j) std::swap(i, j);
  return (int64_t)j * (j + 1) / 2 + i;
}
inline double svec_scale(int i, int j) { return i == j ? 1.0 : 1.0 / std::sqrt(2.0); }

// A monomial packed into 64 bits: 4 bits per variable up to 16 variables,
// 3 bits per variable for 17..21. Every monomial the relaxation forms has
// total degree <= 2 kappa = 4 (the degrees of f, g and h are checked on
// input), so no exponent exceeds 4 and a sum of two keys never carries into
// the next variable's field.
using Key = uint64_t;
constexpr int kMaxCliqueVars = 21;
inline int key_bits(int nv) { return nv <= 16 ? 4 : 3; }
inline Key key_of(const uint8_t* e, int nv) {
  const int b = key_bits(nv);
  Key k = 0;
  for (int i = 0; i < nv; ++i) k |= (Key)e[i] << (b * i);
  return k;
}
inline Key key_add(Key a, Key b) { return a + b; }

struct MomentIndex {
  int nv, n;
  std::vector<Key> basis;
  std::unordered_map<Key, std::pair<int, int>> rep;
  std::unordered_map<Key, std::vector<std::pair<int, int>>> entries;
  std::vector<Key> order;  // monomials in order of first occurrence
  MomentIndex(int nv_, int kappa) : nv(nv_) {
    for (auto& e : monomial_basis(nv, kappa)) basis.push_back(key_of(e.data(), nv));
    n = (int)basis.size();
    for (int j = 0; j < n; ++j)
      for (int i = 0; i <= j; ++i) {
        Key a = key_add(basis[i], basis[j]);
        auto it = rep.find(a);
        if (it == rep.end()) {
          rep.emplace(a, std::make_pair(i, j));
          order.push_back(a);
        }
        entries[a].push_back({i, j});
      }
  }
};

struct Term { double c; Key e; };

std::vector<Term> terms_of(const Poly& p, int nv) {
  std::vector<Term> t;
  for (int i = 0; i < p.nterms(); ++i) t.push_back({p.coef[i], key_of(&p.expo[(size_t)i * nv], nv)});
  return t;
}

}  // namespace

Sdp* build_relaxation(const Problem& p) {
  const int N = p.N, nv = p.nv(), kappa = p.kappa, dx = p.dx;
  if (kappa != 2) throw std::runtime_error("relaxation order kappa must be 2");
  if (nv > kMaxCliqueVars) throw std::runtime_error("at most 21 variables per clique");
  MomentIndex mi(nv, kappa);
  const int nM = mi.n;
  Sdp* s = new Sdp();
  s->N = N; s->nv = nv; s->dx = p.dx; s->du = p.du; s->kappa = kappa;

  // ---- blocks
  struct Loc { int blk; std::vector<Key> basis; std::vector<Term> g; };
  std::vector<std::vector<Loc>> locs(N);
  std::vector<int> mblk(N);
  int64_t off = 0;
  for (int k = 0; k < N; ++k) {
    mblk[k] = (int)s->block_n.size();
    s->block_n.push_back(nM); s->block_off.push_back(off); s->block_kind.push_back(0);
    s->block_clique.push_back(k); s->block_index.push_back(-1);
    off += (int64_t)nM * (nM + 1) / 2;
    for (size_t i = 0; i < p.cl[k].g.size(); ++i) {
      const Poly& g = p.cl[k].g[i];
      int dg = (g.degree(nv) + 1) / 2;
      Loc L;
      L.blk = (int)s->block_n.size();
      for (auto& e : monomial_basis(nv, kappa - dg)) L.basis.push_back(key_of(e.data(), nv));
      L.g = terms_of(g, nv);
      int n = (int)L.basis.size();
      s->block_n.push_back(n); s->block_off.push_back(off); s->block_kind.push_back(1);
      s->block_clique.push_back(k); s->block_index.push_back((int)i);
      off += (int64_t)n * (n + 1) / 2;
      locs[k].push_back(std::move(L));
    }
  }
  s->nsvec = off;
  s->C.assign(off, 0.0);
  s->omega.assign(off, 0.0);
  s->inv_rep_s.assign(off, 0.0);

  auto mpos = [&](int k, Key a, double* sc) -> int64_t {
    auto it = mi.rep.find(a);
    if (it == mi.rep.end()) throw std::runtime_error("monomial degree exceeds 2 kappa");
    int i = it->second.first, j = it->second.second;
    *sc = svec_scale(i, j);
    return s->block_off[mblk[k]] + svec_index(i, j);
  };

  std::vector<std::pair<int64_t, double>> ent;
  std::map<int64_t, double> acc;
  auto emit = [&](double rhs, int kind, int k) {
    acc.clear();
    for (auto& pv : ent) acc[pv.first] += pv.second;
    for (auto& pv : acc)
      if (pv.second != 0.0) { s->col.push_back((int32_t)pv.first); s->val.push_back(pv.second); }
    s->rowptr.push_back((int64_t)s->val.size());
    s->b.push_back(rhs);
    s->row_kind.push_back((int8_t)kind);
    s->row_clique.push_back(k);
  };
  s->rowptr.push_back(0);
  if (off > INT32_MAX) throw std::runtime_error("svec length exceeds int32 column indices");

  s->grp_ptr.push_back(0);
  for (int k = 0; k < N; ++k) {
    const CliqueData& cl = p.cl[k];
    const int64_t Mo = s->block_off[mblk[k]];
    double sc;
    // objective <C_k, M_k> = ell(f_k)
    for (auto& t : terms_of(cl.f, nv)) {
      int64_t q = mpos(k, t.e, &sc);
      s->C[q] += t.c * sc;
    }
    // star data and omega of M_k
    for (Key a : mi.order) {
      const auto& ents = mi.entries[a];
      double occ = 0.0;
      for (auto& ij : ents) occ += (ij.first == ij.second) ? 1.0 : 2.0;
      auto r = mi.rep[a];
      double sr = svec_scale(r.first, r.second);
      int64_t q = Mo + svec_index(r.first, r.second);
      s->omega[q] = (1.0 / occ) / (sr * sr);
      s->inv_rep_s[q] = 1.0 / sr;
    }
    // A_mom rows (column-major upper order of the duplicate entry); the star
    // classes of this clique are numbered in order of their first duplicate
    std::unordered_map<Key, int> cls_of;
    std::vector<std::vector<std::pair<int64_t, double>>> per_cls;
    std::vector<std::pair<int64_t, double>> cls_rep;  // (rep position, s_rep^2)
    for (int j = 0; j < nM; ++j)
      for (int i = 0; i <= j; ++i) {
        Key a = key_add(mi.basis[i], mi.basis[j]);
        auto r = mi.rep[a];
        if (r.first == i && r.second == j) continue;
        int64_t qr = mpos(k, a, &sc);
        ent.clear();
        ent.push_back({Mo + svec_index(i, j), svec_scale(i, j)});
        ent.push_back({qr, -sc});
        int64_t row = (int64_t)s->b.size();
        emit(0.0, STROM_ROW_MOM, k);
        auto it = cls_of.find(a);
        if (it == cls_of.end()) {
          it = cls_of.emplace(a, (int)per_cls.size()).first;
          per_cls.emplace_back();
          cls_rep.push_back({qr, sc * sc});
        }
        double sp = svec_scale(i, j);
        per_cls[it->second].push_back({row, 1.0 / (sp * sp)});
      }
    for (size_t c = 0; c < per_cls.size(); ++c) {
      s->star_rep.push_back(cls_rep[c].first);
      s->star_c.push_back(cls_rep[c].second);
      s->star_ptr.push_back((int32_t)s->star_row.size());
      double d = 0.0;
      for (auto& rv : per_cls[c]) {
        s->star_row.push_back(rv.first);
        s->star_inv_s2.push_back(rv.second);
        d += rv.second;
      }
      s->star_d.push_back(d);
    }
    int64_t grp_first = (int64_t)s->b.size();
    // A_ineq rows: L(a,b) - sum_t c_t M(rep(e_t + z^a z^b)) = 0
    for (auto& L : locs[k]) {
      int n = s->block_n[L.blk];
      int64_t Lo = s->block_off[L.blk];
      for (int j = 0; j < n; ++j)
        for (int i = 0; i <= j; ++i) {
          ent.clear();
          ent.push_back({Lo + svec_index(i, j), svec_scale(i, j)});
          Key mab = key_add(L.basis[i], L.basis[j]);
          for (auto& t : L.g) {
            int64_t q = mpos(k, key_add(t.e, mab), &sc);
            ent.push_back({q, -t.c * sc});
          }
          emit(0.0, STROM_ROW_INEQ, k);
          s->omega[Lo + svec_index(i, j)] = 1.0;
        }
    }
    // A_eq rows: ell(h * z^m) = 0 for z^m in [z]_{2 kappa - deg h}
    for (auto& h : cl.h) {
      auto ht = terms_of(h, nv);
      int dh = h.degree(nv);
      if (dh > 2 * kappa) throw std::runtime_error("equality degree exceeds 2 kappa");
      for (auto& mono : monomial_basis(nv, 2 * kappa - dh)) {
        Key mk = key_of(mono.data(), nv);
        ent.clear();
        for (auto& t : ht) {
          int64_t q = mpos(k, key_add(t.e, mk), &sc);
          ent.push_back({q, t.c * sc});
        }
        emit(0.0, STROM_ROW_EQ, k);
      }
    }
    // phi_0 = 1
    ent.clear();
    ent.push_back({Mo + svec_index(0, 0), 1.0});
    emit(1.0, STROM_ROW_PHI0, k);
    // consensus with clique k+1 on the monomials of degree 1..2 kappa of x_k
    int ncons = 0;
    if (k + 1 < N) {
      auto ob = monomial_basis(dx, 2 * kappa);
      for (size_t t = 1; t < ob.size(); ++t) {
        std::vector<uint8_t> ek(nv, 0), ek1(nv, 0);
        for (int i = 0; i < dx; ++i) { ek[nv - dx + i] = ob[t][i]; ek1[i] = ob[t][i]; }
        double s1, s2;
        int64_t q1 = mpos(k, key_of(ek.data(), nv), &s1);
        int64_t q2 = mpos(k + 1, key_of(ek1.data(), nv), &s2);
        ent.clear();
        ent.push_back({q1, s1});
        ent.push_back({q2, -s2});
        emit(0.0, STROM_ROW_CONS, k);
        ++ncons;
      }
    }
    for (int64_t r = grp_first; r < (int64_t)s->b.size(); ++r) s->oth_rows.push_back(r);
    s->grp_ptr.push_back((int32_t)s->oth_rows.size());
    s->grp_cons.push_back(ncons);
  }
  s->star_ptr.push_back((int32_t)s->star_row.size());
  return s;
}

}  // namespace strom
