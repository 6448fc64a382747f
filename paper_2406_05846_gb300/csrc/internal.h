// Internal host-side structures shared by the translation units of libstrom.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/strom.h"

namespace strom {

void set_error(const std::string& msg);
void count_launches(int64_t n);   // bookkeeping behind strom_launch_count()
int64_t thread_launch_count();    // the calling host thread's share of it
void count_h2d(uint64_t bytes);
void count_d2h(uint64_t bytes);

struct Poly {
  std::vector<double> coef;
  std::vector<uint8_t> expo;  // nterms * nv
  int nterms() const { return (int)coef.size(); }
  int degree(int nv) const;
};

struct CliqueData {
  Poly f;
  std::vector<Poly> g, h;
};

struct Problem {
  int N = 0, dx = 0, du = 0, kappa = 2;
  double R = 1.0;
  std::vector<CliqueData> cl;
  int nv() const { return 2 * dx + du; }
  int nz() const { return N * (dx + du) + dx; }
};

struct Sdp {
  int N = 0, nv = 0, dx = 0, du = 0, kappa = 2;
  // blocks
  std::vector<int32_t> block_n, block_clique, block_index;
  std::vector<int64_t> block_off;
  std::vector<int8_t> block_kind;  // 0 = M, 1 = L
  int64_t nsvec = 0;
  std::vector<double> C;
  // rows (CSR, columns sorted)
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<double> b;
  std::vector<int8_t> row_kind;
  std::vector<int32_t> row_clique;
  // structure used by the y-solve (star elimination of the A_mom rows)
  std::vector<double> omega;       // [nsvec] weights of the Schur Gram of the other rows
  std::vector<double> inv_rep_s;   // [nsvec] 1/s_p at representative entries of M blocks, else 0
  std::vector<int64_t> star_rep;   // [nclass] svec position of the representative
  std::vector<double> star_c;      // [nclass] s_rep^2
  std::vector<double> star_d;      // [nclass] sum over its duplicates of 1/s_p^2
  std::vector<int32_t> star_ptr;   // [nclass+1]
  std::vector<int64_t> star_row;   // row id of each duplicate's A_mom row
  std::vector<double> star_inv_s2; // 1/s_p^2 of each duplicate entry
  std::vector<int32_t> grp_ptr;    // [N+1] into oth_rows: rows of clique k other than A_mom
  std::vector<int32_t> grp_cons;   // [N] trailing consensus rows of group k
  std::vector<int64_t> oth_rows;   // global row ids (natural order inside a clique)
  int64_t m() const { return (int64_t)b.size(); }
  int64_t nnz() const { return (int64_t)val.size(); }
};

Sdp* build_relaxation(const Problem& p);  // throws std::runtime_error

// certificate of one instance from the eigen data of its blocks (certify.cpp)
void certify_one(const Problem& p, const std::vector<int32_t>& bn, const std::vector<int8_t>& bk,
                 const std::vector<int32_t>& bc, const int64_t* lo, const double* lamX, const double* topX,
                 const double* lamZ, double by, double rank_tol, double xi_tol, strom_certificate* out,
                 double* zbar_out, double* zhat_out);

std::vector<std::vector<uint8_t>> monomial_basis(int nv, int d);

// warm-start neighbours of key among n stored keys (row-major n x d): fills
// idx / wt (length d + 1) and returns how many are used (warm_select.cpp)
int warm_select(const double* keys, int n, int d, const double* key, int32_t* idx, double* wt);

}  // namespace strom

struct strom_problem { strom::Problem p; };
struct strom_sdp { strom::Sdp* s; };
