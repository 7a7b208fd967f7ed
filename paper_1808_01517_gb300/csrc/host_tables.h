// Host-side FP64 tables of the spherical layers: SH basis, regularised
// pseudo-inverse, LSC kernel geometry, collapse matrices and integer tables.
// Built once per gradient table (Sec. 2.2 and 2.3 constructors); no GPU needed.
#pragma once

#include <string>
#include <vector>

namespace delimit {

int sh_ncoef(int order);                         // (L+1)(L+2)/2 for even L >= 0, else -1
void sh_eval(int order, const double g[3], double* out);  // N real even-order values at unit g

struct ShellHost {
  double bval = 0;
  int m = 0;                 // directions in the shell
  int dir_off = 0;           // first grouped row
  std::vector<int> dir_index;  // original row of each grouped row
  std::vector<double> dirs;  // m x 3
  std::vector<double> B;     // m x N   (B[i,j] = Y_j(g_i))
  std::vector<double> P;     // N x m   ((B^T B + lambda L)^-1 B^T)
};

struct BasisHost {
  int order = 0, N = 0, n_dirs = 0;
  double lambda = 0;
  bool has_pinv = true;
  std::vector<ShellHost> shells;
};

// Returns 0 on success, 1 invalid argument, 2 rank deficient; err gets a message.
// need_pinv = false skips the pseudo-inverse (P is left zero): an evaluation-only basis.
int build_basis(const double* dirs, const double* bvals, int n, int order, double lambda, BasisHost& out,
                std::string& err, bool need_pinv = true);

struct LscShellHost {
  std::vector<double> kpts;       // m x K x 3
  std::vector<double> M;          // K x Nout x Nin; resampling-free form: S_in x K x Nout x Nin
  std::vector<double> q;          // Nout
  std::vector<long long> nb_indptr, nb_indices;  // neighbour CSR
  std::vector<unsigned char> window;             // S_in
  // resampling-free form, per input shell s': acquired neighbours of every direction
  // of this shell among shell s' (CSR, ascending) and the kernel point of each
  std::vector<std::vector<long long>> pair_indptr, pair_indices;
  std::vector<std::vector<int>> pair_bins;
};

struct LscHost {
  int order_in = 0, n_in = 0, n_out = 0, s_in = 0, s_out = 0, K = 0, rings = 0, sectors = 0, window = 0;
  double radius = 0;
  bool neighbours = false;  // resampling-free form (acquired neighbours binned to kernel points)
  std::vector<LscShellHost> shells;
};

// neighbours = false: the resampled LSC of Sec. 2.3, M_{s,k} = P_out,s B^K_{s,k}.
// neighbours = true: the resampling-free form over acquired neighbours, input shell s'
// sampled on the table's shell s' (shells_in must equal the table's shell count),
// M_{s,s',k} = P_out,s A^{s,s'}_k B_in,s' with A_k the mean over the neighbours binned
// to kernel point k.
int build_lsc(const BasisHost& out_basis, int order_in, int shells_in, double radius, int rings, int sectors,
              int window, bool neighbours, LscHost& out, std::string& err);

}  // namespace delimit
