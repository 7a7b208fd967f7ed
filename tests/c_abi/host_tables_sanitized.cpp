// Host FP64 table code (csrc/host_tables.cpp) under AddressSanitizer and
// UndefinedBehaviorSanitizer: builds bases and LSC geometries (both forms) over a range
// of orders, regularisations, windows and kernel shapes, plus the refused inputs, and
// checks sizes and finiteness.  Any out-of-bounds access, use after free, overflow or
// other undefined behaviour aborts the program under the sanitizers.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "host_tables.h"

using namespace delimit;

namespace {

int g_fail = 0;

void expect(bool ok, const char* what) {
  if (!ok) {
    std::printf("FAILED: %s\n", what);
    ++g_fail;
  }
}

// n directions on the upper hemisphere (golden-angle spiral), unit length
std::vector<double> spiral(int n, double twist) {
  std::vector<double> d(3 * n);
  const double ga = M_PI * (3.0 - std::sqrt(5.0));
  for (int i = 0; i < n; ++i) {
    const double z = 1.0 - (i + 0.5) / n;  // (0, 1]
    const double r = std::sqrt(1.0 - z * z);
    const double ph = ga * i + twist;
    d[3 * i] = r * std::cos(ph);
    d[3 * i + 1] = r * std::sin(ph);
    d[3 * i + 2] = z;
  }
  return d;
}

struct Table {
  std::vector<double> dirs, bvals;
};

Table table(const std::vector<int>& m, const std::vector<double>& b) {
  Table t;
  for (size_t s = 0; s < m.size(); ++s) {
    const std::vector<double> d = spiral(m[s], 0.37 * (double)s);
    t.dirs.insert(t.dirs.end(), d.begin(), d.end());
    t.bvals.insert(t.bvals.end(), (size_t)m[s], b[s]);
  }
  return t;
}

bool all_finite(const std::vector<double>& v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

void check_basis(const BasisHost& B, int n_shells, int order) {
  expect((int)B.shells.size() == n_shells, "shell count");
  expect(B.N == sh_ncoef(order), "coefficient count");
  for (const ShellHost& s : B.shells) {
    expect((int)s.B.size() == s.m * B.N && (int)s.P.size() == s.m * B.N, "basis sizes");
    expect(all_finite(s.B) && all_finite(s.P), "basis finite");
  }
}

void check_lsc(const LscHost& L, const BasisHost& out, int s_in) {
  expect(L.shells.size() == out.shells.size(), "lsc shell count");
  for (size_t s = 0; s < L.shells.size(); ++s) {
    const LscShellHost& h = L.shells[s];
    const int m = out.shells[s].m;
    expect((int)h.kpts.size() == m * L.K * 3, "kernel point count");
    const size_t per = (size_t)L.K * L.n_out * L.n_in;
    expect(h.M.size() == (L.neighbours ? per * s_in : per), "collapse matrix size");
    expect((int)h.q.size() == L.n_out, "bias projection size");
    expect(all_finite(h.kpts) && all_finite(h.M) && all_finite(h.q), "lsc finite");
    expect((int)h.nb_indptr.size() == m + 1, "neighbour indptr size");
    expect(h.nb_indptr.back() == (long long)h.nb_indices.size(), "neighbour indptr end");
    if (L.neighbours) {
      expect((int)h.pair_indptr.size() == s_in, "pair tables");
      for (int p = 0; p < s_in; ++p) {
        expect(h.pair_indptr[p].back() == (long long)h.pair_indices[p].size(), "pair indptr end");
        expect(h.pair_bins[p].size() == h.pair_indices[p].size(), "pair bins size");
        for (int k : h.pair_bins[p]) expect(k >= 0 && k < L.K, "bin in range");
      }
    }
  }
}

}  // namespace

int main() {
  const Table t3 = table({30, 40, 50}, {1000.0, 2000.0, 3000.0});
  const int n3 = (int)t3.bvals.size();
  for (int order : {0, 2, 4, 8}) {
    for (double lam : {0.0, 0.006}) {
      BasisHost B;
      std::string err;
      const int rc = build_basis(t3.dirs.data(), t3.bvals.data(), n3, order, lam, B, err);
      // the 30-direction shell cannot fit 45 order-8 coefficients without regularisation
      const bool deficient = lam == 0.0 && sh_ncoef(order) > 30;
      expect(rc == (deficient ? 2 : 0), "basis builds, or reports rank deficiency");
      if (rc) continue;
      check_basis(B, 3, order);
      for (int window : {0, 1, -1}) {
        for (bool nb : {false, true}) {
          for (int order_in : {0, order}) {
            const int rings = order == 8 ? 4 : 1, sectors = order == 8 ? 12 : 1;
            LscHost L;
            const int rc2 = build_lsc(B, order_in, 3, 0.44, rings, sectors, window, nb, L, err);
            expect(rc2 == 0, "lsc builds");
            if (rc2 == 0) check_lsc(L, B, 3);
          }
        }
      }
      // all-shell mixing from fewer input shells (resampled form only)
      LscHost L2;
      expect(build_lsc(B, 2, 2, M_PI / 2, 2, 6, -1, false, L2, err) == 0, "all-shell mixing");
      if (L2.shells.size()) check_lsc(L2, B, 2);
    }
  }
  // evaluation-only basis (no pseudo-inverse)
  {
    BasisHost B;
    std::string err;
    expect(build_basis(t3.dirs.data(), t3.bvals.data(), n3, 8, 0.0, B, err, false) == 0, "eval-only basis");
  }
  // refused inputs: odd order, a b = 0 row, a non-unit direction, rank deficiency,
  // a bad radius or kernel, mismatched shell counts for the resampling-free form
  {
    BasisHost B;
    std::string err;
    expect(build_basis(t3.dirs.data(), t3.bvals.data(), n3, 3, 0.0, B, err) == 1, "odd order refused");
    Table bad = t3;
    bad.bvals[5] = 0.0;
    expect(build_basis(bad.dirs.data(), bad.bvals.data(), n3, 4, 0.0, B, err) == 1, "b = 0 refused");
    bad = t3;
    bad.dirs[7] *= 1.01;
    expect(build_basis(bad.dirs.data(), bad.bvals.data(), n3, 4, 0.0, B, err) == 1, "non-unit refused");
    const Table few = table({10}, {1000.0});
    expect(build_basis(few.dirs.data(), few.bvals.data(), 10, 4, 0.0, B, err) == 2, "rank deficiency reported");
    BasisHost ok;
    expect(build_basis(t3.dirs.data(), t3.bvals.data(), n3, 4, 0.006, ok, err) == 0, "basis for lsc errors");
    LscHost L;
    expect(build_lsc(ok, 4, 3, 0.0, 2, 6, 0, false, L, err) == 1, "zero radius refused");
    expect(build_lsc(ok, 4, 3, 2.0, 2, 6, 0, false, L, err) == 1, "radius past pi/2 refused");
    expect(build_lsc(ok, 4, 3, 0.4, 0, 6, 0, false, L, err) == 1, "no rings refused");
    expect(build_lsc(ok, 3, 3, 0.4, 2, 6, 0, false, L, err) == 1, "odd input order refused");
    expect(build_lsc(ok, 4, 2, 0.4, 2, 6, -1, true, L, err) == 1, "resampling-free shell mismatch refused");
  }
  if (g_fail) {
    std::printf("%d checks failed\n", g_fail);
    return 1;
  }
  std::printf("host tables ok\n");
  return 0;
}
